"""Python binding of libbie.so (the B300 surface-BIE library).

Argument marshalling only: every step of the method runs in the CUDA library.
Device memory and streams come from PyTorch.  There is no CPU path: importing
this package without the built library raises.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbie.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError("libbie.so is not built; run python paper_2608_16208_b300/build.py "
                      "(there is no CPU fallback)")
lib = ctypes.CDLL(_LIB_PATH)

KERNEL_S, KERNEL_K = 1, 2
OP_S, OP_K, OP_K_PLUS_I, OP_K_MINUS_I, OP_CFIE = 0, 1, 2, 3, 4
UNWEIGHTED = 0x100
MAX_TERMS = 96

_vp, _i64, _i32, _d, _u = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint


class SurfaceDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_terms", ctypes.c_int), ("axes", ctypes.c_double * 3),
                ("terms", ctypes.POINTER(ctypes.c_double))]


class QuadTables(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double * (3 * 16 * 16)), ("w", ctypes.c_double * (3 * 16 * 16)),
                ("gl_x", ctypes.c_double * 16), ("gl_w", ctypes.c_double * 16)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("prec", ctypes.c_int), ("precond", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("bie_last_error", ctypes.c_char_p, [])
_sig("bie_ctx_create", _i32, [ctypes.POINTER(_vp), _vp])
_sig("bie_ctx_free", None, [_vp])
_sig("bie_ctx_sync", _i32, [_vp])
_sig("bie_surface_sample", _i32, [_vp, ctypes.POINTER(SurfaceDesc), _i32, _i32, ctypes.POINTER(QuadTables),
                                  ctypes.POINTER(_vp)])
_sig("bie_surface_free", None, [_vp])
_sig("bie_surface_unknowns", _i64, [_vp])
_sig("bie_surface_near_pairs", _i64, [_vp])
_sig("bie_surface_points", _vp, [_vp])
_sig("bie_surface_normals", _vp, [_vp])
_sig("bie_surface_jacobians", _vp, [_vp])
_sig("bie_kernel_modes", _i32, [_vp, _vp, _u, _d, _vp, _vp, _i64, _vp])
_sig("bie_kernel_modes_noalloc", _i32, [_vp, _vp, _u, _d, _vp, _vp, _i64, _vp])


class BieError(RuntimeError):
    pass


def check(status, what):
    if status != 0:
        raise BieError("%s failed (status %d): %s" % (what, status, lib.bie_last_error().decode()))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A library context bound to the current device and PyTorch's current stream."""

    def __init__(self, stream=None):
        stream = stream or torch.cuda.current_stream()
        self.stream = stream
        self.h = _vp()
        check(lib.bie_ctx_create(ctypes.byref(self.h), _vp(stream.cuda_stream)), "bie_ctx_create")

    def sync(self):
        check(lib.bie_ctx_sync(self.h), "bie_ctx_sync")

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_ctx_free(self.h)
            self.h = None


class Surface:
    """A sampled surface (library-owned device data)."""

    def __init__(self, ctx, desc, Np, Mt, ggq):
        self.ctx, self.Np, self.Mt = ctx, Np, Mt
        d = SurfaceDesc()
        d.kind = 0 if desc["kind"] == "ellipsoid" else 1
        if d.kind == 0:
            d.axes[:] = list(desc["axes"])
            d.n_terms = 0
            self._terms = None
        else:
            terms = np.ascontiguousarray(np.asarray(desc["terms"], dtype=np.float64).reshape(-1, 5))
            d.n_terms = len(terms)
            self._terms = terms
            d.terms = terms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        q = QuadTables()
        gx, gw = ggq[0], ggq[1]
        q.x[:] = np.ascontiguousarray(gx, dtype=np.float64).ravel().tolist()
        q.w[:] = np.ascontiguousarray(gw, dtype=np.float64).ravel().tolist()
        glx, glw = (ggq[2], ggq[3]) if len(ggq) > 2 else np.polynomial.legendre.leggauss(16)
        q.gl_x[:] = [float(v) for v in glx]
        q.gl_w[:] = [float(v) for v in glw]
        self.h = _vp()
        check(lib.bie_surface_sample(ctx.h, ctypes.byref(d), Np, Mt, ctypes.byref(q), ctypes.byref(self.h)),
              "bie_surface_sample")
        self.N = lib.bie_surface_unknowns(self.h)
        self.near_pairs = lib.bie_surface_near_pairs(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_surface_free(self.h)
            self.h = None


def kernel_modes(surface, kernels, k, rows, srcs, out=None):
    """Kernel modes K_m, m = -M..M, per pair: complex128 tensor [n, nk, Mt+1]."""
    n = rows.numel()
    nk = bin(kernels).count("1")
    if out is None:
        out = torch.empty((n, nk, surface.Mt + 1), dtype=torch.complex128, device="cuda")
    check(lib.bie_kernel_modes(surface.ctx.h, surface.h, kernels, float(k), _ptr(rows), _ptr(srcs), n,
                               _ptr(out)), "bie_kernel_modes")
    return out


_sig("bie_assemble", _i32, [_vp, _vp, _i32, _d, _d, _vp])
_sig("bie_assemble_near", _i32, [_vp, _vp, _u, _d, _d, _d, _d, _d, _vp])
_sig("bie_solve", _i32, [_vp, _i64, _vp, _vp, _i32, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)])
_sig("bie_rhs", _i32, [_vp, _vp, _i32, ctypes.POINTER(ctypes.c_double), _d, _vp])
_sig("bie_field_eval", _i32, [_vp, _vp, _i32, _d, _d, _vp, _vp, _i64, _i32, _vp])


def assemble(surface, op, k, eta=None, out=None):
    """Dense operator matrix [N, N] complex128 (row = target)."""
    N = surface.N
    if out is None:
        out = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    check(lib.bie_assemble(surface.ctx.h, surface.h, op, float(k), float(k if eta is None else eta), _ptr(out)),
          "bie_assemble")
    return out


def assemble_near(surface, kernels, k, A, ws=1.0, wk=0.0):
    """Add ws * (near blocks of S) + wk * (near blocks of K) to A (correction stage)."""
    ws, wk = complex(ws), complex(wk)
    check(lib.bie_assemble_near(surface.ctx.h, surface.h, kernels, float(k), ws.real, ws.imag, wk.real, wk.imag,
                                _ptr(A)), "bie_assemble_near")
    return A


def solve(ctx, A, b, x=None, tol=1e-8, restart=100, maxit=2000, prec=0):
    """FGMRES solve of A x = b (b: [N] or [nrhs, N]); returns (x, report dict)."""
    n = A.shape[0]
    bb = b.reshape(-1, n).contiguous()
    nrhs = bb.shape[0]
    if x is None:
        x = torch.zeros_like(bb)
    o = SolveOpts(tol, restart, maxit, prec, 0)
    r = SolveReport()
    st = lib.bie_solve(ctx.h, n, _ptr(A), _ptr(bb), nrhs, _ptr(x), ctypes.byref(o), ctypes.byref(r))
    rep = {"iterations": r.iterations, "refinements": r.refinements, "rel_residual": r.rel_residual,
           "seconds": r.seconds, "status": st}
    check(st, "bie_solve")
    return x.reshape(b.shape), rep


def rhs(surface, kind, param, k, out=None):
    """Boundary data: kind 0 plane wave -e^{ik d.x} (param = d), kind 1 point source (param = source)."""
    if out is None:
        out = torch.empty(surface.N, dtype=torch.complex128, device="cuda")
    p = (ctypes.c_double * 3)(*[float(v) for v in param])
    check(lib.bie_rhs(surface.ctx.h, surface.h, kind, p, float(k), _ptr(out)), "bie_rhs")
    return out


def field_eval(surface, rep, k, density, points, far_field=False, eta=None):
    """u(x) at points [n, 3] (or the far-field pattern in directions [n, 3])."""
    pts = torch.as_tensor(points, dtype=torch.float64).reshape(-1, 3).contiguous().cuda()
    out = torch.empty(pts.shape[0], dtype=torch.complex128, device="cuda")
    check(lib.bie_field_eval(surface.ctx.h, surface.h, rep, float(k), float(k if eta is None else eta),
                             _ptr(density), _ptr(pts), pts.shape[0], 1 if far_field else 0, _ptr(out)),
          "bie_field_eval")
    return out


_sig("bie_batch_create", _i32, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_double), _u, _vp, _i64,
                                ctypes.POINTER(_vp)])
_sig("bie_batch_run", _i32, [_vp])
_sig("bie_batch_pairs", _i64, [_vp])
_sig("bie_batch_offset", _i64, [_vp, _i32])
_sig("bie_batch_config", None, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)])
_sig("bie_batch_free", None, [_vp])


class Batch:
    """A device-resident plan running the pair pipeline of many surfaces in one persistent launch."""

    def __init__(self, ctx, surfaces, ks, kernels, weights, slot_pairs):
        self.ctx, self.surfaces, self.weights = ctx, list(surfaces), weights
        hs = (_vp * len(surfaces))(*[s.h for s in surfaces])
        kk = (ctypes.c_double * len(surfaces))(*[float(k) for k in ks])
        self.h = _vp()
        check(lib.bie_batch_create(ctx.h, len(surfaces), hs, kk, kernels, _ptr(weights), int(slot_pairs),
                                   ctypes.byref(self.h)), "bie_batch_create")
        self.pairs = lib.bie_batch_pairs(self.h)
        self.offsets = [lib.bie_batch_offset(self.h, i) for i in range(len(surfaces))]
        a, b, c = _i32(), _i32(), _i32()
        lib.bie_batch_config(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        self.config = {"item_pairs": a.value, "warps_per_block": b.value, "blocks": c.value}

    def run(self):
        check(lib.bie_batch_run(self.h), "bie_batch_run")

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_batch_free(self.h)
            self.h = None
