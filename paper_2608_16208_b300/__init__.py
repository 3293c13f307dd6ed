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

KERNEL_S, KERNEL_K, KERNEL_KP = 1, 2, 4
OP_S, OP_K, OP_K_PLUS_I, OP_K_MINUS_I, OP_CFIE, OP_KP, OP_KP_PLUS_I, OP_KP_MINUS_I = 0, 1, 2, 3, 4, 5, 6, 7
RHS_PLANE_WAVE, RHS_POINT_SOURCE, RHS_POINT_SOURCE_NORMAL_DERIVATIVE = 0, 1, 2
_KINDS = {"ellipsoid": 0, "star": 1, "bean": 2, "torus": 3, "fourier_torus": 4}
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
                ("prec", ctypes.c_int), ("precond", ctypes.c_int), ("block", ctypes.c_void_p),
                ("net", ctypes.c_void_p), ("surface", ctypes.c_void_p), ("k", ctypes.c_double)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("fallback_used", ctypes.c_int), ("matvecs", ctypes.c_int)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


NET_PARAMS = 20258
PRECOND_NONE, PRECOND_BLOCK, PRECOND_LEARNED = 0, 1, 2


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("bie_last_error", ctypes.c_char_p, [])
_sig("bie_ctx_create", _i32, [ctypes.POINTER(_vp), _vp])
_sig("bie_ctx_free", None, [_vp])
_sig("bie_ctx_sync", _i32, [_vp])
_sig("bie_ctx_trace", _i32, [_vp, _i32])
_sig("bie_ctx_set_option", _i32, [_vp, _i32, _i32])
OPT_FP64_TRANSFORMS = 1
_sig("bie_ctx_trace_read", _i32, [_vp, _vp, _vp])
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
_sig("bie_rho_inv_modes", _i32, [_vp, _vp, _vp, _vp, _vp, _i64, _i32, _d, _vp, _vp])
_sig("bie_kernel_modes_banded", _i32, [_vp, _vp, _d, _vp, _vp, _i64, _d, _vp])


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

    def set_option(self, option, value):
        check(lib.bie_ctx_set_option(self.h, int(option), int(value)), "bie_ctx_set_option")

    def trace(self, enable=True):
        """Record CUDA events around the pair, near-fill and far-fill launches of this context."""
        check(lib.bie_ctx_trace(self.h, 1 if enable else 0), "bie_ctx_trace")

    def trace_read(self):
        """{family: (ms, launches)} of the launches recorded since the trace was switched on or last read."""
        ms = (ctypes.c_double * 5)()
        n = (ctypes.c_int * 5)()
        check(lib.bie_ctx_trace_read(self.h, ms, n), "bie_ctx_trace_read")
        names = ("pair_root", "pair_transform", "pair_fused", "near_fill", "far_fill")
        return {names[i]: (ms[i], n[i]) for i in range(5)}

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_ctx_free(self.h)
            self.h = None


class Surface:
    """A sampled surface (library-owned device data)."""

    def __init__(self, ctx, desc, Np, Mt, ggq):
        self.ctx, self.Np, self.Mt = ctx, Np, Mt
        d = SurfaceDesc()
        d.kind = _KINDS[desc["kind"]]
        terms = None
        if d.kind == 0:
            d.axes[:] = list(desc["axes"])
        elif d.kind == 1:
            terms = np.asarray(desc["terms"], dtype=np.float64).reshape(-1, 5)
        elif d.kind == 3:   # torus: axes (a, b, c), one term (R, eps, m)
            d.axes[:] = [desc["a"], desc["b"], desc["c"]]
            terms = np.array([[desc["R"], desc["eps"], desc["m"], 0.0, 0.0]])
        elif d.kind == 4:   # Fourier torus: axes[0] = R, terms (c, m, n)
            d.axes[:] = [desc["R"], 0.0, 0.0]
            tt = np.asarray(desc["terms"], dtype=np.float64).reshape(-1, 3)
            terms = np.concatenate([tt, np.zeros((len(tt), 2))], axis=1)
        self._terms = None
        d.n_terms = 0
        if terms is not None:
            self._terms = np.ascontiguousarray(terms)
            d.n_terms = len(terms)
            d.terms = self._terms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
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

    def _copy(self, ptr, shape):
        """Copy of a library-owned device array of doubles (the view goes through the CUDA array interface)."""
        view = type("_DeviceDoubles", (), {})()
        view.__cuda_array_interface__ = {"shape": shape, "typestr": "<f8", "data": (ptr, False), "version": 2}
        return torch.as_tensor(view, device="cuda").clone()

    def points(self):
        """Node positions [N, 3]."""
        return self._copy(lib.bie_surface_points(self.h), (self.N, 3))

    def normals(self):
        """Unit normals [N, 3]."""
        return self._copy(lib.bie_surface_normals(self.h), (self.N, 3))

    def jacobians(self):
        """Surface Jacobians J = |r_t x r_theta| [N]."""
        return self._copy(lib.bie_surface_jacobians(self.h), (self.N,))

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


def rho_inv_modes(surface, t, th, ts, lmax, eps0=1e-14):
    """O(M) route: <rho^{-1}>_l, l = 0..lmax, of the queries (t, th, ts) (float64 CUDA tensors):
    complex128 tensor [n, lmax+1] and the int32 m0 of each query."""
    t, th, ts = (torch.as_tensor(v, dtype=torch.float64, device="cuda").contiguous() for v in (t, th, ts))
    n = t.numel()
    out = torch.empty((n, lmax + 1), dtype=torch.complex128, device="cuda")
    m0 = torch.zeros(n, dtype=torch.int32, device="cuda")
    check(lib.bie_rho_inv_modes(surface.ctx.h, surface.h, _ptr(t), _ptr(th), _ptr(ts), n, int(lmax), float(eps0),
                                _ptr(out), _ptr(m0)), "bie_rho_inv_modes")
    return out, m0


def kernel_modes_banded(surface, k, rows, srcs, eps0=1e-14, out=None):
    """Single-layer modes K_m, m = -M..M, per pair through the O(M) route: complex128 [n, Mt+1]."""
    n = rows.numel()
    if out is None:
        out = torch.empty((n, surface.Mt + 1), dtype=torch.complex128, device="cuda")
    check(lib.bie_kernel_modes_banded(surface.ctx.h, surface.h, float(k), _ptr(rows), _ptr(srcs), n, float(eps0),
                                      _ptr(out)), "bie_kernel_modes_banded")
    return out


_sig("bie_assemble", _i32, [_vp, _vp, _i32, _d, _d, _vp])
_sig("bie_assemble_near", _i32, [_vp, _vp, _u, _d, _d, _d, _d, _d, _vp])
_sig("bie_assemble_near_band", _i32, [_vp, _vp, _u, _d, _d, _d, _d, _d, _vp])
_sig("bie_solve", _i32, [_vp, _i64, _vp, _vp, _i32, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)])
_sig("bie_solve_matrix", _i32, [_vp, _vp, _vp, _i32, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)])
_sig("bie_matrix_create", _i32, [_vp, _i64, _vp, _u, ctypes.POINTER(_vp)])
_sig("bie_matrix_free", None, [_vp])
_sig("bie_matrix_size", _i64, [_vp])
_sig("bie_matrix_matvec", _i32, [_vp, _i32, _vp, _i32, _vp])
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


def assemble_near_band(surface, kernels, k, out=None, ws=1.0, wk=0.0, host=False):
    """Near band of ws * S + wk * K: complex128 [N, 3, 16 Mt] (slot d = source panel - target panel + 1).

    out: a device tensor, or a page-locked host tensor (host=True allocates one); with host memory the
    copies of finished panel groups overlap the pair kernels of the next.  Complete after ctx.sync()."""
    ws, wk = complex(ws), complex(wk)
    shape = (surface.N, 3, 16 * surface.Mt)
    if out is None:
        out = (torch.empty(shape, dtype=torch.complex128, pin_memory=True) if host
               else torch.empty(shape, dtype=torch.complex128, device="cuda"))
    if tuple(out.shape) != shape or out.dtype != torch.complex128 or not out.is_contiguous():
        raise ValueError("out must be a contiguous complex128 tensor of shape %s" % (shape,))
    check(lib.bie_assemble_near_band(surface.ctx.h, surface.h, kernels, float(k), ws.real, ws.imag, wk.real,
                                     wk.imag, _ptr(out)), "bie_assemble_near_band")
    return out


STORE_FP32, STORE_BF16X2 = 1, 2
PREC_FP64, PREC_FP32, PREC_BF16X2, PREC_DW = 0, 1, 2, 3


def _solve_call(fn, ctx, target, n, b, x, tol, restart, maxit, prec, precond, block, net, surface, k,
                raise_on_noconv):
    bb = b.reshape(-1, n).contiguous()
    nrhs = bb.shape[0]
    if x is None:
        x = torch.zeros_like(bb)
    o = SolveOpts(tol, restart, maxit, prec, precond, block.h if block is not None else None,
                  net.h if net is not None else None, surface.h if surface is not None else None, float(k))
    r = SolveReport()
    st = fn(ctx.h, *target, _ptr(bb), nrhs, _ptr(x), ctypes.byref(o), ctypes.byref(r))
    rep = {"iterations": r.iterations, "refinements": r.refinements, "rel_residual": r.rel_residual,
           "seconds": r.seconds, "fallback_used": r.fallback_used, "matvecs": r.matvecs, "status": st}
    if st != 4 or raise_on_noconv:   # 4 = BIE_ENOCONV: the report still holds the iterations and residual
        check(st, "bie_solve")
    return x.reshape(b.shape), rep


def solve(ctx, A, b, x=None, tol=1e-8, restart=100, maxit=2000, prec=0, precond=0, block=None, net=None,
          surface=None, k=0.0, raise_on_noconv=True):
    """FGMRES solve of A x = b (b: [N] or [nrhs, N], right-hand sides in lockstep); returns (x, report).

    prec: 0 FP64, 1 FP32 storage + FP64-accurate refinement, 2 split-BF16 tensor-core products +
    refinement.  precond: 0 none, 1 block-diagonal (block), 2 learned (net on the grid of surface,
    wavenumber k, on top of block if given; falls back to block when it does not converge)."""
    n = A.shape[0]
    return _solve_call(lib.bie_solve, ctx, (n, _ptr(A)), n, b, x, tol, restart, maxit, prec, precond, block, net,
                       surface, k, raise_on_noconv)


class Matrix:
    """An FP64 system matrix (kept by the caller) with the low-precision copies the mixed solves read."""

    def __init__(self, ctx, A, store=0):
        self.ctx, self.A, self.n = ctx, A, A.shape[0]
        self.h = _vp()
        check(lib.bie_matrix_create(ctx.h, self.n, _ptr(A), int(store), ctypes.byref(self.h)), "bie_matrix_create")

    def matvec(self, x, prec=PREC_FP64, out=None):
        """y = A x for x [n] or [nr, n] (nr <= 16)."""
        xx = x.reshape(-1, self.n).contiguous()
        y = torch.empty_like(xx) if out is None else out
        check(lib.bie_matrix_matvec(self.h, int(prec), _ptr(xx), xx.shape[0], _ptr(y)), "bie_matrix_matvec")
        return y.reshape(x.shape)

    def solve(self, b, x=None, tol=1e-8, restart=100, maxit=2000, prec=0, precond=0, block=None, net=None,
              surface=None, k=0.0, raise_on_noconv=True):
        return _solve_call(lib.bie_solve_matrix, self.ctx, (self.h,), self.n, b, x, tol, restart, maxit, prec,
                           precond, block, net, surface, k, raise_on_noconv)

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_matrix_free(self.h)
            self.h = None


_sig("bie_blockdiag_create", _i32, [_vp, _i64, _vp, _i32, ctypes.POINTER(_vp)])
_sig("bie_blockdiag_apply", _i32, [_vp, _vp, _i32, _vp])
_sig("bie_blockdiag_size", _i64, [_vp])
_sig("bie_blockdiag_free", None, [_vp])
_sig("bie_net_create", _i32, [_vp, _vp, ctypes.c_uint64, ctypes.POINTER(_vp)])
_sig("bie_net_get_params", _i32, [_vp, _vp])
_sig("bie_net_free", None, [_vp])
_sig("bie_net_forward", _i32, [_vp, _i32, _i32, _i32, _vp, _vp])
_sig("bie_net_backward", _i32, [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp])
_sig("bie_train_set_create", _i32, [_vp, _vp, _d, _vp, _vp, ctypes.POINTER(_vp)])
_sig("bie_train_set_free", None, [_vp])
_sig("bie_net_loss_grad", _i32, [_vp, _vp, _vp, _i32, _vp, ctypes.POINTER(ctypes.c_float)])
_sig("bie_net_train", _i32, [_vp, ctypes.POINTER(_vp), _i32, ctypes.POINTER(TrainOpts), _vp])
_sig("bie_net_precond_apply", _i32, [_vp, _vp, _vp, _d, _vp, _i32, _vp])


class BlockDiag:
    """LU factors (FP32 complex, partial pivoting) of the diagonal blocks of A."""

    def __init__(self, ctx, A, block):
        self.ctx = ctx
        self.h = _vp()
        check(lib.bie_blockdiag_create(ctx.h, A.shape[0], _ptr(A), int(block), ctypes.byref(self.h)),
              "bie_blockdiag_create")

    def apply(self, r, out=None):
        rr = r.reshape(-1, r.shape[-1]).contiguous()
        z = torch.empty_like(rr) if out is None else out
        check(lib.bie_blockdiag_apply(self.h, _ptr(rr), rr.shape[0], _ptr(z)), "bie_blockdiag_apply")
        return z.reshape(r.shape)

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_blockdiag_free(self.h)
            self.h = None


class Net:
    """The learned preconditioner's network (4 convolutional layers, width 32)."""

    def __init__(self, ctx, params=None, seed=0):
        self.ctx = ctx
        self.h = _vp()
        hp = None
        if params is not None:
            self._init = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
            hp = self._init.ctypes.data_as(_vp)
        check(lib.bie_net_create(ctx.h, hp, int(seed), ctypes.byref(self.h)), "bie_net_create")

    def params(self):
        out = np.empty(NET_PARAMS, dtype=np.float32)
        check(lib.bie_net_get_params(self.h, out.ctypes.data_as(_vp)), "bie_net_get_params")
        return out

    def forward(self, x):
        B, _, nt, mt = x.shape
        x = x.contiguous()
        y = torch.empty((B, 2, nt, mt), dtype=torch.float32, device=x.device)
        check(lib.bie_net_forward(self.h, B, nt, mt, _ptr(x), _ptr(y)), "bie_net_forward")
        return y

    def backward(self, x, gy, want_gx=True):
        B, _, nt, mt = x.shape
        x, gy = x.contiguous(), gy.contiguous()
        gp = torch.empty(NET_PARAMS, dtype=torch.float32, device=x.device)
        gx = torch.empty_like(x) if want_gx else None
        check(lib.bie_net_backward(self.h, B, nt, mt, _ptr(x), _ptr(gy), _ptr(gp),
                                   _ptr(gx) if gx is not None else None), "bie_net_backward")
        return gp, gx

    def loss_grad(self, tset, r):
        """Training loss of residuals r (complex64 [nv, N]) and its parameter gradient."""
        r = r.contiguous()
        gp = torch.empty(NET_PARAMS, dtype=torch.float32, device=r.device)
        loss = ctypes.c_float()
        check(lib.bie_net_loss_grad(self.h, tset.h, _ptr(r), r.shape[0], _ptr(gp), ctypes.byref(loss)),
              "bie_net_loss_grad")
        return float(loss.value), gp

    def train(self, sets, steps, batch=16, lr=1e-3, seed=0, beta1=0.9, beta2=0.999, eps=1e-8):
        hs = (_vp * len(sets))(*[t.h for t in sets])
        o = TrainOpts(int(steps), int(batch), float(lr), float(beta1), float(beta2), float(eps), int(seed))
        hist = np.empty(int(steps), dtype=np.float32)
        check(lib.bie_net_train(self.h, hs, len(sets), ctypes.byref(o), hist.ctypes.data_as(_vp)), "bie_net_train")
        return hist

    def precond_apply(self, surface, k, v, block=None):
        vv = v.reshape(-1, v.shape[-1]).contiguous()
        z = torch.empty_like(vv)
        check(lib.bie_net_precond_apply(self.h, block.h if block is not None else None, surface.h, float(k),
                                        _ptr(vv), vv.shape[0], _ptr(z)), "bie_net_precond_apply")
        return z.reshape(v.shape)

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_net_free(self.h)
            self.h = None


class TrainSet:
    """A training system for the network: surface grid, k, FP32 copy of A, block preconditioner."""

    def __init__(self, ctx, surface, k, A, block=None):
        self.ctx, self.surface, self.block = ctx, surface, block
        self.h = _vp()
        check(lib.bie_train_set_create(ctx.h, surface.h, float(k), _ptr(A), block.h if block is not None else None,
                                       ctypes.byref(self.h)), "bie_train_set_create")

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_train_set_free(self.h)
            self.h = None


def rhs(surface, kind, param, k, out=None):
    """Boundary data: kind 0 plane wave -e^{ik d.x} (param = d), kind 1 point source G(x; src), kind 2 its
    normal derivative dG/dnu(x) (param = source; the Neumann data)."""
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
_sig("bie_batch_launches", _i32, [_vp])
_sig("bie_batch_set_fill", _i32, [_vp, _vp, _i32])
_sig("bie_shard_surfaces", _i32, [_i32, _vp, _i32, _vp, _vp])


def shard_surfaces(costs, world):
    """Owner rank of each surface (greedy longest-processing-time over world ranks) and the ranks' loads."""
    c = np.ascontiguousarray(np.asarray(costs, dtype=np.float64))
    owner = np.empty(len(c), dtype=np.int32)
    load = np.empty(world, dtype=np.float64)
    check(lib.bie_shard_surfaces(len(c), c.ctypes.data_as(_vp), int(world), owner.ctypes.data_as(_vp),
                                 load.ctypes.data_as(_vp)), "bie_shard_surfaces")
    return owner, load


class Batch:
    """A device-resident plan running the pair pipeline of many surfaces in a few launches (one class of
    equal grid size after another: chunks through the root and transform kernels for the single layer,
    one persistent launch per class with a double layer)."""

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
        self.config = {"item_pairs": a.value, "warps_per_block": b.value, "blocks": c.value,
                       "launches": lib.bie_batch_launches(self.h)}

    def set_fill(self, band, slots):
        """GGQ fill into a ring of `slots` near-band slots (band: complex128 [slots, 16 maxMt, 3, 16 maxMt]),
        or off with band=None."""
        self.band = band
        check(lib.bie_batch_set_fill(self.h, None if band is None else _ptr(band), int(slots)), "bie_batch_set_fill")
        a, b, c = _i32(), _i32(), _i32()
        lib.bie_batch_config(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        self.config = {"item_pairs": a.value, "warps_per_block": b.value, "blocks": c.value,
                       "launches": lib.bie_batch_launches(self.h)}

    def run(self):
        check(lib.bie_batch_run(self.h), "bie_batch_run")

    def __del__(self):
        if getattr(self, "h", None):
            lib.bie_batch_free(self.h)
            self.h = None
