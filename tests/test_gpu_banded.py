"""The O(M) route on the GPU (Section 3.3, "An O(M) approach"): <rho^{-1}>_l from the banded system
Eq. (Axb) against their plain definition (the refined trapezoid rule; m0 against the oracle's
rho_inv_modes_banded), and the single-layer modes of Eq. (Sphi:appr2)
built on it against the oracle's method_modes_banded (the same route: the same truncation of the
smooth factors).  Per query, normwise: <= 1e-12, and for <rho^{-1}>_l at large lmax the route's
own rounding bound (route_tol); m0 (Eq. (crt:M0)) identical.  The two GPU routes to
the single layer (this one and singularity swapping) agree where the grid resolves the smooth
factors."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import kernel_modes as km
from tests.pairs import pair_geometry, sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def route_tol(lmax):
    """Error bound of the O(M) route against the definition: the route sees rho^2 only through its
    modes, and the banded system amplifies their rounding with the number of modes and with the
    closeness of the pair.  The oracle's own FP64 rendering of the route (numpy, LU of the whole
    band matrix, boundary values from the definition) has, over lmax = 64, 256, 1024 and
    separations 0.05 .. 5e-4 on the ellipsoid and the bumpy star, errors below 0.15 eps lmax^2
    (eps = 2^-52); the bound takes eps lmax^2 / 4, and 1e-12 where that is smaller."""
    return max(TOL, 2.0 ** -52 * lmax * lmax / 4)


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


@pytest.fixture(scope="module")
def ctx(bie):
    return bie.Context()


def _queries(seed, n, dts):
    rs = wl.Stream(seed, 31)
    t = 0.2 + 2.7 * rs.uniform(n)
    th = 2 * np.pi * rs.uniform(n)
    dt = np.array([dts[i % len(dts)] for i in range(n)]) * np.where(rs.uniform(n) < 0.5, -1.0, 1.0)
    return t, th, np.clip(t + dt, 1e-3, np.pi - 1e-3)


SURFACES = [("ellipsoid", wl.ellipsoid(1.0, 0.8, 0.6), 2), ("bumpy", wl.bumpy(), 10),
            ("star", wl.harmonic_star(3, 0, 0.15), None), ("bean", wl.bean(), 2),
            ("wiggly_torus", wl.wiggly_torus(), 2)]


@pytest.mark.parametrize("name,surface,m0", SURFACES, ids=[s[0] for s in SURFACES])
@pytest.mark.parametrize("lmax", [64, 257, 1024])
def test_rho_inv_modes_match_oracle(bie, ctx, ggq, name, surface, m0, lmax):
    s = bie.Surface(ctx, surface, 4, 40 if "torus" in name or name == "bean" else 32, ggq)
    t, th, ts = _queries(lmax, 10, [0.3, 0.05, 0.006, 0.002, 0.0005])
    got, gm0 = bie.rho_inv_modes(s, t, th, ts, lmax)
    ctx.sync()
    got, gm0 = got.cpu().numpy(), gm0.cpu().numpy()
    for q in range(len(t)):
        _, rm0 = km.rho_inv_modes_banded(surface, t[q], th[q], ts[q], lmax)
        assert gm0[q] == rm0, (name, q, gm0[q], rm0)
        if m0 is not None:
            assert rm0 == m0
        # the quantity has a plain definition: the refined trapezoid rule decides
        ref, _ = km.definition_rho_inv(surface, t[q], th[q], ts[q], lmax)
        ref = ref[lmax:]
        err = np.max(np.abs(got[q] - ref)) / np.max(np.abs(ref))
        assert err <= route_tol(lmax), (name, lmax, q, t[q] - ts[q], err)


def test_rho_inv_modes_against_definition_at_large_lmax(bie, ctx, ggq):
    # lmax = 4096: the quadrature panels shrink with 1/lmax; the plain definition decides
    surface = wl.ellipsoid(1.0, 0.8, 0.6)
    s = bie.Surface(ctx, surface, 4, 32, ggq)
    t, th, ts = np.array([1.1, 2.0]), np.array([0.4, 5.0]), np.array([1.103, 2.05])
    got, _ = bie.rho_inv_modes(s, t, th, ts, 4096)
    ctx.sync()
    got = got.cpu().numpy()
    for q in range(2):
        ref, _ = km.definition_rho_inv(surface, t[q], th[q], ts[q], 4096)
        ref = ref[4096:]
        assert np.max(np.abs(got[q] - ref)) <= TOL * np.max(np.abs(ref)), q


CASES = [("ellipsoid", wl.ellipsoid(1.0, 0.8, 0.6), 4, 64, 3.0), ("bumpy", wl.bumpy(), 4, 64, 5.0),
         ("star", wl.harmonic_star(5, 0, 0.12), 4, 96, 8.0), ("wiggly_torus", wl.wiggly_torus(), 5, 30, 1.0)]


def _torus_geometry(Np, Mt, rows, srcs, ggq_x):
    from oracle import nystrom as ny
    t_nodes, h = ny.nodes(Np, 2 * np.pi)
    tn = rows // Mt
    j, l = tn // 16, tn % 16
    d, g = srcs // 16, srcs % 16
    ts = (j + d - 1 + 0.5) * h + (h / 2) * ggq_x[d, l, g]
    return t_nodes[tn], 2 * np.pi * (rows % Mt) / Mt, ts


@pytest.mark.parametrize("name,surface,Np,Mt,k", CASES, ids=[c[0] for c in CASES])
def test_single_layer_modes_match_oracle(bie, ctx, ggq, name, surface, Np, Mt, k):
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    rows, srcs = sample_pairs(Np, Mt, 60, seed=7)
    if "torus" in name:   # every source of a seam row (cyclic neighbours)
        rows = np.concatenate([rows, np.zeros(48, np.int64)])
        srcs = np.concatenate([srcs, np.arange(48, dtype=np.int32)])
    got = bie.kernel_modes_banded(s, k, torch.from_numpy(rows).cuda(), torch.from_numpy(srcs).cuda())
    ctx.sync()
    got = got.cpu().numpy()
    if "torus" in name:
        t, th, ts = _torus_geometry(Np, Mt, rows, srcs, ggq[0])
    else:
        t, th, ts = pair_geometry(Np, Mt, rows, srcs, ggq[0])
    ref = km.method_modes_banded(surface, t, th, ts, Mt, k)
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= TOL, (name, int(err.argmax()), err.max())


def test_two_gpu_routes_agree(bie, ctx, ggq):
    # singularity swapping (bie_kernel_modes) and the O(M) route on every near pair of two target rows
    surface, Np, Mt, k = wl.ellipsoid(1.0, 0.8, 0.6), 4, 64, 3.0
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    rows = np.repeat(np.array([16 * Mt + 5 * Mt + 3, 2 * 16 * Mt + 7], np.int64), 48)
    srcs = np.tile(np.arange(48, dtype=np.int32), 2)
    r, c = torch.from_numpy(rows).cuda(), torch.from_numpy(srcs).cuda()
    a = bie.kernel_modes(s, bie.KERNEL_S, k, r, c)[:, 0]
    b = bie.kernel_modes_banded(s, k, r, c)
    ctx.sync()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    err = np.max(np.abs(a - b), axis=1) / np.max(np.abs(a), axis=1)
    assert err.max() <= 1e-12, err.max()


def test_invalid_queries(bie, ctx, ggq):
    s = bie.Surface(ctx, wl.ellipsoid(1.0, 0.8, 0.6), 4, 32, ggq)
    with pytest.raises(RuntimeError):
        bie.rho_inv_modes(s, [1.0], [0.5], [1.1], 4)          # lmax below 4d + 1
    got, _ = bie.rho_inv_modes(s, [1.0, 1.2], [0.5, 0.5], [1.0, float("nan")], 64)
    with pytest.raises(RuntimeError):
        ctx.sync()                                             # t == t_s and a NaN: BIE_ENAN
    assert torch.isnan(torch.view_as_real(got)).all()
    ok, _ = bie.rho_inv_modes(s, [1.0], [0.5], [1.1], 64)     # the context stays usable
    ctx.sync()
    assert torch.isfinite(torch.view_as_real(ok)).all()
