"""Block matrix products and the lockstep multi-right-hand-side solve.

The paper states the system (Section 3.4) and no solver.  The products are checked against numpy's
FP64 product of the same matrix (ragged sizes: rows not a multiple of the 128-row tile, columns not
a multiple of the 32-column k-tile; 1..16 right-hand sides), with bounds from each storage format's
rounding: FP64 and the double-word product at 1e-13, FP32 storage at 1e-6, split BF16 (16
significant bits per component) at 5e-5 normwise.  The block solve is checked against solving the
right-hand sides one at a time, and the mixed solves against the FP64 solve."""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

BOUND = {0: 1e-13, 1: 1e-6, 2: 5e-5, 3: 1e-13}


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


@pytest.fixture(scope="module")
def ctx(bie):
    return bie.Context()


def _check_products(bie, ctx, A, nrs, seed):
    n = A.shape[0]
    Ad = torch.from_numpy(A).cuda()
    M = bie.Matrix(ctx, Ad, bie.STORE_FP32 | bie.STORE_BF16X2)
    for nr in nrs:
        x = wl.random_complex((nr, n), seed, nr)
        ref = x @ A.T
        xd = torch.from_numpy(x).cuda()
        for prec in (0, 1, 2, 3):
            y = M.matvec(xd, prec)
            ctx.sync()   # raises on a device-side error flag (an expired bounded wait)
            y = y.cpu().numpy()
            err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert np.all(np.isfinite(y)) and err.max() <= BOUND[prec], (n, nr, prec, err.max())
            if prec == 2:   # the lo half is used: a single BF16 copy would be ~1e-3 off
                assert err.max() <= 5e-5


def test_products_ragged_random(bie, ctx):
    n = 1000
    A = wl.random_complex((n, n), 40, 0) / np.sqrt(n) + np.eye(n)
    _check_products(bie, ctx, A, (1, 3, 8, 9, 16), 41)


def test_products_stream_k_boundaries(bie, ctx):
    # 40 row tiles x 157 k-tiles over all SMs: every CTA's share crosses row-tile boundaries
    n = 5017
    A = wl.random_complex((n, n), 42, 0) / np.sqrt(n)
    _check_products(bie, ctx, A, (2, 16), 43)


def test_products_of_an_assembled_operator(bie, ctx, ggq):
    s = bie.Surface(ctx, wl.ellipsoid(1.0, 0.8, 0.6), 4, 32, ggq)
    A = bie.assemble(s, bie.OP_CFIE | bie.UNWEIGHTED, 3.0).cpu().numpy()
    _check_products(bie, ctx, A, (5,), 44)


def _system(bie, ctx, ggq, k=4.0):
    surf = wl.ellipsoid(1.0, 0.8, 0.6)
    s = bie.Surface(ctx, surf, 6, 48, ggq)
    A = bie.assemble(s, bie.OP_CFIE | bie.UNWEIGHTED, k)
    dirs = wl.Stream(0, 1).directions(4)
    B = torch.stack([bie.rhs(s, 0, d, k) for d in dirs] + [bie.rhs(s, 1, [0.1, 0.1, -0.05], k)])
    return s, A, B


def test_block_solve_matches_one_at_a_time(bie, ctx, ggq):
    s, A, B = _system(bie, ctx, ggq)
    X, rep = bie.solve(ctx, A, B, tol=1e-11, restart=100, maxit=500)
    assert rep["rel_residual"] <= 1e-11
    for c in range(B.shape[0]):
        xc, rc = bie.solve(ctx, A, B[c], tol=1e-11, restart=100, maxit=500)
        assert rc["rel_residual"] <= 1e-11
        assert float(torch.linalg.norm(X[c] - xc) / torch.linalg.norm(xc)) <= 1e-9
    # one block product per iteration for all five right-hand sides
    assert rep["matvecs"] <= rep["iterations"] + 40


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_block_solves_match_fp64(bie, ctx, ggq, prec):
    s, A, B = _system(bie, ctx, ggq)
    X64, r64 = bie.solve(ctx, A, B, tol=1e-10, restart=100, maxit=1000, prec=0)
    M = bie.Matrix(ctx, A, bie.STORE_FP32 if prec == 1 else bie.STORE_BF16X2)
    X, rep = M.solve(B, tol=1e-10, restart=100, maxit=1000, prec=prec)
    assert rep["rel_residual"] <= 1e-10 and rep["refinements"] >= 1
    pts = wl.exterior_points(16, 3.0)
    for c in range(B.shape[0]):
        u64 = bie.field_eval(s, bie.OP_CFIE | bie.UNWEIGHTED, 4.0, X64[c].contiguous(), pts).cpu().numpy()
        u = bie.field_eval(s, bie.OP_CFIE | bie.UNWEIGHTED, 4.0, X[c].contiguous(), pts).cpu().numpy()
        assert np.linalg.norm(u - u64) / np.linalg.norm(u64) <= 1e-8, (prec, c)
