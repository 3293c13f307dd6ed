"""GPU parity of the assembled matrix rows against the oracle, and end-to-end
solves against closed-form solutions (Mie series, manufactured point source)."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import exact
from oracle import nystrom as ny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


@pytest.fixture(scope="module")
def ctx(bie):
    return bie.Context()


@pytest.mark.parametrize("op", ["S", "CFIE"])
@pytest.mark.parametrize("surface,Np,Mt,k", [(wl.sphere(), 4, 32, 1.0), (wl.ellipsoid(1.0, 0.8, 0.6), 5, 48, 4.0),
                                             (wl.bumpy(), 4, 64, 3.0)])
def test_assembled_rows_match_oracle(bie, ctx, ggq, surface, Np, Mt, k, op):
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    A = bie.assemble(s, bie.OP_S if op == "S" else bie.OP_CFIE, k)
    ctx.sync()
    rows = wl.sample_rows(Np, Mt, 40)
    rows = np.unique(np.concatenate([rows, [0, s.N - 1, 16 * Mt - 1, 16 * Mt]]))
    ref = ny.operator_rows(surface, Np, Mt, k, ggq[0], ggq[1], rows, op=op, eta=k)
    got = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= 1e-12, err.max()


def test_sphere_solve_matches_mie(bie, ctx, ggq):
    k, d = 1.0, [0.0, 0.0, 1.0]
    s = bie.Surface(ctx, wl.sphere(), 4, 32, ggq)
    A = bie.assemble(s, bie.OP_S, k)
    g = bie.rhs(s, 0, d, k)
    x, rep = bie.solve(ctx, A, g, tol=1e-12)
    pts = wl.exterior_points(10, 3.0)
    u = bie.field_eval(s, bie.OP_S, k, x, pts).cpu().numpy()
    ue = exact.mie_sound_soft(k, pts, d)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) <= 1e-8
    dirs = wl.Stream(0, 9).directions(8)
    ff = bie.field_eval(s, bie.OP_S, k, x, dirs, far_field=True).cpu().numpy()
    assert np.linalg.norm(ff - exact.mie_far_field(k, dirs, d)) / np.linalg.norm(ff) <= 1e-8
    # the solution agrees with the oracle's dense LU solve of its own matrix
    N = s.N
    Ao = ny.operator_rows(wl.sphere(), 4, 32, k, ggq[0], ggq[1], np.arange(N), op="S")
    xo = np.linalg.solve(Ao, ny.plane_wave_rhs(wl.sphere(), 4, 32, k, d))
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-9


def test_mixed_precision_solve_reaches_tolerance(bie, ctx, ggq):
    k, src = 4.0, [0.1, 0.1, -0.05]
    surf = wl.ellipsoid(1.0, 0.8, 0.6)
    s = bie.Surface(ctx, surf, 6, 48, ggq)
    A = bie.assemble(s, bie.OP_S, k)
    g = bie.rhs(s, 1, src, k)
    x64, r64 = bie.solve(ctx, A, g, tol=1e-8, prec=0)
    x32, r32 = bie.solve(ctx, A, g, tol=1e-8, prec=1)
    assert r64["rel_residual"] <= 1e-8 and r32["rel_residual"] <= 1e-8
    assert r32["refinements"] >= 1
    pts = wl.exterior_points(10, 3.0)
    ue = exact.point_source(k, pts, src)
    for x in (x64, x32):
        u = bie.field_eval(s, bie.OP_S, k, x, pts).cpu().numpy()
        assert np.linalg.norm(u - ue) / np.linalg.norm(ue) <= 1e-6


@pytest.mark.parametrize("op", ["S", "CFIE"])
def test_mixed_solve_fields_match_fp64_solve(bie, ctx, ggq, op):
    """The mixed solve (FP32 storage inside FGMRES, FP64 refinement) against the FP64 GPU solve of the
    same system: scattered fields at exterior points and far-field directions agree to 1e-8 relative."""
    k, d = 4.0, [0.3, -0.2, 0.93]
    surf = wl.ellipsoid(1.0, 0.8, 0.6)
    s = bie.Surface(ctx, surf, 6, 48, ggq)
    flag = bie.OP_S if op == "S" else bie.OP_CFIE | bie.UNWEIGHTED
    A = bie.assemble(s, flag, k)
    g = bie.rhs(s, 0, d, k)
    tol = 1e-10
    x64, r64 = bie.solve(ctx, A, g, tol=tol, restart=300, maxit=3000, prec=0)
    x32, r32 = bie.solve(ctx, A, g, tol=tol, restart=300, maxit=3000, prec=1)
    assert r64["rel_residual"] <= tol and r32["rel_residual"] <= tol and r32["refinements"] >= 1
    pts = wl.exterior_points(16, 3.0)
    dirs = wl.Stream(0, 9).directions(32)
    for where, far in ((pts, False), (dirs, True)):
        u64 = bie.field_eval(s, flag, k, x64, where, far_field=far).cpu().numpy()
        u32 = bie.field_eval(s, flag, k, x32, where, far_field=far).cpu().numpy()
        assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) <= 1e-8, (op, far)


def test_cfie_exterior_point_source(bie, ctx, ggq):
    # exterior Dirichlet problem through the combined-field operator I + K - i k S
    k, src = 4.0, [0.1, 0.1, -0.05]
    surf = wl.ellipsoid(1.0, 0.8, 0.6)
    s = bie.Surface(ctx, surf, 6, 48, ggq)
    A = bie.assemble(s, bie.OP_CFIE, k)
    x, rep = bie.solve(ctx, A, bie.rhs(s, 1, src, k), tol=1e-11)
    pts = wl.exterior_points(10, 3.0)
    u = bie.field_eval(s, bie.OP_CFIE, k, x, pts).cpu().numpy()
    ue = exact.point_source(k, pts, src)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) <= 1e-7
    assert rep["iterations"] < 400


def test_unweighted_cfie(bie, ctx, ggq):
    # columns times the source Jacobian, identity I: same system, better conditioned
    k, src = 4.0, [0.1, 0.1, -0.05]
    s = bie.Surface(ctx, wl.ellipsoid(1.0, 0.8, 0.6), 6, 48, ggq)
    Aw = bie.assemble(s, bie.OP_CFIE, k)
    Au = bie.assemble(s, bie.OP_CFIE | bie.UNWEIGHTED, k)
    J = torch.from_numpy(ny.boundary_nodes(wl.ellipsoid(1.0, 0.8, 0.6), 6, 48)[2]).cuda()
    diff = (Au - Aw * J[None, :]).abs().max() / Au.abs().max()
    assert diff.item() <= 1e-13
    g = bie.rhs(s, 1, src, k)
    xw, rw = bie.solve(ctx, Aw, g, tol=1e-10)
    xu, ru = bie.solve(ctx, Au, g, tol=1e-10)
    assert ru["iterations"] < rw["iterations"]
    pts = wl.exterior_points(10, 3.0)
    u = bie.field_eval(s, bie.OP_CFIE | bie.UNWEIGHTED, k, xu, pts).cpu().numpy()
    ue = exact.point_source(k, pts, src)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) <= 1e-7


def test_solver_reports_nonconvergence(bie, ctx, ggq):
    s = bie.Surface(ctx, wl.sphere(), 2, 16, ggq)
    A = bie.assemble(s, bie.OP_S, 1.0)
    g = bie.rhs(s, 0, [0, 0, 1], 1.0)
    with pytest.raises(bie.BieError):
        bie.solve(ctx, A, g, tol=1e-14, restart=2, maxit=3)


@pytest.mark.parametrize("rep", ["S", "K", "CFIE"])
@pytest.mark.parametrize("far", [False, True])
def test_field_eval_matches_oracle(bie, ctx, ggq, rep, far):
    """The layer potentials (and far-field patterns) of a random density against the oracle's sums.
    The kernel sums in double words, so the bound (1e-11 of the largest value) sits well inside the
    1e-8 required of scattered fields; a dropped term or a wrong sign misses it by orders."""
    surface, Np, Mt, k = wl.bumpy(), 4, 32, 3.0
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    dens = wl.random_complex((s.N,), 4, 1)
    op = {"S": bie.OP_S, "K": bie.OP_K, "CFIE": bie.OP_CFIE}[rep]
    pts = wl.Stream(0, 9).directions(8) if far else wl.exterior_points(8, 2.5)
    got = bie.field_eval(s, op, k, torch.from_numpy(dens).cuda(), pts, far_field=far).cpu().numpy()
    fn = ny.far_field if far else ny.field
    ref = fn(surface, Np, Mt, k, dens, pts, rep=rep)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref)), np.max(np.abs(got - ref)) / np.max(np.abs(ref))
