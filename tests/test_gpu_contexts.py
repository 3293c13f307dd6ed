"""Per-context work buffers, plan lifetime and host-made faults.

 - Two contexts on two streams run the pair pipeline at the same time (different grids, so the
   work buffers differ in size); their outputs equal those of the same calls made one after the
   other, bit for bit.
 - A batch plan made at a small grid still matches the oracle after a larger call on the same
   device (the recurrence table the plan points to is never reallocated).
 - Non-finite inputs are refused or reported with BIE_ENAN: a NaN right-hand side in the FP64 and
   the mixed solve, a NaN coefficient in a surface descriptor; a network whose parameters are NaN
   makes the learned solve fall back to the block preconditioner."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import kernel_modes as km
from oracle import nystrom as ny
from tests.pairs import pair_geometry, sample_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


def _prepare(bie, ctx, ggq, surface, Np, Mt, n, seed):
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    rows, srcs = sample_pairs(Np, Mt, n, seed)
    return s, torch.from_numpy(rows).to("cuda"), torch.from_numpy(srcs).to("cuda")


def test_two_contexts_concurrent_equal_sequential(bie, ggq):
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ca, cb = bie.Context(sa), bie.Context(sb)
    jobs = [(ca, wl.bumpy(), 6, 96, 5.0, bie.KERNEL_S, 20000, 1),
            (cb, wl.ellipsoid(1.0, 0.8, 0.6), 4, 128, 9.0, bie.KERNEL_S | bie.KERNEL_K, 6000, 2),
            (ca, wl.harmonic_star(0, 320, 0.1), 4, 64, 3.0, bie.KERNEL_S | bie.KERNEL_K, 8000, 3),
            (cb, wl.sphere(), 4, 48, 1.0, bie.KERNEL_S, 30000, 4)]
    prepared = [(ctx,) + _prepare(bie, ctx, ggq, sf, Np, Mt, n, seed) + (k, kern)
                for ctx, sf, Np, Mt, k, kern, n, seed in jobs]
    torch.cuda.synchronize()
    # sequential reference: each call completes before the next
    seq = []
    for ctx, s, r, c, k, kern in prepared:
        with torch.cuda.stream(ctx.stream):
            seq.append(bie.kernel_modes(s, kern, k, r, c))
        ctx.sync()
    # concurrent: all four enqueued before any synchronisation, alternating contexts
    conc = []
    for ctx, s, r, c, k, kern in prepared:
        with torch.cuda.stream(ctx.stream):
            conc.append(bie.kernel_modes(s, kern, k, r, c))
    ca.sync()
    cb.sync()
    for x, y in zip(seq, conc):
        assert torch.equal(torch.view_as_real(x), torch.view_as_real(y))


def test_batch_plan_survives_a_larger_call(bie, ggq):
    ctx = bie.Context()
    sp, Np, Mt, k = wl.harmonic_star(0, 330, 0.08), 2, 64, 6.0
    s = bie.Surface(ctx, sp, Np, Mt, ggq)
    total = 16 * Np * 48 * Mt
    W = torch.full((1, total, Mt), complex("nan"), dtype=torch.complex128, device="cuda")
    plan = bie.Batch(ctx, [s], [k], bie.KERNEL_S, W, total)
    # a larger grid with the double layer on the same device (the largest recurrence table the
    # library uses), then the plan made before it
    big = bie.Surface(ctx, wl.sphere(), 2, 256, ggq)
    rows, srcs = sample_pairs(2, 256, 500, seed=5)
    bie.kernel_modes(big, bie.KERNEL_S | bie.KERNEL_K, 2.0, torch.from_numpy(rows).cuda(),
                     torch.from_numpy(srcs).cuda())
    plan.run()
    ctx.sync()
    rs = wl.Stream(5, 3)
    ps = np.unique(rs.integers(0, total - 1, 200))
    i = ps % Mt
    rest = ps // Mt
    g, d, tn = rest % 16, (rest // 16) % 3, rest // 48
    rows, srcs = tn * Mt + i, d * 16 + g
    ok = (rows // (16 * Mt) + srcs // 16 - 1 >= 0) & (rows // (16 * Mt) + srcs // 16 - 1 < Np)
    got = W[0, torch.from_numpy(ps).cuda()].cpu().numpy()
    assert np.all(got[~ok] == 0)
    t, th, ts = pair_geometry(Np, Mt, rows[ok], srcs[ok], ggq[0])
    o = km.method_modes(sp, t, th, ts, Mt, k, ("S",))
    ref = ny.parseval_weights_split(o["S_sing"], o["S_smooth"])
    err = np.max(np.abs(got[ok] - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= 1e-12, err.max()


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_right_hand_side_reports_enan(bie, ggq, prec):
    ctx = bie.Context()
    s = bie.Surface(ctx, wl.sphere(), 4, 32, ggq)
    A = bie.assemble(s, bie.OP_CFIE | bie.UNWEIGHTED, 1.0)
    g = bie.rhs(s, 0, [0.0, 0.0, 1.0], 1.0)
    g[17] = complex("nan")
    with pytest.raises(bie.BieError) as ei:
        bie.solve(ctx, A, g, tol=1e-8, prec=prec)
    assert "status 5" in str(ei.value)
    # the context stays usable
    g2 = bie.rhs(s, 0, [0.0, 0.0, 1.0], 1.0)
    _, rep = bie.solve(ctx, A, g2, tol=1e-8, prec=prec)
    assert rep["rel_residual"] <= 1e-8


def test_nan_surface_coefficient_reports_enan(bie, ggq):
    ctx = bie.Context()
    bad = wl.bumpy()
    bad = dict(bad, terms=[list(t) for t in bad["terms"]])
    bad["terms"][1][0] = float("nan")
    with pytest.raises(bie.BieError) as ei:
        bie.Surface(ctx, bad, 4, 32, ggq)
    assert "status 5" in str(ei.value)


def test_nan_network_falls_back(bie, ggq):
    ctx = bie.Context()
    Np, Mt, k = 4, 32, 1.0
    s = bie.Surface(ctx, wl.sphere(), Np, Mt, ggq)
    A = bie.assemble(s, bie.OP_S, k)
    B = bie.BlockDiag(ctx, A, 16 * Mt)
    net = bie.Net(ctx, params=np.full(bie.NET_PARAMS, np.nan, dtype=np.float32))
    g = bie.rhs(s, 0, [0.0, 0.0, 1.0], k)
    x, rep = bie.solve(ctx, A, g, tol=1e-8, restart=100, maxit=500, precond=bie.PRECOND_LEARNED, block=B,
                       net=net, surface=s, k=k)
    assert rep["fallback_used"] == 1 and rep["rel_residual"] <= 1e-8
    assert bool(torch.isfinite(torch.view_as_real(x)).all())
