"""Block-diagonal and learned preconditioners on the GPU against the oracle (oracle/precond.py),
and their use inside FGMRES."""
import numpy as np
import pytest
import torch

import oracle.nystrom as ny
import oracle.precond as P
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


@pytest.fixture(scope="module")
def sphere(bie, ggq):
    """Unit sphere, Np = 4, Mth = 32 (N = 2048): its single-layer system (first kind)."""
    ctx = bie.Context()
    c = wl.config("sphere_np4_m32_k1")
    s = bie.Surface(ctx, c["surface"], c["Np"], c["Mt"], ggq)
    A = bie.assemble(s, bie.OP_S, 1.0)
    return ctx, s, A, c


def _normwise(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("n,block", [(240, 80), (240, 48), (512, 256)])
def test_blockdiag_apply_matches_oracle(bie, n, block):
    ctx = bie.Context()
    A = wl.random_complex((n, n), 21, n + block) / np.sqrt(n) + 2.0 * np.eye(n)
    r = wl.random_complex((3, n), 22, n + block)
    Ad = torch.from_numpy(A).cuda()
    B = bie.BlockDiag(ctx, Ad, block)
    z = B.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    ref = P.block_diag_apply(A, block, r)
    assert _normwise(z, ref) < 1e-5
    # backward error of each block solve, a property that holds at any conditioning
    for b0 in range(0, n, block):
        sl = slice(b0, b0 + block)
        res = np.linalg.norm(z[:, sl] @ A[sl, sl].T - r[:, sl]) / (np.linalg.norm(A[sl, sl]) * np.linalg.norm(z[:, sl]))
        assert res < 1e-6


def test_blockdiag_on_the_single_layer_system(bie, sphere):
    ctx, s, A, c = sphere
    block = 16 * c["Mt"]
    B = bie.BlockDiag(ctx, A, block)
    r = wl.random_complex((2, s.N), 23, 0)
    z = B.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    An = A.cpu().numpy()
    ref = P.block_diag_apply(An, block, r)
    assert _normwise(z, ref) < 1e-4
    for b0 in range(0, s.N, block):
        sl = slice(b0, b0 + block)
        res = np.linalg.norm(z[:, sl] @ An[sl, sl].T - r[:, sl]) / (np.linalg.norm(An[sl, sl]) * np.linalg.norm(z[:, sl]))
        assert res < 1e-6


def test_blockdiag_singular_block_is_reported(bie):
    ctx = bie.Context()
    n, block = 128, 64
    A = wl.random_complex((n, n), 24, 0) + 4 * np.eye(n)
    A[:, 70] = 0.0                                  # block 1 has a zero column
    with pytest.raises(bie.BieError, match="singular"):
        bie.BlockDiag(ctx, torch.from_numpy(A).cuda(), block)


def _params(stream, scale=0.15):
    p = wl.random_complex((P.N_PARAMS,), 25, stream).real * scale * np.sqrt(2.0)
    return p.astype(np.float32)


@pytest.mark.parametrize("B,nt,mt", [(2, 20, 24), (1, 16, 72)])
def test_network_forward_backward_match_oracle(bie, B, nt, mt):
    """Ragged shapes: 20 rows (weight-gradient tiles of 8), 72 columns (two theta chunks of 64)."""
    ctx = bie.Context()
    p = _params(1)
    net = bie.Net(ctx, params=p)
    pq = P.bf16_round(p)
    x = wl.random_complex((B, 4, nt, mt), 26, nt).real.astype(np.float32)
    gy = wl.random_complex((B, 2, nt, mt), 27, nt).real.astype(np.float32)
    xd, gyd = torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda()
    y = net.forward(xd).cpu().numpy()
    y_ref, _ = P.forward(pq, x.astype(np.float64))
    assert _normwise(y, y_ref) < 1e-5
    gp, gx = net.backward(xd, gyd)
    gp_ref, gx_ref = P.backward(pq, x.astype(np.float64), gy.astype(np.float64))
    gp = gp.cpu().numpy()
    o = 0
    for ci, co, _, _ in P.LAYERS:          # each layer's weights and biases separately
        for size in (co * ci * 9, co):
            assert _normwise(gp[o:o + size], gp_ref[o:o + size]) < 1e-4, (o, size)
            o += size
    assert _normwise(gx.cpu().numpy(), gx_ref) < 1e-4


def test_loss_gradient_matches_oracle(bie, sphere):
    """Training loss and parameter gradient on a synthetic system over the sphere's grid."""
    ctx, s, _, c = sphere
    Np, Mt = c["Np"], c["Mt"]
    nt, N = 16 * Np, s.N
    A = np.eye(N) + 0.5 * wl.random_complex((N, N), 28, 0) / np.sqrt(N)
    k = 3.0
    block = 16 * Mt
    Ad = torch.from_numpy(A).cuda()
    B = bie.BlockDiag(ctx, Ad, block)
    ts = bie.TrainSet(ctx, s, k, Ad, B)
    p = _params(2, 0.1)
    net = bie.Net(ctx, params=p)
    r = wl.random_complex((4, N), 29, 0).astype(np.complex64)
    loss, gp = net.loss_grad(ts, torch.from_numpy(r).cuda())
    J = ny.boundary_nodes(c["surface"], Np, Mt)[2]
    r64 = r.astype(np.complex128)
    zb = P.block_diag_apply(A, block, r64)
    loss_ref, gp_ref = P.loss_and_grad(P.bf16_round(p), A, r64, J, k, nt, Mt, zb)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    assert _normwise(gp.cpu().numpy(), gp_ref) < 1e-3


def test_precond_apply_matches_oracle(bie, sphere):
    ctx, s, A, c = sphere
    Np, Mt = c["Np"], c["Mt"]
    block = 16 * Mt
    B = bie.BlockDiag(ctx, A, block)
    p = _params(3, 0.1)
    net = bie.Net(ctx, params=p)
    v = wl.random_complex((2, s.N), 30, 0)
    z = net.precond_apply(s, 1.0, torch.from_numpy(v).cuda(), block=B).cpu().numpy()
    J = ny.boundary_nodes(c["surface"], Np, Mt)[2]
    zb = P.block_diag_apply(A.cpu().numpy(), block, v)
    ref = P.precond_apply(P.bf16_round(p), v, J, 1.0, 16 * Np, Mt, zb)
    assert _normwise(z, ref) < 1e-4


@pytest.fixture(scope="module")
def trained(bie, sphere):
    ctx, s, A, c = sphere
    B = bie.BlockDiag(ctx, A, 16 * c["Mt"])
    ts = bie.TrainSet(ctx, s, c["k"], A, B)
    net = bie.Net(ctx, seed=5)
    p0 = net.params()
    hist = net.train([ts], steps=200, batch=8, lr=1e-3, seed=3)
    return net, B, hist, p0


def test_training_reduces_the_loss(trained):
    net, _, hist, p0 = trained
    assert np.all(np.isfinite(hist))
    assert np.mean(hist[-40:]) < 0.9 * np.mean(hist[:10])
    assert not np.array_equal(net.params(), p0)


def test_block_preconditioned_fgmres(bie, sphere):
    ctx, s, A, c = sphere
    g = bie.rhs(s, 0, c["dirs"][0], c["k"])
    x0, r0 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=2000)
    B = bie.BlockDiag(ctx, A, 16 * c["Mt"])
    x1, r1 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=2000, precond=bie.PRECOND_BLOCK, block=B)
    assert r1["rel_residual"] <= 1e-8 and r0["rel_residual"] <= 1e-8
    assert r1["iterations"] < r0["iterations"]
    assert float(torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)) < 1e-6


def test_learned_preconditioned_fgmres(bie, sphere, trained):
    ctx, s, A, c = sphere
    net, B, _, _ = trained
    g = bie.rhs(s, 0, c["dirs"][0], c["k"])
    x0, _ = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=2000)
    x2, r2 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=2000, precond=bie.PRECOND_LEARNED, block=B,
                       net=net, surface=s, k=c["k"])
    assert r2["rel_residual"] <= 1e-8
    assert float(torch.linalg.norm(x2 - x0) / torch.linalg.norm(x0)) < 1e-6


def test_learned_solve_falls_back_to_the_block_preconditioner(bie, sphere):
    """A network that cannot converge within the budget hands the solve to the block preconditioner."""
    ctx, s, A, c = sphere
    B = bie.BlockDiag(ctx, A, 16 * c["Mt"])
    bad = _params(4, 3.0)                       # large random output layer: a poor preconditioner
    net = bie.Net(ctx, params=bad)
    g = bie.rhs(s, 0, c["dirs"][0], c["k"])
    _, r1 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=2000, precond=bie.PRECOND_BLOCK, block=B)
    x, r = bie.solve(ctx, A, g, tol=1e-8, restart=40, maxit=r1["iterations"] + 5,
                     precond=bie.PRECOND_LEARNED, block=B, net=net, surface=s, k=c["k"])
    assert r["rel_residual"] <= 1e-8
    assert r["fallback_used"] == 1


def test_learned_on_a_held_out_system(bie, ggq):
    """Train on two systems of a harmonic-star family (first-kind S), then solve a held-out member
    three ways: plain FGMRES, block-diagonal, learned + block.  The learned form reaches 1e-8 and
    needs fewer iterations than plain FGMRES; against the block-diagonal form, its yardstick, it
    does not win (the hard directions of the first-kind S are global, beyond the network's
    receptive field), and the test records both counts rather than asserting a gain it lacks."""
    ctx = bie.Context()
    Np, Mt = 4, 32
    def system(seed, k):
        s = bie.Surface(ctx, wl.harmonic_star(seed, 400, 0.12), Np, Mt, ggq)
        A = bie.assemble(s, bie.OP_S, k)
        return s, A, bie.BlockDiag(ctx, A, 16 * Mt), k
    train = [system(1, 5.5), system(2, 7.0)]
    net = bie.Net(ctx, seed=7)
    sets = [bie.TrainSet(ctx, s, k, A, B) for s, A, B, k in train]
    hist = net.train(sets, steps=300, batch=8, lr=1e-3, seed=4)
    assert np.mean(hist[-40:]) < np.mean(hist[:10])
    s, A, B, k = system(3, 6.3)                  # held out
    g = bie.rhs(s, 0, [0.0, 0.0, 1.0], k)
    x0, r0 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=3000)
    x1, r1 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=3000, precond=bie.PRECOND_BLOCK, block=B)
    x2, r2 = bie.solve(ctx, A, g, tol=1e-8, restart=200, maxit=3000, precond=bie.PRECOND_LEARNED, block=B,
                       net=net, surface=s, k=k)
    for r in (r0, r1, r2):
        assert r["rel_residual"] <= 1e-8
    assert float(torch.linalg.norm(x2 - x1) / torch.linalg.norm(x1)) < 1e-6
    assert r2["iterations"] < r0["iterations"], (r2["iterations"], r0["iterations"])
    print("held-out k = %.1f: plain %d it %.3f s, block %d it %.3f s, learned + block %d it %.3f s (fallback %d)"
          % (k, r0["iterations"], r0["seconds"], r1["iterations"], r1["seconds"], r2["iterations"], r2["seconds"],
             r2["fallback_used"]))
