"""Pins of the preconditioner oracle (oracle/precond.py)."""
import numpy as np
import pytest
import scipy.signal
import torch

import oracle.precond as P
import workloads as wl


def _rand(shape, stream, scale=1.0):
    return scale * wl.Stream(11, stream).normal(int(np.prod(shape))).reshape(shape)


@pytest.mark.parametrize("d", [1, 2, 4])
def test_conv_matches_library_correlation(d):
    """One layer against scipy.signal.correlate2d on an explicitly padded image (zero rows in t,
    periodic columns in theta) with a dilated kernel."""
    cin, cout, nt, mt = 3, 2, 9, 12
    x = _rand((1, cin, nt, mt), 1)
    W = _rand((cout, cin, 3, 3), 2)
    b = _rand((cout,), 3)
    y = P.conv(x, W, b, d)
    for o in range(cout):
        ref = np.full((nt, mt), b[o])
        for c in range(cin):
            padded = np.pad(np.pad(x[0, c], ((d, d), (0, 0)), mode="constant"), ((0, 0), (d, d)), mode="wrap")
            ker = np.zeros((2 * d + 1, 2 * d + 1))
            ker[::d, ::d] = W[o, c]
            ref += scipy.signal.correlate2d(padded, ker, mode="valid")
        assert np.max(np.abs(y[0, o] - ref)) < 1e-12


@pytest.mark.parametrize("d", [1, 4])
def test_conv_adjoint_identity(d):
    x = _rand((2, 3, 7, 10), 4)
    g = _rand((2, 5, 7, 10), 5)
    W = _rand((5, 3, 3, 3), 6)
    lhs = np.sum(P.conv(x, W, None, d) * g)
    rhs = np.sum(x * P.conv_adjoint(g, W, d))
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


def _small_params(stream):
    p = _rand((P.N_PARAMS,), stream, 0.2)
    return p


def test_backward_matches_finite_differences():
    params = _small_params(7)
    x = _rand((1, 4, 6, 8), 8)
    gy = _rand((1, 2, 6, 8), 9)
    gp, gx = P.backward(params, x, gy)
    f = lambda p, xx: np.sum(gy * P.forward(p, xx)[0])
    rs = wl.Stream(11, 10)
    h = 1e-6
    for idx in rs.integers(0, P.N_PARAMS - 1, 12):
        e = np.zeros(P.N_PARAMS)
        e[idx] = h
        fd = (f(params + e, x) - f(params - e, x)) / (2 * h)
        assert abs(fd - gp[idx]) <= 1e-6 * max(1.0, abs(fd)), idx
    # the biases of every layer, where a dropped term would show
    for off in np.cumsum([co * ci * 9 + co for ci, co, _, _ in P.LAYERS]) - 1:
        e = np.zeros(P.N_PARAMS)
        e[off] = h
        fd = (f(params + e, x) - f(params - e, x)) / (2 * h)
        assert abs(fd - gp[off]) <= 1e-6 * max(1.0, abs(fd))
    for flat in rs.integers(0, x.size - 1, 8):
        e = np.zeros(x.size)
        e[flat] = h
        e = e.reshape(x.shape)
        fd = (f(params, x + e) - f(params, x - e)) / (2 * h)
        assert abs(fd - gx.ravel()[flat]) <= 1e-6 * max(1.0, abs(fd))


def test_loss_gradient_matches_finite_differences():
    nt, mt = 4, 8
    N = nt * mt
    rs = wl.Stream(11, 12)
    A = np.eye(N) + 0.3 * (rs.normal(N * N) + 1j * rs.normal(N * N)).reshape(N, N) / np.sqrt(N)
    r = (rs.normal(2 * N) + 1j * rs.normal(2 * N)).reshape(2, N)
    J = 1.0 + 0.5 * rs.uniform(N)
    k = 7.0
    zb = P.block_diag_apply(A, 8, r)
    params = _small_params(13)
    loss, gp = P.loss_and_grad(params, A, r, J, k, nt, mt, zb)

    def L(p):
        z = P.precond_apply(p, r, J, k, nt, mt, zb)
        e = z @ A.T - r
        return np.mean(np.sum(np.abs(e) ** 2, 1) / np.sum(np.abs(r) ** 2, 1))

    assert abs(L(params) - loss) < 1e-12
    h = 1e-6
    idxs = list(rs.integers(0, P.N_PARAMS - 1, 10)) + [P.N_PARAMS - 1, P.N_PARAMS - 2]
    for idx in idxs:
        e = np.zeros(P.N_PARAMS)
        e[idx] = h
        fd = (L(params + e) - L(params - e)) / (2 * h)
        assert abs(fd - gp[idx]) <= 1e-6 * max(1e-3, abs(fd)), idx


def test_block_diag_apply_solves_each_block():
    rs = wl.Stream(11, 14)
    n, block = 24, 8
    A = (rs.normal(n * n) + 1j * rs.normal(n * n)).reshape(n, n) + 4 * np.eye(n)
    r = rs.normal(n) + 1j * rs.normal(n)
    z = P.block_diag_apply(A, block, r)
    for b0 in range(0, n, block):
        sl = slice(b0, b0 + block)
        assert np.max(np.abs(A[sl, sl] @ z[sl] - r[sl])) < 1e-12
    assert np.max(np.abs(P.block_diag_apply(A, n, r) - np.linalg.solve(A, r))) < 1e-12


def test_bf16_round_matches_torch():
    x = wl.Stream(11, 15).normal(4096).astype(np.float32) * 10.0
    ours = P.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    # ties go to even
    assert P.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert P.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6
