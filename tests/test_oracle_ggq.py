"""Pin of the 16-node GGQ tables (Section 3.1): each rule integrates P_n(s) and
P_n(s) log|s - tau|, n < 16, over the reference panel; moments computed here
independently by tanh-sinh quadrature (mpmath), split at the singular point."""
import mpmath as mp
import numpy as np
import pytest

XL, _ = np.polynomial.legendre.leggauss(16)


def _moments(tau):
    mp.mp.dps = 20
    out = []
    pts = [-1, tau, 1] if -1 < tau < 1 else [-1, 1]
    for n in range(16):
        out.append(float(mp.quad(lambda s: mp.legendre(n, s) * mp.log(abs(s - tau)), pts)))
    return np.array(out)


@pytest.mark.parametrize("delta", [-1, 0, 1])
@pytest.mark.parametrize("l", [0, 3, 7, 8, 12, 15])
def test_ggq_rule_is_exact(ggq, delta, l):
    gx, gw = ggq[0], ggq[1]
    x, w = gx[delta + 1, l], gw[delta + 1, l]
    tau = XL[l] - 2.0 * delta
    P = np.polynomial.legendre.legvander(x, 15).T          # P_n(x_g)
    assert np.max(np.abs(P @ w - np.eye(16)[0] * 2.0)) <= 5e-14
    assert np.max(np.abs((P * np.log(np.abs(x - tau))) @ w - _moments(tau))) <= 1e-13
    assert np.all(w > 0) and np.all(np.abs(x) < 1) and np.all(np.diff(x) > 0)


def test_ggq_mirror_symmetry(ggq):
    gx, gw = ggq[0], ggq[1]
    for l in range(16):
        assert np.allclose(gx[2, l], -gx[0, 15 - l][::-1], atol=0)
        assert np.allclose(gx[1, l], -gx[1, 15 - l][::-1], atol=0)
        assert np.allclose(gw[2, l], gw[0, 15 - l][::-1], atol=0)
