"""The oracle's O(M) route (Section 3.3, "An O(M) approach") pinned to the plain definition: the
single-layer modes of Eq. (Sphi:appr2) with <rho^{-1}>_l from the difference equation Eq. (lin:diff)
agree with the refined trapezoid rule of <e^{ik rho}/rho>_m where the grid resolves the smooth
factors (the ellipsoid at Mth = 64, k = 3), from well-separated to close pairs."""
import numpy as np
import pytest

import workloads as wl
from oracle import kernel_modes as km

ELL = wl.ellipsoid(1.0, 0.8, 0.6)


@pytest.mark.parametrize("dt", [0.3, 0.05, 0.006, 0.0005])
def test_banded_single_layer_matches_definition(dt):
    Mt, k, t, th = 64, 3.0, 1.1, 2 * np.pi * 5 / 64
    got = km.method_modes_banded(ELL, [t], [th], [t + dt], Mt, k)[0]
    ref, _ = km.definition_modes(ELL, t, th, t + dt, Mt // 2, k, "S")
    assert np.max(np.abs(got - ref)) <= 2e-13 * np.max(np.abs(ref))


def test_banded_route_satisfies_the_recurrence_identity():
    # Eq. (iter:formula) at every m whose terms stay inside the computed modes, including the m whose
    # equations the banded solve never imposed (they involve the quadrature boundary values)
    t, th, ts, lmax = 0.7, 1.3, 0.75, 96
    R, m0 = km.rho_inv_modes_banded(ELL, t, th, ts, lmax)
    n = 256
    thq = 2 * np.pi * np.arange(n) / n
    Y, _ = km._near_difference(ELL, np.full(n, ts), thq, np.full(n, t), np.full(n, th))
    c = np.fft.fft(np.sum(Y * Y, -1)) / n
    full = np.concatenate([np.conj(R[:0:-1]), R])                 # l = -lmax..lmax
    worst = 0.0
    for m in range(-lmax + m0, lmax - m0 + 1):
        terms = [(2 * m + j) * c[j % n] * full[lmax - (m + j)] for j in range(-m0, m0 + 1)
                 if abs(m + j) <= lmax]
        scale = max(abs(x) for x in terms)
        worst = max(worst, abs(sum(terms)) / scale)
    assert worst <= 1e-12
