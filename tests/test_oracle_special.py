"""Pins of the oracle's special functions against quadrature, library routines
and the paper's own identities (Section 3.3 Eqs. (Am), (Am-Q), (diff-recurrence);
Section 4 Prop. "lem:Bm", Eq. (B0))."""
import mpmath as mp
import numpy as np
import pytest
from scipy import special as ss

from oracle import special as sp

mp.mp.dps = 30


def _a_quad(m, b):
    q = mp.e ** (-mp.mpf(b))
    f = lambda p: mp.cos(m * p) / mp.sqrt(1 + q * q - 2 * q * mp.cos(p))
    return float(mp.quad(f, mp.linspace(0, mp.pi, 4 * m + 8)) / mp.pi)


def _b_quad(m, b):
    q = mp.e ** (-mp.mpf(b))
    f = lambda p: mp.cos(m * p) / (1 + q * q - 2 * q * mp.cos(p)) ** 1.5
    pts = [0, mp.mpf(b) / 4, mp.mpf(b), 4 * mp.mpf(b)] + list(mp.linspace(5 * mp.mpf(b), mp.pi, 4 * m + 8))
    pts = sorted(set(p for p in pts if p <= mp.pi))
    return float(mp.quad(f, pts) / mp.pi)


def test_ellipke_matches_library():
    m = np.array([0.0, 1e-6, 0.3, 0.9, 0.999999, 1 - 1e-12])
    K, E = sp.ellipke(m, 1 - m)
    assert np.allclose(K, ss.ellipk(m), rtol=1e-14, atol=0)
    assert np.allclose(E, ss.ellipe(m), rtol=1e-14, atol=0)


@pytest.mark.parametrize("b", [1e-4, 3e-3, 0.02, 0.3, 1.5, 3.5])
def test_a_modes_match_quadrature(b):
    L = 200
    A, D = sp.a_modes(np.array([b]), L)
    for m in [0, 1, 2, 7, 30]:
        assert abs(A[0, m] - _a_quad(m, b)) <= 2e-15 * A[0, 0]
    # the differences are the differences
    assert np.allclose(D[0, 1:], np.diff(A[0]), rtol=0, atol=1e-15 * A[0, 0])


@pytest.mark.parametrize("b", [0.05, 0.7])
def test_a_modes_are_scaled_legendre_q(b):
    # Eq. (Am-Q): A_m = e^{b/2}/pi Q_{m-1/2}(cosh b)
    A, _ = sp.a_modes(np.array([b]), 12)
    for m in [0, 1, 5, 12]:
        q = mp.legenq(m - 0.5, 0, mp.cosh(b), type=3)
        assert abs(A[0, m] - float(mp.re(q) * mp.e ** (b / 2) / mp.pi)) <= 1e-14 * A[0, 0]


def test_forward_and_miller_branches_agree():
    # same b on both sides of the L*b threshold
    b = 0.035
    A1, _ = sp.a_modes(np.array([b]), 199)      # L*b = 6.97 -> forward
    A2, _ = sp.a_modes(np.array([b]), 201)      # L*b = 7.04 -> Miller
    assert np.max(np.abs(A1[0] - A2[0, :200])) <= 1e-13 * A1[0, 0]


def test_three_term_recurrence_holds():
    for b in [0.01, 0.4, 2.0]:
        A, _ = sp.a_modes(np.array([b]), 100)
        m = np.arange(1, 100)
        lhs = (2 * m + 1) * A[0, m + 1]
        rhs = 4 * m * np.cosh(b) * A[0, m] - (2 * m - 1) * A[0, m - 1]
        assert np.max(np.abs(lhs - rhs)) <= 1e-13 * A[0, 0] * 100


@pytest.mark.parametrize("b", [0.003, 0.05, 0.5, 2.0])
def test_b_modes_match_quadrature_and_b0(b):
    A, D = sp.a_modes(np.array([b]), 60)
    B = sp.b_modes(np.array([b]), A, D)
    for m in [0, 1, 4, 20]:
        assert abs(B[0, m] - _b_quad(m, b)) <= 1e-13 * B[0, 0]
    # Eq. (B0)
    assert abs(B[0, 0] - sp.b0_closed_form(b)) <= 1e-13 * B[0, 0]


def test_b_modes_satisfy_paper_forward_recurrence_where_it_is_stable():
    # Eq. (Bm-recurrence) at a = 0: B_m = cosh b B_{m-1} - (2m-1)/2 e^b A_{m-1}
    b = 0.02
    A, D = sp.a_modes(np.array([b]), 20)
    B = sp.b_modes(np.array([b]), A, D)
    for m in range(1, 20):
        rec = np.cosh(b) * B[0, m - 1] - (2 * m - 1) / 2 * np.exp(b) * A[0, m - 1]
        assert abs(B[0, m] - rec) <= 1e-12 * B[0, 0]


@pytest.mark.parametrize("b", [4e-5, 0.01, 0.3])
def test_b_difference_identity(b):
    # B_{m-1} - B_{m+1} = <2i sin(th) s^{-3/2}>_m = 2 m e^b A_m  (from d/dth s^{-1/2} = -e^{-b} sin th s^{-3/2});
    # checked against independent quadrature of both B's
    A, _ = sp.a_modes(np.array([b]), 12)
    for m in (1, 4):
        assert abs(2 * m * np.exp(b) * A[0, m] - (_b_quad(m - 1, b) - _b_quad(m + 1, b))) <= 1e-9 * abs(_b_quad(m, b)) * b
