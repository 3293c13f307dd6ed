"""Pins of the oracle's per-pair pipeline (Sections 3.2-3.3, 4):
  * the sphere through the general path, where everything has a closed form;
  * the plain definition (brute-force trapezoid, no singularity swapping), for S, K and K';
  * invariants the paper states: Eq. (iter:formula), conjugate symmetry;
  * a planted mistake that the pins must catch."""
import numpy as np
import pytest

import workloads as wl
from oracle import kernel_modes as km
from oracle import special as sp

ELL = wl.ellipsoid(1.0, 0.8, 0.6)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_sphere_special_case_closed_form():
    # r = (sin t cos th, sin t sin th, cos t): rho^2 = 2 r r_s (cosh b - cos(th_s - th)),
    # so a = th, F = sqrt(q/(r r_s)) and
    # <rho^{-1}>_l = e^{-il th} sqrt(q/(r r_s)) A_{|l|}(b)  (axisymmetric case, Section 3.2 Remark)
    M, Mt = 16, 32
    t = np.array([0.7, 1.3, 2.0, 0.2])
    ts = np.array([0.7004, 1.25, 2.3, 0.5])
    th = 2 * np.pi * np.array([3, 0, 17, 9]) / Mt
    out = km.method_modes(wl.sphere(), t, th, ts, Mt, 1.0, ("S",), return_details=True)
    r, rs = np.sin(t), np.sin(ts)
    # cosh b - 1 = ((r - r_s)^2 + (z - z_s)^2)/(2 r r_s) = 2 sin^2((t - t_s)/2)/(r r_s)
    b = 2 * np.arcsinh(np.abs(np.sin((t - ts) / 2)) / np.sqrt(r * rs))
    assert np.allclose(out["_a"], th, atol=1e-14)
    assert np.allclose(out["_b"], b, rtol=1e-12)
    A, _ = sp.a_modes(b, 2 * M)
    l = np.arange(-2 * M, 2 * M + 1)
    R = np.exp(-1j * l[None, :] * th[:, None]) * np.sqrt(np.exp(-b) / (r * rs))[:, None] * A[:, np.abs(l)]
    for i in range(len(t)):
        assert _rel(out["_R"][i], R[i]) <= 1e-13


@pytest.mark.parametrize("surface,Mt,k", [(ELL, 64, 10.0), (wl.bumpy(), 256, 1.0), (wl.sphere(), 32, 1.0)])
@pytest.mark.parametrize("dt", [2e-4, 0.006, 0.05, 0.3])
def test_method_matches_definition(surface, Mt, k, dt):
    t, th = 1.1, 2 * np.pi * 5 / Mt
    out = km.method_modes(surface, np.array([t]), np.array([th]), np.array([t + dt]), Mt, k, ("S", "K", "Kp"))
    for kd in ("S", "K", "Kp"):
        d, _ = km.definition_modes(surface, t, th, t + dt, Mt // 2, k, kd)
        assert _rel(out[kd][0], d) <= 1e-12, kd


@pytest.mark.parametrize("Mt", [64, 192])
def test_method_matches_definition_next_to_a_pole(Mt):
    """Targets and source rings within 0.003 of the pole t = 0 (J ~ sin t): the whole ring is physically
    close, so its differences and tau_0 must take the cancellation-free forms (Section 4 Remark) beyond
    the parameter window.  With plain subtraction there, tau_0 ~ kappa rho^2 / 2 carries relative errors
    ~1e-10 and the brute-force definition itself does not converge (method vs definition 2.8e-9 for K)."""
    surface, k = wl.harmonic_star(0, 300, 0.12), 12.0
    t = np.array([0.0020811215478220846, 0.0020811215478220846, 0.0011])
    ts = np.array([0.0022492321685155803, 0.0005, 0.0029])
    th = 2 * np.pi * np.array([0, 3, 11]) / Mt
    out = km.method_modes(surface, t, th, ts, Mt, k, ("S", "K", "Kp"))
    for i in range(len(t)):
        for kd in ("S", "K", "Kp"):
            d, _ = km.definition_modes(surface, t[i], th[i], ts[i], Mt // 2, k, kd)
            assert _rel(out[kd][i], d) <= 1e-12, (i, kd, _rel(out[kd][i], d))


def test_recurrence_identity_and_conjugate_symmetry():
    # Eq. (iter:formula): sum_n (2m+n) <rho^2>_n <rho^{-1}>_{-(m+n)} = 0 ; <rho^{-1}>_{-l} = conj <rho^{-1}>_l
    Mt, M = 64, 32
    t, th, ts = np.array([1.1]), np.array([2 * np.pi * 5 / Mt]), np.array([1.13])
    out = km.method_modes(ELL, t, th, ts, Mt, 3.0, ("S",), return_details=True)
    R, rmax = out["_R"][0], out["_rmax"]
    assert np.max(np.abs(R[::-1] - np.conj(R))) <= 1e-15 * np.max(np.abs(R))
    thq = 2 * np.pi * np.arange(Mt) / Mt
    _, _, _, _, _, _, Y = km._pair_samples(ELL, t, th, ts, Mt)
    c = np.fft.fft(np.sum(Y[0] ** 2, -1)) / Mt
    m0 = 2                                   # rho^2 of an ellipsoid is a trig polynomial of degree 2
    for m in range(-20, 21):
        acc = sum((2 * m + n) * c[n % Mt] * R[-(m + n) + rmax] for n in range(-m0, m0 + 1))
        assert abs(acc) <= 1e-12 * np.max(np.abs(R))


def test_planted_sign_error_is_caught(monkeypatch):
    # flip the phase of the singular convolution: the definition pin must fail
    orig = km.swap_convolution

    def wrong(f, a, A, lmax):
        return orig(f, -a, A, lmax)

    monkeypatch.setattr(km, "swap_convolution", wrong)
    t, th, dt, Mt, k = 1.1, 2 * np.pi * 5 / 64, 0.006, 64, 10.0
    out = km.method_modes(ELL, np.array([t]), np.array([th]), np.array([t + dt]), Mt, k, ("S",))
    dS, _ = km.definition_modes(ELL, t, th, t + dt, Mt // 2, k, "S")
    assert _rel(out["S"][0], dS) > 1e-6


def test_far_root_is_capped():
    # a target at the pole and a ring near the other pole: b would exceed the cap
    out = km.method_modes(wl.sphere(), np.array([0.0083]), np.array([0.0]), np.array([3.13]), 16, 1.0,
                          ("S",), return_details=True)
    assert out["_b"][0] == km.B_CAP
    dS, _ = km.definition_modes(wl.sphere(), 0.0083, 0.0, 3.13, 8, 1.0, "S")
    assert _rel(out["S"][0], dS) <= 1e-13


@pytest.mark.parametrize("surface,Mt", [(ELL, 64), (wl.bumpy(), 128)])
@pytest.mark.parametrize("dt", [0.006, 0.05, 0.3])
def test_banded_route_matches_swapped_route(surface, Mt, dt):
    # two of the paper's routes to <rho^{-1}>_l: the O(M) difference equation Eq. (lin:diff) with
    # quadrature boundary values, and singularity swapping Eq. (convolution); they share no step
    # beyond the geometry
    t, th = 1.1, 2 * np.pi * 5 / Mt
    out = km.method_modes(surface, np.array([t]), np.array([th]), np.array([t + dt]), Mt, 1.0, ("S",),
                          return_details=True)
    R, rmax = out["_R"][0], out["_rmax"]
    Rb, m0 = km.rho_inv_modes_banded(surface, t, th, t + dt, rmax)
    assert m0 == (2 if surface is ELL else 10)   # rho^2 of the ellipsoid is a trig polynomial of degree 2
    assert _rel(Rb, R[rmax:]) <= 1e-12


@pytest.mark.parametrize("t,th,ts", [(4.186, 1.571, 4.213), (3.651, 1.508, 3.647), (2.518, 4.650, 2.531)])
def test_paper_p_rule_on_the_twisted_torus(t, th, ts):
    # On the twisted torus of Example 4 other complex roots of rho^2 come close to the real axis for
    # some pairs, and F needs more than Mth modes: with p = M these pairs are off by 2e-11..6e-11 at
    # Mth = 100; the paper's rule for p (Eq. (F-expansion), a criterion like Eq. (crt:M0)) recovers
    # the definition to rounding.
    S = wl.twisted_torus()
    d, _ = km.definition_modes(S, t, th, ts, 50, 1.0, "S")
    plain = km.method_modes(S, np.array([t]), np.array([th]), np.array([ts]), 100, 1.0, ("S",))
    rule = km.method_modes(S, np.array([t]), np.array([th]), np.array([ts]), 100, 1.0, ("S",), f_rule=True)
    assert _rel(plain["S"][0], d) > 1e-11
    assert _rel(rule["S"][0], d) <= 1e-13
