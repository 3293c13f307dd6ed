"""The oracle's surfaces (Section 2, Eq. (para); Section 5 examples): analytic first and second
derivatives against central differences, at real and complex theta (the continuation the root
finder uses); unit outward normals; t-periodicity of the torus-like surfaces; and the bean's
implicit equation."""
import numpy as np
import pytest

import workloads as wl
from oracle import geometry as geo

SURFACES = {"ellipsoid": wl.ellipsoid(1.0, 2.0, 3.0), "bumpy": wl.bumpy(), "bean": wl.bean(),
            "wiggly_torus": wl.wiggly_torus(), "twisted_torus": wl.twisted_torus()}


@pytest.mark.parametrize("name", sorted(SURFACES))
@pytest.mark.parametrize("th", [1.3, 1.3 + 0.15j])
def test_derivatives_match_central_differences(name, th):
    S, t, h = SURFACES[name], 0.77, 1e-5
    r, rt, rth, rtt, rtth, rthth = geo.evaluate(S, t, th)
    f = lambda tt, hh: geo.evaluate(S, tt, hh)
    pairs = [((f(t + h, th)[0] - f(t - h, th)[0]) / (2 * h), rt),
             ((f(t, th + h)[0] - f(t, th - h)[0]) / (2 * h), rth),
             ((f(t + h, th)[1] - f(t - h, th)[1]) / (2 * h), rtt),
             ((f(t, th + h)[1] - f(t, th - h)[1]) / (2 * h), rtth),
             ((f(t, th + h)[2] - f(t, th - h)[2]) / (2 * h), rthth)]
    for num, ana in pairs:
        assert np.max(np.abs(num - ana)) <= 1e-8 * (1 + np.max(np.abs(ana)))


@pytest.mark.parametrize("name", sorted(SURFACES))
def test_normals_are_unit_and_outward(name):
    # divergence theorem: V = (1/3) int r . nu dS is positive exactly when nu points outward; the
    # integrand is smooth and periodic in theta (and in t on the tori, J -> 0 at the poles otherwise),
    # so the trapezoid rule in theta is spectrally accurate and the midpoint rule in t second order
    S = SURFACES[name]
    L = geo.parameter_length(S)
    nt, nth = 400, 256
    t = ((np.arange(nt) + 0.5) * L / nt)[:, None]
    th = (2 * np.pi * np.arange(nth) / nth)[None, :]
    r = geo.evaluate(S, t, th)[0]
    nu, J = geo.normal_and_jacobian(S, t, th)
    assert np.allclose(np.sum(nu * nu, -1), 1.0) and np.all(J > 0)
    V = np.sum(np.sum(r * nu, -1) * J) * (L / nt) * (2 * np.pi / nth) / 3
    assert V > 0
    if name == "ellipsoid":
        assert abs(V - 4 * np.pi * 1 * 2 * 3 / 3) <= 1e-5 * V   # midpoint rule in t: O((pi/400)^2)


@pytest.mark.parametrize("name", ["wiggly_torus", "twisted_torus"])
def test_torus_like_surfaces_are_periodic_in_t(name):
    S = SURFACES[name]
    assert geo.is_periodic(S) and geo.parameter_length(S) == 2 * np.pi
    th = np.linspace(0, 2 * np.pi, 7)
    for a, b in zip(geo.evaluate(S, 0.0, th), geo.evaluate(S, 2 * np.pi, th)):
        assert np.allclose(a, b, atol=1e-12)


def test_bean_satisfies_its_implicit_equation():
    T, TH = np.meshgrid(np.linspace(0.05, np.pi - 0.05, 9), np.linspace(0, 2 * np.pi, 13))
    R = geo.evaluate(wl.bean(), T, TH)[0]
    x, y, z = R[..., 0], R[..., 1], R[..., 2]
    lhs = x ** 2 / (0.64 * (1 - 0.1 * np.cos(np.pi * z))) + (y + 0.3 * np.cos(np.pi * z)) ** 2 / (
        0.64 * (1 - 0.4 * np.cos(np.pi * z))) + z ** 2
    assert np.max(np.abs(lhs - 1)) <= 1e-14
