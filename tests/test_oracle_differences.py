"""The oracle's cancellation-free differences (Section 4, Remark) pinned to 40-digit arithmetic.

Both oracle routes to the kernel modes (the method and the brute-force definition) take r_s - r and
tau_0 = nu(t_s, th_s) . (r(t_s, th_s) - r(t, th)) (Section 4, the definition of tau_j) from the same
two functions, geometry.difference (the line integral of the first derivatives) and
geometry.tau0_stable (the second-derivative line integral), so the definition pin cannot see a
mistake in them.  Here they are checked against the plain subtraction and projection carried out in
40-digit mpmath arithmetic from the surfaces' own parameterisations (the normal from mpmath
derivatives), at pairs 1e-6 to 1e-2 apart, on every surface kind with a closed parameterisation:
the differences to 1e-14 of |r_s - r|, tau_0 (which vanishes like rho^2) to 1e-13 of rho^2."""
import mpmath as mp
import numpy as np
import pytest

import workloads as wl
from oracle import geometry as geo

mp.mp.dps = 40


def _r_ellipsoid(axes):
    a, b, c = (mp.mpf(v) for v in axes)
    return lambda t, th: mp.matrix([a * mp.sin(t) * mp.cos(th), b * mp.sin(t) * mp.sin(th), c * mp.cos(t)])


def _r_star(terms):
    def h(t, th):
        v = mp.mpf(1)
        for c, p, q, m, s in terms:
            trig = mp.cos(int(m) * th) if int(s) == 0 else mp.sin(int(m) * th)
            v += mp.mpf(c) * mp.sin(t) ** int(p) * mp.cos(t) ** int(q) * trig
        return v
    return lambda t, th: h(t, th) * mp.matrix([mp.sin(t) * mp.cos(th), mp.sin(t) * mp.sin(th), mp.cos(t)])


def _r_torus(sf):
    a, b, c, R, eps, m = (mp.mpf(sf[k]) for k in ("a", "b", "c", "R", "eps", "m"))
    def r(t, th):
        w = R + mp.cos(th) + eps * mp.cos(m * t)
        return mp.matrix([a * w * mp.cos(t), b * w * mp.sin(t), c * mp.sin(th)])
    return r


def _r_bean():
    def r(t, th):
        z = mp.cos(t)
        A = mp.mpf("0.64") * (1 - mp.mpf("0.1") * mp.cos(mp.pi * z))
        B = mp.mpf("0.64") * (1 - mp.mpf("0.4") * mp.cos(mp.pi * z))
        return mp.matrix([mp.sqrt(A) * mp.sin(t) * mp.cos(th), -mp.mpf("0.3") * mp.cos(mp.pi * z) +
                          mp.sqrt(B) * mp.sin(t) * mp.sin(th), z])
    return r


SURFACES = [("ellipsoid", wl.ellipsoid(1.0, 0.8, 0.6), lambda sf: _r_ellipsoid(sf["axes"])),
            ("bumpy", wl.bumpy(), lambda sf: _r_star(sf["terms"])),
            ("harmonic_star", wl.harmonic_star(4, 2, 0.15), lambda sf: _r_star(sf["terms"])),
            ("wiggly_torus", wl.wiggly_torus(), _r_torus),
            ("bean", wl.bean(), lambda sf: _r_bean())]


def _pairs(seed):
    rs = wl.Stream(seed, 17)
    out = []
    for sep in (1e-6, 1e-4, 1e-3, 1e-2):
        t = 0.3 + 2.5 * rs.uniform()
        th = 2 * np.pi * rs.uniform()
        u = rs.uniform() * 2 * np.pi
        out.append((t + sep * np.cos(u), th + sep * np.sin(u), t, th))
    return out


@pytest.mark.parametrize("name,surface,mk", SURFACES, ids=[s[0] for s in SURFACES])
def test_difference_matches_40_digit_subtraction(name, surface, mk):
    r = mk(surface)
    for ts, ths, t, th in _pairs(1):
        got = geo.difference(surface, np.array([ts]), np.array([ths]), np.array([t]), np.array([th]), True)[0]
        ref = r(mp.mpf(ts), mp.mpf(ths)) - r(mp.mpf(t), mp.mpf(th))
        ref = np.array([float(ref[i]) for i in range(3)])
        assert np.max(np.abs(got - ref)) <= 1e-14 * np.linalg.norm(ref), (name, ts - t, got, ref)


@pytest.mark.parametrize("name,surface,mk", SURFACES, ids=[s[0] for s in SURFACES])
def test_tau0_matches_40_digit_projection(name, surface, mk):
    r = mk(surface)
    for ts, ths, t, th in _pairs(2):
        T, H = mp.mpf(ts), mp.mpf(ths)
        rt = mp.matrix([mp.diff(lambda x: r(x, H)[i], T) for i in range(3)])
        rth = mp.matrix([mp.diff(lambda y: r(T, y)[i], H) for i in range(3)])
        n = mp.matrix([rt[1] * rth[2] - rt[2] * rth[1], rt[2] * rth[0] - rt[0] * rth[2], rt[0] * rth[1] - rt[1] * rth[0]])
        n = n / mp.norm(n)
        d = r(T, H) - r(mp.mpf(t), mp.mpf(th))
        ref = sum(n[i] * d[i] for i in range(3))
        nu, _ = geo.normal_and_jacobian(surface, np.array([ts]), np.array([ths]))
        sign = 1.0 if np.dot(nu[0], [float(n[i]) for i in range(3)]) > 0 else -1.0   # orientation only
        got = geo.tau0_stable(surface, np.array([ts]), np.array([ths]), np.array([t]), np.array([th]))[0]
        # tau_0 = nu(r_s) . (r - r_s) vanishes to second order; compare against the size of rho^2
        rho2 = float(sum(d[i] ** 2 for i in range(3)))
        assert abs(got - sign * float(ref)) <= 1e-13 * rho2, (name, ts - t, got, float(ref))
