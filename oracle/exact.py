"""Oracle: closed-form reference solutions (no discretisation).

TEST INFRASTRUCTURE ONLY.

  mie_sound_soft(k, x, d, R)      scattered field of a plane wave e^{ik d.x}
                                  by a sound-soft sphere of radius R (textbook
                                  separation of variables):
                                  u^s = -sum_n i^n (2n+1) j_n(kR)/h_n(kR) h_n(k|x|) P_n(cos g)
  mie_far_field(k, xhat, d, R)    its far-field pattern, u^s ~ e^{ik|x|}/|x| u_inf:
                                  u_inf = (i/k) sum_n (2n+1) j_n(kR)/h_n(kR) P_n(cos g)
  point_source(k, x, src)         G(x; src) = e^{ik|x-src|}/(4 pi |x-src|)  (Eq. (helm:green))
"""
import numpy as np
from scipy import special as ss


def _nmax(k, R, r=None):
    return int(np.ceil(k * max(R, 1.0))) + 40


def mie_sound_soft(k, x, d, R=1.0):
    x = np.atleast_2d(np.asarray(x, float))
    d = np.asarray(d, float) / np.linalg.norm(d)
    r = np.linalg.norm(x, axis=1)
    cg = (x @ d) / r
    out = np.zeros(len(x), complex)
    for n in range(_nmax(k, R)):
        jR = ss.spherical_jn(n, k * R)
        hR = jR + 1j * ss.spherical_yn(n, k * R)
        hr = ss.spherical_jn(n, k * r) + 1j * ss.spherical_yn(n, k * r)
        out -= (1j ** n) * (2 * n + 1) * (jR / hR) * hr * ss.eval_legendre(n, cg)
    return out


def mie_far_field(k, xhat, d, R=1.0):
    xhat = np.atleast_2d(np.asarray(xhat, float))
    xhat = xhat / np.linalg.norm(xhat, axis=1)[:, None]
    d = np.asarray(d, float) / np.linalg.norm(d)
    cg = xhat @ d
    out = np.zeros(len(xhat), complex)
    for n in range(_nmax(k, R)):
        jR = ss.spherical_jn(n, k * R)
        hR = jR + 1j * ss.spherical_yn(n, k * R)
        out += (1j / k) * (2 * n + 1) * (jR / hR) * ss.eval_legendre(n, cg)
    return out


def point_source(k, x, src):
    x = np.atleast_2d(np.asarray(x, float))
    dd = np.linalg.norm(x - np.asarray(src, float), axis=1)
    return np.exp(1j * k * dd) / (4 * np.pi * dd)
