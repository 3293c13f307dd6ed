"""Seeded synthetic inputs shared by the tests, the bench and the oracle's callers.

This module holds input generation only (surface descriptors, random
directions, pair samples, the quadrature table file reader); none of the
method's arithmetic lives here.

Random numbers come from a counter-based generator: splitmix64 of
(seed * 2^32 + stream) advanced by a counter, mapped to doubles in [0, 1)
with the top 53 bits, and to normals by Box-Muller.

Surface descriptors are plain dicts:
  {"kind": "ellipsoid", "axes": (a, b, c)}
  {"kind": "star", "terms": [[c, p, q, m, s], ...]}   h = 1 + sum c sin^p t cos^q t T(m th)
with t in [0, pi] (the "semicircle" generating curve), T = cos (s=0) or sin (s=1).
"""
import math
import os
import numpy as np

_MASK = (1 << 64) - 1
_TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2608_16208_b300", "tables", "ggq16.txt")


# ----------------------------------------------------------------------------
# counter-based random numbers
# ----------------------------------------------------------------------------
def splitmix64(x):
    x = (x + 0x9E3779B97F4A7C15) & _MASK
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


class Stream:
    """Uniform / normal draws from splitmix64(seed, stream, counter)."""

    def __init__(self, seed, stream=0):
        self.key = ((int(seed) & 0xFFFFFFFF) << 32) | (int(stream) & 0xFFFFFFFF)
        self.counter = 0

    def uniform(self, n=None):
        count = 1 if n is None else int(n)
        out = np.empty(count)
        for i in range(count):
            v = splitmix64((self.key * 0x100000001B3 + self.counter) & _MASK)
            self.counter += 1
            out[i] = (v >> 11) * (1.0 / (1 << 53))
        return out[0] if n is None else out

    def normal(self, n=None):
        count = 1 if n is None else int(n)
        u1 = self.uniform(count)
        u2 = self.uniform(count)
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2 * np.pi * u2)
        return z[0] if n is None else z

    def integers(self, lo, hi, n=None):
        """Integers in [lo, hi]."""
        u = self.uniform(n)
        return (lo + np.floor(u * (hi - lo + 1))).astype(int)

    def directions(self, n):
        v = self.normal(3 * n).reshape(n, 3)
        return v / np.linalg.norm(v, axis=1)[:, None]


# ----------------------------------------------------------------------------
# quadrature table
# ----------------------------------------------------------------------------
def load_ggq(path=None):
    """GGQ nodes and weights, arrays [3, 16, 16] indexed [delta+1, l, g], and the
    16-point Gauss-Legendre rule on [-1, 1] that both the oracle and the library use."""
    tab = np.loadtxt(path or _TABLE)
    gx = np.zeros((3, 16, 16))
    gw = np.zeros((3, 16, 16))
    for row in tab:
        d, l = int(row[0]) + 1, int(row[1])
        gx[d, l] = row[3:19]
        gw[d, l] = row[19:35]
    glx, glw = np.polynomial.legendre.leggauss(16)
    return gx, gw, glx, glw


# ----------------------------------------------------------------------------
# surfaces
# ----------------------------------------------------------------------------
def sphere(radius=1.0):
    return {"kind": "ellipsoid", "axes": (radius, radius, radius)}


def ellipsoid(a, b, c):
    return {"kind": "ellipsoid", "axes": (float(a), float(b), float(c))}


def bumpy():
    """h = 1 + 0.1 cos(5 th) sin^2 t + 0.05 sin(3 th) sin^3 t."""
    return {"kind": "star", "terms": [[0.1, 2, 0, 5, 0], [0.05, 3, 0, 3, 1]]}


def _legendre_poly(l):
    """Coefficients (ascending powers of x) of the Legendre polynomial P_l."""
    return np.polynomial.legendre.leg2poly([0] * l + [1])


def harmonic_star(seed, stream, eps, lmax=4, grid=64):
    """h = 1 + eps * Y(t, th), Y = sum_{l<=lmax,|m|<=l} c_lm Y_lm (real orthonormal
    harmonics), c_lm ~ N(0,1), scaled so that max over a grid of |Y| is 1."""
    rs = Stream(seed, stream)
    terms = []
    for l in range(lmax + 1):
        P = _legendre_poly(l)
        for m in range(0, l + 1):
            dP = np.polynomial.polynomial.polyder(P, m) if m else P
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            if m:
                norm *= math.sqrt(2.0)
            for s in ((0,) if m == 0 else (0, 1)):
                c = rs.normal()
                for q, coef in enumerate(dP):
                    if coef != 0.0:
                        terms.append([c * norm * coef, m, q, m, s])
    terms = np.array(terms)
    # scale to max |Y| = 1 on a grid
    t = (np.arange(grid) + 0.5) * np.pi / grid
    th = 2 * np.pi * np.arange(2 * grid) / (2 * grid)
    T, TH = np.meshgrid(t, th, indexing="ij")
    Y = np.zeros_like(T)
    for c, p, q, m, s in terms:
        trig = np.cos(m * TH) if s == 0 else np.sin(m * TH)
        Y += c * np.sin(T) ** int(p) * np.cos(T) ** int(q) * trig
    scale = eps / np.max(np.abs(Y))
    terms[:, 0] *= scale
    return {"kind": "star", "terms": terms.tolist()}


# ----------------------------------------------------------------------------
# the configurations
# ----------------------------------------------------------------------------
CONFIGS = {
    # unit sphere through the general path
    "sphere_np4_m32_k1": dict(surface=sphere(), Np=4, Mt=32, k=1.0,
                              dirs=[[0.0, 0.0, 1.0]], src=[0.1, 0.2, -0.1]),
    # triaxial ellipsoid
    "ellipsoid_np16_m128_k10": dict(surface=ellipsoid(1.0, 0.8, 0.6), Np=16, Mt=128, k=10.0,
                                    dirs=None, src=[0.1, 0.1, -0.05]),
    # bumpy star, k = 20
    "bumpy_np24_m128_k20": dict(surface=bumpy(), Np=24, Mt=128, k=20.0,
                                dirs=[[0.0, 0.0, 1.0]], src=[0.1, 0.1, -0.05]),
}


def config(name):
    c = dict(CONFIGS[name])
    if c["dirs"] is None:
        c["dirs"] = Stream(0, 1).directions(4).tolist()
    return c


def batch_surfaces(seed=0, count=64):
    """Uneven batch: harmonic stars, k ~ U[1,20], Np ~ U{8..32}, Mt in {64..256}, nrhs ~ U{1..16}."""
    rs = Stream(seed, 7)
    out = []
    for i in range(count):
        eps = 0.15 * rs.uniform()
        k = 1.0 + 19.0 * rs.uniform()
        Np = int(rs.integers(8, 32))
        Mt = [64, 96, 128, 192, 256][int(rs.integers(0, 4))]
        nrhs = int(rs.integers(1, 16))
        out.append(dict(surface=harmonic_star(seed, 100 + i, eps), Np=Np, Mt=Mt, k=k, nrhs=nrhs))
    return out


def near_pair_count(Np, Mt):
    """Near pairs (target node, GGQ source node) of a non-periodic surface: 256 Mt (3Np - 2)."""
    return 256 * Mt * (3 * Np - 2)


def sample_rows(Np, Mt, n, seed=0, stream=3):
    """n distinct target rows (flat indices (panel*16 + node)*Mt + theta)."""
    N = 16 * Np * Mt
    rs = Stream(seed, stream)
    rows = set()
    while len(rows) < min(n, N):
        rows.add(int(rs.integers(0, N - 1)))
    return np.array(sorted(rows))


def exterior_points(n, radius, seed=0, stream=5):
    """n points on a sphere of the given radius (Fibonacci lattice, rotated by a seeded angle)."""
    rs = Stream(seed, stream)
    phase = 2 * np.pi * rs.uniform()
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    ph = np.pi * (3 - math.sqrt(5)) * i + phase
    return radius * np.stack([r * np.cos(ph), r * np.sin(ph), z], -1)


def random_complex(shape, seed, stream):
    """Complex normal array (E|z|^2 = 1) from numpy's PCG64 seeded by (seed, stream); for large
    synthetic test matrices, where the per-value splitmix64 stream above is too slow in Python."""
    g = np.random.default_rng([int(seed), int(stream)])
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2.0)


def wiggly_torus():
    """The wiggly torus of the paper's Example 3: r = (1.2 w cos t, w sin t, 1.7 sin th),
    w = 2 + cos th + 0.25 cos 5t, t and th in [0, 2 pi) (t periodic)."""
    return {"kind": "torus", "a": 1.2, "b": 1.0, "c": 1.7, "R": 2.0, "eps": 0.25, "m": 5}


def bean():
    """The bean-shaped surface of the paper's Example 2 (given there implicitly; the oracle's geometry
    parameterises it by z = cos t and the angle th around each horizontal elliptic cross-section)."""
    return {"kind": "bean"}


def twisted_torus():
    """The twisted torus of the paper's Example 4, with the six terms as printed there (two of them,
    cos th and -0.25 cos th, could be one term 0.75 cos th; kept as printed)."""
    return {"kind": "fourier_torus", "R": 4.5,
            "terms": [[0.17, 2, -1], [0.11, 2, 0], [1.0, 1, 0], [-0.25, 1, 0], [0.01, 1, 1], [-0.45, -1, 1]]}
