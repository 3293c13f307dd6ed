"""Conditioning of the double-layer modes (Section 4, Eqs. (tau3-standard), (tau3-modified)): the
tau_3 term multiplies the modes of H3 = tau_0 F^3 by B_m(0, b) ~ 1/b^2 while H3 vanishes to second
order at the root, so rounding in the H3 transform that is small next to H3's own size is strongly
amplified in K.  Measured on the oracle's method mode by adding normwise-relative noise of size eps
to the H3 samples (equivalently to their modes, by Parseval) or to the output of the convolutions."""
import numpy as np

import workloads as wl
from oracle import kernel_modes as km
from tests.pairs import pair_geometry, sample_pairs

EPS = 2.0 ** -46


def _noisy(x, rng):
    sc = np.sqrt(np.mean(np.abs(x) ** 2, axis=-1, keepdims=True))
    noise = rng.standard_normal(x.shape) + (1j * rng.standard_normal(x.shape) if np.iscomplexobj(x) else 0.0)
    return x + EPS * sc * noise


def _amplification(monkeypatch, name, wrap):
    ggq = wl.load_ggq()
    cfg = wl.config("ellipsoid_np16_m128_k10")
    rows, srcs = sample_pairs(cfg["Np"], cfg["Mt"], 48, seed=5)
    t, th, ts = pair_geometry(cfg["Np"], cfg["Mt"], np.asarray(rows), np.asarray(srcs), ggq[0])
    args = (cfg["surface"], t, th, ts, cfg["Mt"], cfg["k"], ("K",))
    ref = km.method_modes(*args)["K"]
    monkeypatch.setattr(km, name, wrap(getattr(km, name)))
    got = km.method_modes(*args)["K"]
    return np.max(np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)) / EPS


def test_h3_transform_is_amplified(monkeypatch):
    rng = np.random.default_rng(0)
    amp = _amplification(monkeypatch, "tau3_modes", lambda f: lambda H3, *a: f(_noisy(H3, rng), *a))
    assert amp > 200, amp


def test_convolutions_are_not_amplified(monkeypatch):
    rng = np.random.default_rng(1)
    amp = _amplification(monkeypatch, "linear_convolution", lambda f: lambda *a: _noisy(f(*a), rng))
    assert amp < 20, amp


def test_k_next_to_the_target_is_at_the_fp64_floor(monkeypatch):
    """Next to the target (a harmonic star at Mth = 256, the self-panel ring nearest two targets,
    t - t_s ~ 3e-5) noise of the size of one rounding (2^-53, relative) in the H3 samples moves the
    oracle's K modes by more than 3e-13 normwise: any FP64 evaluation of H3 = tau_0 F^3 carries such
    an error, so two FP64 implementations of K differ there by about 1e-12.  Moving an input (t, th,
    t_s) by one ulp moves K by a similar amount, the per-pair scale the GPU parity test of those
    pairs uses (1e-12 plus four times it)."""
    from tests.pairs import ulp_sensitivity
    ggq = wl.load_ggq()
    surface, Np, Mt, k = wl.harmonic_star(0, 300, 0.12), 8, 256, 12.0
    t, th, ts = pair_geometry(Np, Mt, np.array([16711, 16729]), np.array([19, 19]), ggq[0])
    assert np.all(np.abs(t - ts) < 1e-4)
    args = (surface, t, th, ts, Mt, k, ("K",))
    ref = km.method_modes(*args)["K"]
    rng = np.random.default_rng(2)
    orig = km.tau3_modes

    def noisy(H3, *a):
        sc = np.sqrt(np.mean(np.abs(H3) ** 2, axis=-1, keepdims=True))
        return orig(H3 + 2.0 ** -53 * sc * rng.standard_normal(H3.shape), *a)
    monkeypatch.setattr(km, "tau3_modes", noisy)
    moved = np.zeros(len(t))
    for _ in range(4):   # the largest change over four draws of the noise
        got = km.method_modes(*args)["K"]
        moved = np.maximum(moved, np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1))
    monkeypatch.setattr(km, "tau3_modes", orig)
    assert np.all(moved > 3e-13), moved
    assert np.all(ulp_sensitivity(surface, t, th, ts, Mt, k, "K") > 3e-13)
