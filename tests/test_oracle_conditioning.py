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
