"""Test helpers: map (target row, source) pairs to the oracle's (t, th, t_s)."""
import numpy as np

import workloads as wl
from oracle import nystrom as ny


def pair_geometry(Np, Mt, rows, srcs, ggq_x):
    t_nodes, h = ny.nodes(Np)
    rows = np.asarray(rows)
    srcs = np.asarray(srcs)
    tn = rows // Mt
    i = rows % Mt
    j, l = tn // 16, tn % 16
    d, g = srcs // 16, srcs % 16
    ip = j + d - 1
    ts = (ip + 0.5) * h + (h / 2) * ggq_x[d, l, g]
    return t_nodes[tn], 2 * np.pi * i / Mt, ts


def sample_pairs(Np, Mt, n, seed=0):
    """n valid pairs (row, src), plus every source of the first and last target rows."""
    rs = wl.Stream(seed, 11)
    N = 16 * Np * Mt
    rows, srcs = [], []
    while len(rows) < n:
        r = int(rs.integers(0, N - 1))
        s = int(rs.integers(0, 47))
        ip = r // (16 * Mt) + s // 16 - 1
        if 0 <= ip < Np:
            rows.append(r)
            srcs.append(s)
    for r in (0, N - 1):
        for s in range(48):
            ip = r // (16 * Mt) + s // 16 - 1
            if 0 <= ip < Np:
                rows.append(r)
                srcs.append(s)
    return np.array(rows, dtype=np.int64), np.array(srcs, dtype=np.int32)


def method_modes_chunk(args):
    """Process-pool worker: the oracle's method-mode modes of one chunk of pairs,
    args = (surface, t, th, t_s, Mt, k, kernels)."""
    from oracle import kernel_modes as km
    surface, t, th, ts, Mt, k, kernels = args
    return km.method_modes(surface, t, th, ts, Mt, k, kernels)


def ulp_sensitivity(surface, t, th, ts, Mt, k, kernel):
    """Per pair, the largest normwise change of the oracle's modes when one of the pair's FP64
    inputs (t, th, t_s) moves by one ulp: a per-pair scale of the coefficients' sensitivity."""
    from oracle import kernel_modes as km
    base = km.method_modes(surface, t, th, ts, Mt, k, (kernel,))[kernel]
    nb = np.max(np.abs(base), axis=1)
    out = np.zeros(len(t))
    for tt, hh, ss in ((np.nextafter(t, 10), th, ts), (t, np.nextafter(th, 10), ts), (t, th, np.nextafter(ts, 10))):
        v = km.method_modes(surface, tt, hh, ss, Mt, k, (kernel,))[kernel]
        out = np.maximum(out, np.max(np.abs(v - base), axis=1) / nb)
    return out
