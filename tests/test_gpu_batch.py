"""Batch scheduler: several surfaces of uneven size (panels, Mth, k) in one persistent launch.
Parseval weights of sampled pairs against the oracle; ring output; CUDA-graph replay."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import kernel_modes as km
from oracle import nystrom as ny
from tests.pairs import pair_geometry

pytestmark = pytest.mark.gpu


def _decode(p, Mt):
    i = p % Mt
    rest = p // Mt
    g = rest % 16
    rest //= 16
    d = rest % 3
    tn = rest // 3
    return tn * Mt + i, d * 16 + g


def test_batch_matches_oracle_weights(ggq):
    import paper_2608_16208_b300 as bie
    ctx = bie.Context()
    specs = [(wl.ellipsoid(1.0, 0.8, 0.6), 3, 48, 4.0), (wl.bumpy(), 2, 64, 7.0),
             (wl.harmonic_star(0, 100, 0.1), 4, 32, 2.5)]
    surfs = [bie.Surface(ctx, sp, Np, Mt, ggq) for sp, Np, Mt, _ in specs]
    total = sum(16 * Np * 48 * Mt for _, Np, Mt, _ in specs)
    maxMt = max(Mt for _, _, Mt, _ in specs)
    W = torch.full((1, total, maxMt), complex("nan"), dtype=torch.complex128, device="cuda")
    b = bie.Batch(ctx, surfs, [k for *_, k in specs], bie.KERNEL_S, W, total)
    assert b.pairs == total
    b.run()
    ctx.sync()
    Wc = W[0].cpu().numpy()
    rs = wl.Stream(5, 1)
    for sidx, (sp, Np, Mt, k) in enumerate(specs):
        n_enum = 16 * Np * 48 * Mt
        ps = np.unique(rs.integers(0, n_enum - 1, 300))
        rows, srcs = zip(*[_decode(p, Mt) for p in ps])
        rows, srcs = np.array(rows), np.array(srcs)
        ip = rows // (16 * Mt) + srcs // 16 - 1
        ok = (ip >= 0) & (ip < Np)
        got = Wc[b.offsets[sidx] + ps, :Mt]
        assert np.all(got[~ok] == 0)
        t, th, ts = pair_geometry(Np, Mt, rows[ok], srcs[ok], ggq[0])
        o = km.method_modes(sp, t, th, ts, Mt, k, ("S",))
        ref = ny.parseval_weights_split(o["S_sing"], o["S_smooth"])
        err = np.max(np.abs(got[ok] - ref), axis=1) / np.max(np.abs(ref), axis=1)
        assert err.max() <= 1e-12, (sidx, err.max())


def test_batch_ring_and_graph_replay(ggq):
    import paper_2608_16208_b300 as bie
    ctx = bie.Context()
    surfs = [bie.Surface(ctx, wl.ellipsoid(1.0, 0.8, 0.6), 3, 32, ggq), bie.Surface(ctx, wl.sphere(), 2, 48, ggq)]
    ks = [3.0, 1.5]
    total = 16 * 3 * 48 * 32 + 16 * 2 * 48 * 48
    full = torch.zeros((1, total, 48), dtype=torch.complex128, device="cuda")
    bf = bie.Batch(ctx, surfs, ks, bie.KERNEL_S, full, total)
    bf.run()
    slot = 20000
    ring = torch.zeros((1, slot, 48), dtype=torch.complex128, device="cuda")
    br = bie.Batch(ctx, surfs, ks, bie.KERNEL_S, ring, slot)
    br.run()
    ctx.sync()
    # every ring row holds one of the pairs that map to it (the last writer wins): check rows written once
    once = [r for r in range(slot) if (r + slot) >= total]
    assert torch.equal(ring[0, once], full[0, once])
    # capture the run in a CUDA graph (the plan allocates nothing) and replay it
    stream = torch.cuda.Stream()
    ctx2 = bie.Context(stream)
    surfs2 = [bie.Surface(ctx2, wl.ellipsoid(1.0, 0.8, 0.6), 3, 32, ggq), bie.Surface(ctx2, wl.sphere(), 2, 48, ggq)]
    out = torch.zeros_like(full)
    bg = bie.Batch(ctx2, surfs2, ks, bie.KERNEL_S, out, total)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        bg.run()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, full)
