"""Parity at the full size of the bench workload (ellipsoid (1, 0.8, 0.6), Np = 16, Mth = 128, k = 10,
N = 32,768), in the launch configurations the bench times: the operator S assembled whole (far fill
plus the correction stage over all 1,572,864 enumerated pairs in 2^20-pair chunks, with double-word
weights and near fill), and one kernel-modes launch over every near pair of the surface (two chunks).
Sampled rows and pairs are checked against the FP64 oracle one by one."""
import numpy as np
import pytest
import torch

import oracle.nystrom as ny
import workloads as wl
from oracle import kernel_modes as km
from tests.pairs import pair_geometry

pytestmark = pytest.mark.gpu

CFG = wl.config("ellipsoid_np16_m128_k10")
NP, MT, K = CFG["Np"], CFG["Mt"], CFG["k"]


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


def test_full_operator_rows(bie, ggq):
    ctx = bie.Context()
    s = bie.Surface(ctx, CFG["surface"], NP, MT, ggq)
    A = bie.assemble(s, bie.OP_S, K)
    ctx.sync()
    N = s.N
    # rows at both ends, across a panel boundary, and seeded interior rows; the chunk boundary of the
    # correction stage (enumerated pair 2^20) falls among the pairs of target node 170, so a row of
    # that node has pairs in both chunks
    rows = np.unique(np.concatenate([wl.sample_rows(NP, MT, 6, seed=3), [0, N - 1, 16 * MT - 1, 16 * MT,
                                                                         170 * MT + 7]]))
    got = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    del A
    torch.cuda.empty_cache()
    ref = ny.operator_rows(CFG["surface"], NP, MT, K, ggq[0], ggq[1], rows, op="S")
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= 1e-12, err.max()


def test_full_modes_launch(bie, ggq):
    ctx = bie.Context()
    s = bie.Surface(ctx, CFG["surface"], NP, MT, ggq)
    N = s.N
    rows = torch.arange(N, device="cuda", dtype=torch.int64).repeat_interleave(48)
    srcs = torch.arange(48, device="cuda", dtype=torch.int32).repeat(N)
    panel = rows // (16 * MT) + srcs.to(torch.int64) // 16 - 1
    keep = (panel >= 0) & (panel < NP)
    rows, srcs = rows[keep].contiguous(), srcs[keep].contiguous()
    n = rows.numel()
    assert n == s.near_pairs > (1 << 20)
    out = bie.kernel_modes(s, bie.KERNEL_S, K, rows, srcs)
    ctx.sync()
    rs = wl.Stream(7, 2)
    pick = np.unique(np.concatenate([rs.integers(0, n - 1, 240), [0, (1 << 20) - 1, 1 << 20, n - 1]]))
    got = out[torch.from_numpy(pick).cuda(), 0].cpu().numpy()
    assert np.all(np.isfinite(out[:, 0].abs().max(dim=1).values.cpu().numpy()))
    del out
    r_np, s_np = rows.cpu().numpy()[pick], srcs.cpu().numpy()[pick]
    t, th, ts = pair_geometry(NP, MT, r_np, s_np, ggq[0])
    ref = np.concatenate([km.method_modes(CFG["surface"], t[c:c + 128], th[c:c + 128], ts[c:c + 128], MT, K, ("S",))["S"]
                          for c in range(0, len(t), 128)])
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= 1e-12, (int(pick[err.argmax()]), err.max())
