"""Parity at the full size of the bumpy-surface workload (rho = 1 + 0.1 cos 5th sin^2 t + 0.05 sin 3th sin^3 t,
k = 20, Np = 24, Mth = 128: N = 49,152 unknowns, 2,293,760 near pairs), in the launch configurations the
bench uses for it: the single and double layer together over every near pair of the surface in one
kernel-modes launch, and the combined-field operator I + K - i k S assembled whole (far fill plus the
correction stage over every enumerated pair).  Sampled pairs and rows against the FP64 oracle
(Section 3.3; Section 4, Eqs. (dis:K), (tau3-standard), (tau3-modified); Section 3.4)."""
import numpy as np
import pytest
import torch

import oracle.nystrom as ny
import workloads as wl
from oracle import kernel_modes as km
from tests.pairs import pair_geometry

pytestmark = pytest.mark.gpu

CFG = wl.config("bumpy_np24_m128_k20")
NP, MT, K = CFG["Np"], CFG["Mt"], CFG["k"]


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


def test_bumpy_single_and_double_layer_every_pair(bie, ggq):
    ctx = bie.Context()
    s = bie.Surface(ctx, CFG["surface"], NP, MT, ggq)
    N = s.N
    rows = torch.arange(N, device="cuda", dtype=torch.int64).repeat_interleave(48)
    srcs = torch.arange(48, device="cuda", dtype=torch.int32).repeat(N)
    panel = rows // (16 * MT) + srcs.to(torch.int64) // 16 - 1
    keep = (panel >= 0) & (panel < NP)
    rows, srcs = rows[keep].contiguous(), srcs[keep].contiguous()
    n = rows.numel()
    assert n == s.near_pairs
    out = bie.kernel_modes(s, bie.KERNEL_S | bie.KERNEL_K, K, rows, srcs)
    ctx.sync()
    assert bool(torch.isfinite(torch.view_as_real(out)).all())
    rs = wl.Stream(8, 3)
    pick = np.unique(np.concatenate([rs.integers(0, n - 1, 200), [0, n // 2, n - 1]]))
    got = out[torch.from_numpy(pick).cuda()].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    r_np, s_np = rows.cpu().numpy()[pick], srcs.cpu().numpy()[pick]
    t, th, ts = pair_geometry(NP, MT, r_np, s_np, ggq[0])
    chunks = [km.method_modes(CFG["surface"], t[c:c + 128], th[c:c + 128], ts[c:c + 128], MT, K, ("S", "K"))
              for c in range(0, len(t), 128)]
    for idx, kd in enumerate(("S", "K")):
        ref = np.concatenate([ch[kd] for ch in chunks])
        err = np.max(np.abs(got[:, idx] - ref), axis=1) / np.max(np.abs(ref), axis=1)
        assert err.max() <= 1e-12, (kd, int(pick[err.argmax()]), err.max())


def test_bumpy_combined_field_rows(bie, ggq):
    ctx = bie.Context()
    s = bie.Surface(ctx, CFG["surface"], NP, MT, ggq)
    A = bie.assemble(s, bie.OP_CFIE, K, eta=K)
    ctx.sync()
    N = s.N
    rows = np.unique(np.concatenate([wl.sample_rows(NP, MT, 5, seed=9), [0, N - 1, 16 * MT - 1, 16 * MT,
                                                                         12 * 16 * MT + 77]]))
    got = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    del A
    torch.cuda.empty_cache()
    ref = ny.operator_rows(CFG["surface"], NP, MT, K, ggq[0], ggq[1], rows, op="CFIE", eta=K)
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= 1e-12, err.max()
