"""GPU parity: kernel modes of the CUDA pair pipeline vs the FP64 oracle
(per pair, normwise relative difference max_m |gpu - oracle| / max_m |oracle|)."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import kernel_modes as km
from tests.pairs import pair_geometry, sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


@pytest.fixture(scope="module")
def ctx(bie):
    return bie.Context()


def _check(bie, ctx, ggq, surface, Np, Mt, k, n, seed=0, kernels=("S",)):
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    rows, srcs = sample_pairs(Np, Mt, n, seed)
    mask = (bie.KERNEL_S if "S" in kernels else 0) | (bie.KERNEL_K if "K" in kernels else 0)
    out = bie.kernel_modes(s, mask, k, torch.from_numpy(rows).cuda(), torch.from_numpy(srcs).cuda())
    ctx.sync()
    t, th, ts = pair_geometry(Np, Mt, rows, srcs, ggq[0])
    chunks = [km.method_modes(surface, t[c:c + 256], th[c:c + 256], ts[c:c + 256], Mt, k, tuple(kernels))
              for c in range(0, len(t), 256)]
    worst = 0.0
    for idx, kd in enumerate(kernels):
        gpu = out[:, idx, :].cpu().numpy()
        ref = np.concatenate([ch[kd] for ch in chunks])
        err = np.max(np.abs(gpu - ref), axis=1) / np.max(np.abs(ref), axis=1)
        assert np.all(np.isfinite(gpu))
        assert err.max() <= TOL, "%s: worst pair %d: %.3e" % (kd, err.argmax(), err.max())
        worst = max(worst, err.max())
    return worst


def test_sphere_general_path(bie, ctx, ggq):
    _check(bie, ctx, ggq, wl.sphere(), 4, 32, 1.0, 1500)


def test_ellipsoid_m128(bie, ctx, ggq):
    _check(bie, ctx, ggq, wl.ellipsoid(1.0, 0.8, 0.6), 16, 128, 10.0, 400)


def test_bumpy_m128_k20(bie, ctx, ggq):
    _check(bie, ctx, ggq, wl.bumpy(), 24, 128, 20.0, 400)


def test_ragged_small_grids(bie, ctx, ggq):
    # Mth with a factor 3 (radix-3 passes) and the smallest grid
    _check(bie, ctx, ggq, wl.ellipsoid(1.0, 0.8, 0.6), 3, 24, 2.0, 300)
    _check(bie, ctx, ggq, wl.sphere(), 2, 8, 1.0, 200)


@pytest.mark.parametrize("surface,Np,Mt,k", [(wl.sphere(), 4, 32, 1.0), (wl.ellipsoid(1.0, 0.8, 0.6), 16, 128, 10.0),
                                             (wl.bumpy(), 6, 96, 5.0)])
def test_double_layer_and_single_layer_together(bie, ctx, ggq, surface, Np, Mt, k):
    _check(bie, ctx, ggq, surface, Np, Mt, k, 300, seed=2, kernels=("S", "K"))


def test_double_layer_alone(bie, ctx, ggq):
    _check(bie, ctx, ggq, wl.ellipsoid(1.0, 0.8, 0.6), 3, 24, 2.0, 300, seed=3, kernels=("K",))


def test_invalid_pair_reports_error(bie, ctx, ggq):
    s = bie.Surface(ctx, wl.sphere(), 4, 32, ggq)
    rows = torch.tensor([0, 5], dtype=torch.int64, device="cuda")      # panel 0 has no left neighbour
    srcs = torch.tensor([3, 20], dtype=torch.int32, device="cuda")
    out = bie.kernel_modes(s, bie.KERNEL_S, 1.0, rows, srcs)
    with pytest.raises(bie.BieError):
        ctx.sync()
    assert torch.all(out[0] == 0)
    ctx.sync()  # the status word was cleared


def test_fp64_transforms_option(bie, ggq):
    """The single layer's transforms in FP64 (a context option) against the oracle, per pair and in the
    assembled rows (FP64 weights and near fill)."""
    ctx = bie.Context()
    ctx.set_option(bie.OPT_FP64_TRANSFORMS, 1)
    _check(bie, ctx, ggq, wl.ellipsoid(1.0, 0.8, 0.6), 16, 128, 10.0, 400, seed=7)
    _check(bie, ctx, ggq, wl.bumpy(), 6, 96, 5.0, 300, seed=8)
    from oracle import nystrom as ny
    s = bie.Surface(ctx, wl.ellipsoid(1.0, 0.8, 0.6), 4, 64, ggq)
    A = bie.assemble(s, bie.OP_S, 4.0)
    ctx.sync()
    rows = np.unique(np.concatenate([wl.sample_rows(4, 64, 10, seed=5), [0, s.N - 1]]))
    got = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    ref = ny.operator_rows(wl.ellipsoid(1.0, 0.8, 0.6), 4, 64, 4.0, ggq[0], ggq[1], rows, op="S")
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert err.max() <= TOL, err.max()
