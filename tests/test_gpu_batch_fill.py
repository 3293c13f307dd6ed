"""The batch scheduler's throughput mode with the GGQ fill (Section 3.4, Eq. (S123)): every target
panel of every surface, folded into a bounded ring of near-band slots once its pairs are done, equals
that panel's rows of the single-surface near band (bie_assemble_near_band, single layer, weighted
density) to 1e-13 normwise per row (the batch folds FP64 weights, the single-surface stage double
words; both are within 1e-12 of the oracle's operator rows).  The weight ring is made small enough
that chunks are cut, panels straddle chunks and the ring wraps."""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


SPECS = [(wl.ellipsoid(1.0, 0.8, 0.6), 3, 64, 5.0), (wl.harmonic_star(2, 40, 0.1), 2, 96, 3.0),
         (wl.bumpy(), 3, 64, 8.0)]


@pytest.mark.parametrize("ring_extra_items", [3, 40])
def test_fill_matches_single_surface_band(bie, ggq, ring_extra_items):
    ctx = bie.Context()
    surfs = [bie.Surface(ctx, sp, Np, Mt, ggq) for sp, Np, Mt, _ in SPECS]
    ks = [k for *_, k in SPECS]
    maxMt = max(Mt for _, _, Mt, _ in SPECS)
    max_panel = max(16 * 48 * Mt for _, _, Mt, _ in SPECS)
    slot = max_panel + 1024 * ring_extra_items
    W = torch.zeros((1, slot, maxMt), dtype=torch.complex128, device="cuda")
    plan = bie.Batch(ctx, surfs, ks, bie.KERNEL_S, W, slot)
    n_panels = sum(Np for _, Np, _, _ in SPECS)
    band = torch.full((n_panels, 16 * maxMt, 3, 16 * maxMt), complex("nan"), dtype=torch.complex128, device="cuda")
    plan.set_fill(band, n_panels)
    assert plan.config["item_pairs"] <= slot - max_panel
    plan.run()
    ctx.sync()
    # processing order: classes by decreasing Mth, surfaces in order within a class, panels in order
    order = sorted(range(len(SPECS)), key=lambda i: -SPECS[i][2])
    f = 0
    for i in order:
        _, Np, Mt, k = SPECS[i]
        ref = bie.assemble_near_band(surfs[i], bie.KERNEL_S, k)
        ctx.sync()
        w = 16 * Mt
        for j in range(Np):
            got = band[f].reshape(-1)[: w * 3 * w].reshape(w, 3, w)
            exp = ref[j * w:(j + 1) * w]
            err = ((got - exp).abs().amax(dim=(1, 2)) / exp.abs().amax(dim=(1, 2))).max().item()
            assert err <= 1e-13, (i, j, err)
            f += 1
    assert f == n_panels


def test_fill_refuses_a_ring_without_room(bie, ggq):
    ctx = bie.Context()
    sp, Np, Mt, k = SPECS[0]
    s = bie.Surface(ctx, sp, Np, Mt, ggq)
    slot = 16 * 48 * Mt   # one panel, no room for a chunk
    W = torch.zeros((1, slot, Mt), dtype=torch.complex128, device="cuda")
    plan = bie.Batch(ctx, [s], [k], bie.KERNEL_S, W, slot)
    band = torch.zeros((1, 16 * Mt, 3, 16 * Mt), dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError):
        plan.set_fill(band, 1)


def test_fill_takes_single_layer_plans_only_and_turns_off(bie, ggq):
    ctx = bie.Context()
    sp, Np, Mt, k = SPECS[0]
    s = bie.Surface(ctx, sp, Np, Mt, ggq)
    slot = 16 * 48 * Mt * Np
    W = torch.zeros((2, slot, Mt), dtype=torch.complex128, device="cuda")
    band = torch.zeros((1, 16 * Mt, 3, 16 * Mt), dtype=torch.complex128, device="cuda")
    plan_k = bie.Batch(ctx, [s], [k], bie.KERNEL_S | bie.KERNEL_K, W, slot)
    with pytest.raises(RuntimeError):
        plan_k.set_fill(band, 1)
    plan = bie.Batch(ctx, [s], [k], bie.KERNEL_S, W[:1], slot)
    plan.set_fill(band, 1)
    launches_with = plan.config["launches"]
    plan.set_fill(None, 0)
    assert plan.config["launches"] == launches_with - Np
    plan.run()
    ctx.sync()
