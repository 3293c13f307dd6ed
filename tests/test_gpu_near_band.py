"""Correction stage written as the near band alone (the band layout of bie_assemble_near_band):
the same entries as the correction stage adds to a zero dense matrix, bit for bit, whether the band
goes to device memory or, staged a group of target panels at a time, to page-locked host memory;
and the band rows against the oracle's operator rows (near blocks only)."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import nystrom as ny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bie():
    import paper_2608_16208_b300 as b
    return b


@pytest.fixture(scope="module")
def ctx(bie):
    return bie.Context()


def dense_to_band(A, Np, Mt):
    """Band [N, 3, 16 Mt] of a dense matrix: slot d holds the columns of source panel (target panel + d - 1)."""
    N, w = A.shape[0], 16 * Mt
    band = torch.zeros((N, 3, w), dtype=A.dtype, device=A.device)
    for j in range(Np):
        for d in range(3):
            jp = j + d - 1
            if 0 <= jp < Np:
                band[j * w:(j + 1) * w, d] = A[j * w:(j + 1) * w, jp * w:(jp + 1) * w]
    return band


@pytest.mark.parametrize("kernels,ws,wk", [("S", 1.0, 0.0), ("SK", 0.3 - 1.1j, 0.7 + 0.4j)])
@pytest.mark.parametrize("surface,Np,Mt,k", [(wl.sphere(), 4, 32, 1.0), (wl.ellipsoid(1.0, 0.8, 0.6), 5, 48, 4.0)])
def test_band_equals_dense_correction(bie, ctx, ggq, surface, Np, Mt, k, kernels, ws, wk):
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    km = bie.KERNEL_S | (bie.KERNEL_K if "K" in kernels else 0)
    A = torch.zeros((s.N, s.N), dtype=torch.complex128, device="cuda")
    bie.assemble_near(s, km, k, A, ws=ws, wk=wk)
    dev = bie.assemble_near_band(s, km, k, ws=ws, wk=wk)
    host = bie.assemble_near_band(s, km, k, ws=ws, wk=wk, host=True)
    ctx.sync()
    ref = dense_to_band(A, Np, Mt)
    assert torch.equal(dev, ref)
    assert torch.equal(host, ref.cpu())
    assert torch.all(dev[: 16 * Mt, 0] == 0) and torch.all(dev[-16 * Mt:, 2] == 0)


def test_band_rows_match_oracle(bie, ctx, ggq):
    surface, Np, Mt, k = wl.bumpy(), 4, 64, 3.0
    s = bie.Surface(ctx, surface, Np, Mt, ggq)
    band = bie.assemble_near_band(s, bie.KERNEL_S, k, host=True)
    ctx.sync()
    rows = np.unique(np.concatenate([wl.sample_rows(Np, Mt, 24), [0, s.N - 1, 16 * Mt - 1, 16 * Mt]]))
    ref = ny.operator_rows(surface, Np, Mt, k, ggq[0], ggq[1], rows, op="S")
    w = 16 * Mt
    for r, rr in zip(rows, ref):
        j = r // w
        for d in range(3):
            jp = j + d - 1
            got = band[r, d].numpy()
            if 0 <= jp < Np:
                want = rr[jp * w:(jp + 1) * w]
                assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), (r, d)
            else:
                assert not np.any(got)


def test_band_overwrites_and_refuses_pageable_memory(bie, ctx, ggq):
    s = bie.Surface(ctx, wl.sphere(), 4, 32, ggq)
    first = bie.assemble_near_band(s, bie.KERNEL_S, 1.0, host=True)
    ctx.sync()
    out = torch.full((s.N, 3, 16 * 32), 7.0 + 7.0j, dtype=torch.complex128).pin_memory()
    bie.assemble_near_band(s, bie.KERNEL_S, 1.0, out=out)
    ctx.sync()
    assert torch.equal(out, first)
    pageable = torch.empty((s.N, 3, 16 * 32), dtype=torch.complex128)
    with pytest.raises(bie.BieError, match="pageable"):
        bie.assemble_near_band(s, bie.KERNEL_S, 1.0, out=pageable)
