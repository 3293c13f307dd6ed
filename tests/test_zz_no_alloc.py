"""The allocation-free kernel-modes entry point, for callers that cannot call
cudaMalloc (another allocator holds the device, or the implicit synchronisation
of an allocation is not acceptable).  Called through the C ABI; its output must
match bie_kernel_modes on two calls in a row (the static scratch is shared and
keeps the previous call's contents)."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as wl
from tests.pairs import sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def test_noalloc_matches_kernel_modes_twice(ggq):
    import paper_2608_16208_b300 as bie
    ctx = bie.Context()
    # the last case fills the static scratch: Mth = 128 with the double layer (L = 256)
    for surface, Np, Mt, k, kern in [(wl.ellipsoid(1.0, 0.8, 0.6), 16, 128, 10.0, bie.KERNEL_S),
                                      (wl.bumpy(), 6, 96, 5.0, bie.KERNEL_S | bie.KERNEL_K),
                                      (wl.bumpy(), 8, 128, 20.0, bie.KERNEL_S | bie.KERNEL_K)]:
        s = bie.Surface(ctx, surface, Np, Mt, ggq)
        rows, srcs = sample_pairs(Np, Mt, 3000, seed=4)
        r = torch.from_numpy(rows).cuda()
        c = torch.from_numpy(srcs).cuda()
        nk = bin(kern).count("1")
        ref = bie.kernel_modes(s, kern, k, r, c)
        ctx.sync()
        for call in range(2):
            out = torch.full((len(rows), nk, Mt + 1), complex("nan"), dtype=torch.complex128, device="cuda")
            st = bie.lib.bie_kernel_modes_noalloc(ctx.h, s.h, kern, ctypes.c_double(k), ctypes.c_void_p(r.data_ptr()),
                                                  ctypes.c_void_p(c.data_ptr()), len(rows),
                                                  ctypes.c_void_p(out.data_ptr()))
            assert st == 0, bie.lib.bie_last_error().decode()
            ctx.sync()
            g, f = out.cpu().numpy(), ref.cpu().numpy()
            err = np.max(np.abs(g - f), axis=-1) / np.max(np.abs(f), axis=-1)
            assert np.all(np.isfinite(g)) and err.max() <= TOL, (call, err.max())


def test_noalloc_rejects_oversized_grid(ggq):
    import paper_2608_16208_b300 as bie
    ctx = bie.Context()
    s = bie.Surface(ctx, wl.sphere(), 2, 192, ggq)
    r = torch.zeros(1, dtype=torch.int64, device="cuda")
    c = torch.full((1,), 16, dtype=torch.int32, device="cuda")
    out = torch.empty((1, 1, 193), dtype=torch.complex128, device="cuda")
    st = bie.lib.bie_kernel_modes_noalloc(ctx.h, s.h, bie.KERNEL_S, ctypes.c_double(1.0),
                                          ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(c.data_ptr()), 1,
                                          ctypes.c_void_p(out.data_ptr()))
    assert st == 1 and b"maximum" in bie.lib.bie_last_error()
