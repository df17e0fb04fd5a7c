"""fr3d_fwd_apply_noalloc (static scratch, no device allocation) against fr3d_fwd_apply.

The entry point exists for callers that may not allocate device memory when they apply the
operator (allocator-free real-time loops, frameworks that own all device memory).  This file is
collected last so that a failure here leaves every other test run.
"""

import ctypes as ct

import numpy as np
import pytest

from paper_1703_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    from paper_1703_01216_gb300 import build, fr3d
    assert torch.cuda.is_available()
    build.build()
    return fr3d, fr3d.load()


def _p(t):
    return ct.c_void_p(t.data_ptr())


def test_fwd_apply_noalloc_matches_allocating_entry_point_twice():
    fr3d, lib = _lib()
    w = I.make_workload(64, 8, q=2, seed=901)
    # one handle for the allocating entry point, another used only by the allocation-free one (its
    # workspace is never created, so nothing can fall back on it)
    H_ref = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    H = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    rng = np.random.default_rng(902)
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    zetas = [torch.as_tensor(rng.standard_normal((2, 8, 64, 64)), dtype=torch.float32, device="cuda")
             for _ in range(2)]
    refs = [torch.empty((2, 1, 64, 64), device="cuda") for _ in range(2)]
    gots = [torch.full((2, 1, 64, 64), float("nan"), device="cuda") for _ in range(2)]
    warm = torch.empty_like(gots[0])
    for z, r in zip(zetas, refs):
        assert lib.fr3d_fwd_apply(H_ref.ptr, _p(z), 2, _p(r), fr3d.PREC_FP32, st) == 0
    # the first call on the device looks up the scratch address and loads the kernels
    assert lib.fr3d_fwd_apply_noalloc(H.ptr, _p(zetas[0]), 2, _p(warm), st) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for call in range(2):                       # two calls in a row: the shared scratch is reused
        assert lib.fr3d_fwd_apply_noalloc(H.ptr, _p(zetas[call]), 2, _p(gots[call]), st) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0                       # no device memory was taken by the calls
    for call in range(2):
        r, g = refs[call].double().cpu().numpy(), gots[call].double().cpu().numpy()
        assert np.isfinite(g).all()
        assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r), call


def test_fwd_apply_noalloc_size_limit_accepts_the_boundary_and_rejects_beyond():
    fr3d, lib = _lib()
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(904)
    # n = 256: 8 (M' + M) 129 * 256 bytes; M' + M = 15 fits in 4 MiB, 16 does not
    w = I.make_workload(256, 14, q=1, seed=903)
    H_ref = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    H = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    z = torch.as_tensor(rng.standard_normal((1, 14, 256, 256)), dtype=torch.float32, device="cuda")
    ref = torch.empty((1, 1, 256, 256), device="cuda")
    got = torch.full((1, 1, 256, 256), float("nan"), device="cuda")
    assert lib.fr3d_fwd_apply(H_ref.ptr, _p(z), 1, _p(ref), fr3d.PREC_FP32, st) == 0
    assert lib.fr3d_fwd_apply_noalloc(H.ptr, _p(z), 1, _p(got), st) == 0
    torch.cuda.synchronize()
    r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
    assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r)
    w2 = I.make_workload(256, 15, q=1, seed=905)
    H2 = fr3d.kernel_transform(w2.n, w2.x0, w2.h, w2.zr, w2.zy, w2.nu)
    z2 = torch.zeros((1, 15, 256, 256), device="cuda")
    assert lib.fr3d_fwd_apply_noalloc(H2.ptr, _p(z2), 1, _p(got), st) == -3
