"""fr3d_fwd_apply_noalloc (static scratch, no device allocation) against fr3d_fwd_apply.

The entry point exists for callers that may not allocate device memory when they apply the
operator (graph capture in progress, allocator-free real-time loops, frameworks that own all
device memory).  This file is collected last so that a failure here leaves every other test run.
"""

import ctypes as ct

import numpy as np
import pytest

from paper_1703_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fwd_apply_noalloc_matches_allocating_entry_point_twice():
    from paper_1703_01216_gb300 import build, fr3d
    assert torch.cuda.is_available()
    build.build()
    lib = fr3d.load()
    w = I.make_workload(64, 8, q=2, seed=901)
    H = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    rng = np.random.default_rng(902)
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):                       # two calls in a row: the shared scratch is reused
        zeta = torch.as_tensor(rng.standard_normal((2, 8, 64, 64)), dtype=torch.float32, device="cuda")
        ref = torch.empty((2, 1, 64, 64), device="cuda")
        got = torch.full((2, 1, 64, 64), float("nan"), device="cuda")
        assert lib.fr3d_fwd_apply(H.ptr, ct.c_void_p(zeta.data_ptr()), 2, ct.c_void_p(ref.data_ptr()),
                                  fr3d.PREC_FP32, st) == 0
        assert lib.fr3d_fwd_apply_noalloc(H.ptr, ct.c_void_p(zeta.data_ptr()), 2, ct.c_void_p(got.data_ptr()),
                                          st) == 0
        torch.cuda.synchronize()
        r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
        assert np.isfinite(g).all()
        assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r), call


def test_fwd_apply_noalloc_rejects_requests_beyond_its_scratch():
    from paper_1703_01216_gb300 import build, fr3d
    build.build()
    lib = fr3d.load()
    w = I.make_workload(256, 32, q=1, seed=903)             # 33 half spectra of 256 x 129: 8.7 MB > 4 MiB
    H = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    z = torch.zeros((1, 32, 256, 256), device="cuda")
    u = torch.zeros((1, 1, 256, 256), device="cuda")
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.fr3d_fwd_apply_noalloc(H.ptr, ct.c_void_p(z.data_ptr()), 1, ct.c_void_p(u.data_ptr()), st) == -3
