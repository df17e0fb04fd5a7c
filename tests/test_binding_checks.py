"""The Python binding checks every buffer before it reaches the C ABI (CPU only: the checks run before
any library call): residency (device or host, as the call expects), contiguity, dtype against the
call's precision and element counts against the handle's sizes."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    from paper_1703_01216_gb300 import fr3d
    try:
        fr3d.load()
    except RuntimeError:
        pytest.skip("libfr3d.so is not built")
    return fr3d


class _FakeHandle:
    """The sizes a Handle carries (n, M, M'), no device state: every call below must fail in the binding."""
    n, M, Mp, ptr = 16, 1, 4, None


def test_device_calls_reject_host_tensors(F):
    H = _FakeHandle()
    z = torch.zeros((1, 4, 16, 16))
    u = torch.zeros((1, 1, 16, 16))
    with pytest.raises(F.Fr3dError, match="device"):
        F.fwd_apply(H, z, 1, u)
    with pytest.raises(F.Fr3dError, match="device"):
        F.invert(H, u, 1, torch.zeros((4, 16, 16)), F.Opts(alpha=1e-2))
    with pytest.raises(F.Fr3dError, match="device"):
        F.choose_alpha(H, u, 1, [1e-3, 1e-2], 0.1, 1.1, torch.zeros(1, dtype=torch.int32))


def test_host_call_checks_dtype_size_contiguity_and_residency(F):
    H = _FakeHandle()
    U = torch.zeros((1, 1, 16, 16))
    out = torch.zeros((4, 16, 16))
    with pytest.raises(F.Fr3dError, match="elements"):                 # one depth short
        F.invert_host(H, U, 1, torch.zeros((3, 16, 16)), F.Opts(alpha=1e-2))
    with pytest.raises(F.Fr3dError, match="dtype"):                    # FP64 call, FP32 buffers
        F.invert_host(H, U, 1, out, F.Opts(alpha=1e-2, precision=F.PREC_FP64))
    with pytest.raises(F.Fr3dError, match="contiguous"):
        F.invert_host(H, torch.zeros((1, 1, 16, 32))[..., ::2], 1, out, F.Opts(alpha=1e-2))
    with pytest.raises(F.Fr3dError, match="elements"):                 # ZETA output: Q planes sets
        F.invert_host(H, torch.zeros((2, 1, 16, 16)), 2, out, F.Opts(alpha=1e-2, output=F.OUT_ZETA))
    with pytest.raises(F.Fr3dError, match="dtype"):
        F.invert_host(H, np.zeros((1, 1, 16, 16)), 1, out, F.Opts(alpha=1e-2))   # float64 array
    idx = torch.zeros(2, dtype=torch.int64)
    with pytest.raises(F.Fr3dError, match="device|dtype"):
        F.invert_host(H, U, 1, out, F.Opts(alphas=[1e-3, 1e-2], alpha_idx=idx, given=True))


def test_unet_and_raw_addresses(F):
    class _FakeNet(F.Unet):
        def __init__(self):
            self.shape, self.n_params, self.ptr = (8, 16, 16), 10, None
    net = _FakeNet()
    with pytest.raises(F.Fr3dError, match="device"):
        net.forward(torch.zeros((1, 8, 16, 16)), torch.zeros((1, 8, 16, 16)))
    # raw integer addresses are the caller's responsibility and pass the binding's checks
    F._need(1234, "x")
