"""The one-snapshot power spectrum (Appendix A on the lattice) through the C interface,
against the oracle's O(n^2) transform, on device buffers supplied by torch."""
import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Lx,Lz", [(2, 2), (8, 4), (64, 32), (256, 16), (16, 128)])
def test_power_spectrum_matches_oracle(Lx, Lz):
    import torch
    rng = np.random.default_rng(Lx * 1000 + Lz)
    phi = rng.standard_normal((Lz, Lx))
    dev = torch.from_numpy(phi).cuda()
    out = torch.empty_like(dev)
    s = torch.cuda.current_stream()
    capi.lb_power_spectrum(dev.data_ptr(), Lx, Lz, out.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    want = oracle.dft2_power(phi)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-12 * want.max())


def test_power_spectrum_rejects_host_memory_and_bad_sizes():
    import torch
    dev = torch.zeros(64, dtype=torch.float64, device="cuda")
    host = np.zeros(64)
    with pytest.raises(capi.LBError):
        capi.lb_power_spectrum(host.ctypes.data, 8, 8, dev.data_ptr())
    with pytest.raises(capi.LBError):
        capi.lb_power_spectrum(dev.data_ptr(), 8, 6, dev.data_ptr())
    with pytest.raises(capi.LBError):
        capi.lb_power_spectrum(dev.data_ptr(), 1, 64, dev.data_ptr())
