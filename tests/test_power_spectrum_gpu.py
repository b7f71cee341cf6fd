"""The one-snapshot power spectrum (Appendix A on the lattice) through the C interface,
against the oracle's O(n^2) transform, on device buffers supplied by torch."""
import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Lx,Lz", [(2, 2), (8, 4), (64, 32), (256, 16), (16, 128), (2, 8192), (32, 8192),
                                   (8192, 2)])
def test_power_spectrum_matches_oracle(Lx, Lz):
    """Every size class of the two passes: the largest transforms along z (8192 points, one column
    per block in 196,608 bytes of shared memory) and along x (8192-point rows)."""
    import torch
    rng = np.random.default_rng(Lx * 1000 + Lz)
    phi = rng.standard_normal((Lz, Lx))
    dev = torch.from_numpy(phi).cuda()
    out = torch.empty_like(dev)
    s = torch.cuda.current_stream()
    capi.lb_power_spectrum(dev.data_ptr(), Lx, Lz, out.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    want = oracle.dft2_power(phi, omp=True)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-12 * want.max())


def test_power_spectrum_rejects_host_memory_and_bad_sizes():
    """Host memory (pageable or pinned), sizes that are not powers of two in 2..8192: rejected with
    LB_ERR_BAD_PARAM before anything is launched.  (Memory of another device is rejected the same
    way; a one-GPU machine cannot make such a pointer.)"""
    import torch
    dev = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    host = np.zeros(64)
    pinned = torch.zeros(64, dtype=torch.float64).pin_memory()
    for args in [(host.ctypes.data, 8, 8, dev.data_ptr()), (pinned.data_ptr(), 8, 8, dev.data_ptr()),
                 (dev.data_ptr(), 8, 8, pinned.data_ptr()), (dev.data_ptr(), 8, 6, dev.data_ptr()),
                 (dev.data_ptr(), 1, 64, dev.data_ptr()), (dev.data_ptr(), 16384, 2, dev.data_ptr()),
                 (dev.data_ptr(), 2, 16384, dev.data_ptr())]:
        with pytest.raises(capi.LBError) as e:
            capi.lb_power_spectrum(*args)
        assert e.value.code == capi.LB_ERR_BAD_PARAM, args
