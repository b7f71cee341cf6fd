"""lb_power_spectrum_noalloc, the spectrum for callers that cannot allocate device memory (for
instance while a CUDA graph is being captured by someone else, or when another framework owns
the device memory), through the C interface: it must give the same spectra as
lb_power_spectrum, which allocates its scratch, on consecutive calls that reuse its fixed
scratch array.  This file is collected last so that a failure here stops a run only after every
other test has run."""
import numpy as np
import pytest

from paper_1808_05168_gb300 import capi

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_allocating_one_on_consecutive_calls():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    # calls in a row: a field that fills the array, a smaller one that reuses part of it, and the
    # longest columns (8192 points, one per block)
    for Lx, Lz in [(256, 1024), (64, 32), (32, 8192), (2, 8192)]:
        phi = torch.from_numpy(rng.standard_normal((Lz, Lx))).cuda()
        want = torch.empty_like(phi)
        got = torch.full_like(phi, float("nan"))
        capi.lb_power_spectrum(phi.data_ptr(), Lx, Lz, want.data_ptr(), stream)
        capi.lb_power_spectrum_noalloc(phi.data_ptr(), Lx, Lz, got.data_ptr(), stream)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-12 * w.max())


def test_noalloc_spectrum_rejects_sizes_beyond_its_array():
    """More points than the fixed array holds: LB_ERR_SIZE; a transform longer than 8192 points
    (which lb_power_spectrum rejects too): LB_ERR_BAD_PARAM, before anything is launched."""
    import torch
    a = torch.zeros(2 * capi.LB_NOALLOC_MAX_POINTS, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(capi.LBError) as e:
        capi.lb_power_spectrum_noalloc(a.data_ptr(), 1024, 512, b.data_ptr())
    assert e.value.code == capi.LB_ERR_SIZE
    for Lx, Lz in [(16384, 16), (16, 16384)]:
        with pytest.raises(capi.LBError) as e:
            capi.lb_power_spectrum_noalloc(a.data_ptr(), Lx, Lz, b.data_ptr())
        assert e.value.code == capi.LB_ERR_BAD_PARAM, (Lx, Lz)
