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
    # two calls in a row: a larger field first, then a smaller one that reuses part of the array
    for Lx, Lz in [(256, 128), (64, 32)]:
        phi = torch.from_numpy(rng.standard_normal((Lz, Lx))).cuda()
        want = torch.empty_like(phi)
        got = torch.full_like(phi, float("nan"))
        capi.lb_power_spectrum(phi.data_ptr(), Lx, Lz, want.data_ptr(), stream)
        capi.lb_power_spectrum_noalloc(phi.data_ptr(), Lx, Lz, got.data_ptr(), stream)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-12 * w.max())


def test_noalloc_spectrum_rejects_sizes_beyond_its_array():
    import torch
    buf = torch.zeros(2 * capi.LB_NOALLOC_MAX_POINTS, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.LBError) as e:
        capi.lb_power_spectrum_noalloc(buf.data_ptr(), 1024, 512, buf.data_ptr())
    assert e.value.code == capi.LB_ERR_SIZE
