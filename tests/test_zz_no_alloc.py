"""The W1 entry point that allocates nothing (for callers that cannot allocate device
memory: another allocator owns the GPU's memory, cudaFree's device-wide synchronisation
is not acceptable, or there is no memory to spare) must give the same result as the
entry point that takes a caller work buffer, on consecutive calls that reuse its fixed
scratch array.  This file is collected last so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh process, where
its first call is the one that looks up the scratch array on the device."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
from paper_2608_23786_gb300 import mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _with_work_buffer(a, MA, b, MB, G):
    work = torch.empty(mclbm.mclbm_w1_work_bytes(MA, MB, G), dtype=torch.uint8, device="cuda")
    pp = np.zeros((G, 3))
    W = mclbm.mclbm_w1_restricted(a.data_ptr(), MA, b.data_ptr(), MB, G, work.data_ptr(), work.numel(),
                                  per_point=pp)
    return W, pp


def test_noalloc_w1_matches_work_buffer_entry_point_on_consecutive_calls():
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(33, 17, 512, 70), (64, 64, 4096, 71)]  # (MA, MB, G, seed): the second call reuses the scratch
    for MA, MB, G, seed in cases:
        a = torch.as_tensor(gen.normal(seed, (MA, G, 3)), device="cuda")
        b = torch.as_tensor(gen.normal(seed + 100, (MB, G, 3)) + 0.05, device="cuda")
        W_ref, pp_ref = _with_work_buffer(a, MA, b, MB, G)
        pp = np.zeros((G, 3))
        W = mclbm.mclbm_w1_restricted_noalloc(a.data_ptr(), MA, b.data_ptr(), MB, G, stream, per_point=pp)
        assert abs(W - W_ref) <= 1e-12 * abs(W_ref)
        np.testing.assert_allclose(pp, pp_ref, rtol=1e-12, atol=0)
        # without per-point output as well
        W2 = mclbm.mclbm_w1_restricted_noalloc(a.data_ptr(), MA, b.data_ptr(), MB, G, stream)
        assert abs(W2 - W_ref) <= 1e-12 * abs(W_ref)


def test_noalloc_w1_rejects_more_points_than_its_scratch_holds():
    a = torch.zeros((2, 4097, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_w1_restricted_noalloc(a.data_ptr(), 2, a.data_ptr(), 2, 4097)
    assert e.value.status == "SHAPE" and "4096" in str(e.value)


def test_noalloc_w1_default_stream_is_torch_current_stream():
    """Without an explicit stream the wrapper passes torch's current stream, so inputs filled on a
    torch side stream (created non-blocking) are ordered before the call."""
    MA, MB, G = 40, 24, 512
    a0 = torch.as_tensor(gen.normal(72, (MA, G, 3)), device="cuda")
    b0 = torch.as_tensor(gen.normal(172, (MB, G, 3)) + 0.1, device="cuda")
    W_ref, _ = _with_work_buffer(a0, MA, b0, MB, G)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        a = torch.empty_like(a0)
        b = torch.empty_like(b0)
        a.copy_(a0)
        b.copy_(b0)
        W = mclbm.mclbm_w1_restricted_noalloc(a.data_ptr(), MA, b.data_ptr(), MB, G)
    assert abs(W - W_ref) <= 1e-12 * abs(W_ref)
