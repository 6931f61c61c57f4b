"""Eq. (sample_error) on the GPU against the oracle, on paired RTGV ensembles (the same
parameters at 16^3 and 32^3 after the same physical time), and the EOSC slope pipeline."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
from oracle import stats
from paper_2608_23786_gb300 import Ensemble, convergence, mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def test_sample_error_matches_oracle_on_paired_ensembles():
    X = gen.draw_params(17, 6)
    # diffusive scaling: 4x the steps at twice the resolution reaches the same physical time
    runs = [Ensemble(N, 6, Re=400.0, Ma=0.8 / N, precision="fp32").init(X).step(6 * (N // 8) ** 2) for N in (16, 32, 64)]
    ref = runs[-1]
    errs = []
    for e in runs[:-1]:
        got = e.sample_error(ref, Q=8)
        want = stats.sample_error(e.restrict(8).cpu().numpy(), ref.restrict(8).cpu().numpy())
        np.testing.assert_allclose(got, want, rtol=1e-13)
        errs.append(got[3])
    assert errs[1] < errs[0]  # the coarser run is further from the reference
    assert convergence.eoc_slope([16, 32], errs) < 0


def test_sample_error_work_buffer_check():
    u = torch.zeros((4, 8, 3), dtype=torch.float64, device="cuda")
    nb = mclbm.mclbm_sample_error_work_bytes(4)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_sample_error(u.data_ptr(), u.data_ptr(), 4, 8, work.data_ptr(), nb - 8)
    assert e.value.status == "OOM"

