"""Failure detection without any GPU fault (a bounded wait that runs out, a non-finite
population planted through the C ABI) and checkpoint / resume."""
import os

import numpy as np
import pytest
import torch

import ensemble_inputs as gen
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    ens = Ensemble(16, 2, Re=100.0, Ma=0.1, precision="fp32").init()
    mclbm.mclbm_device_status(ens.ctx)
    mclbm.mclbm_selftest_timeout(ens.ctx)
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_device_status(ens.ctx)
    assert e.value.status == "TIMEOUT"
    # the context keeps working: re-initialise (clears the status) and step
    ens.init().step(3)
    mclbm.mclbm_device_status(ens.ctx)
    assert np.all(np.isfinite(ens.energy()))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_nonfinite_population_is_detected(precision):
    ens = Ensemble(8, 2, Re=100.0, Ma=0.1, precision=precision).init().step(2)
    ens.check_finite()
    f = ens.populations(1)
    f[3, 2, 5, 1] = float("nan")
    ens.set_populations(f, 1)
    with pytest.raises(mclbm.MclbmError) as e:
        ens.check_finite()
    assert e.value.status == "NONFINITE"


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_checkpoint_resume_is_bitwise(tmp_path, pattern):
    """Save after 5 steps (odd: AA parity and pull lattice index must round-trip), restore into a
    fresh context, continue 7 steps: bit-identical to an uninterrupted 12-step run."""
    X = gen.draw_params(14, 3)
    a = Ensemble(16, 3, Re=300.0, Ma=0.1, precision="fp32", pattern=pattern).init(X).step(5)
    path = os.path.join(tmp_path, "state.mclbm")
    mclbm.mclbm_save(a.ctx, path)
    a.step(7)
    b = Ensemble(16, 3, Re=300.0, Ma=0.1, precision="fp32", pattern=pattern).init()
    mclbm.mclbm_load(b.ctx, path)
    assert b.steps_taken == 5
    np.testing.assert_array_equal(b.params(), X)
    b.step(7)
    for m in range(3):
        assert torch.equal(a.populations(m), b.populations(m))
    wrong = Ensemble(8, 3, Re=300.0, Ma=0.1, precision="fp32", pattern=pattern).init()
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_load(wrong.ctx, path)
    assert e.value.status == "SHAPE"
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_load(b.ctx, os.path.join(tmp_path, "missing.mclbm"))
    assert e.value.status == "IO"


def test_checkpoint_rejects_other_dynamics_and_trailing_bytes(tmp_path):
    """A checkpoint restores only into a context with the same lattice, units and options: one
    taken at another Reynolds number, with the exact-gamma option, or by the D3Q27 library is
    rejected (SHAPE), and a file with bytes after the lattice is not taken for a checkpoint (IO)."""
    a = Ensemble(16, 2, Re=300.0, Ma=0.1, precision="fp32").init().step(3)
    path = os.path.join(tmp_path, "a.mclbm")
    mclbm.mclbm_save(a.ctx, path)
    for other in (Ensemble(16, 2, Re=600.0, Ma=0.1, precision="fp32").init(),
                  Ensemble(16, 2, Re=300.0, Ma=0.05, precision="fp32").init(),
                  Ensemble(16, 2, Re=300.0, Ma=0.1, precision="fp32", exact_gamma=True).init()):
        with pytest.raises(mclbm.MclbmError) as e:
            mclbm.mclbm_load(other.ctx, path)
        assert e.value.status == "SHAPE"
    padded = os.path.join(tmp_path, "padded.mclbm")
    with open(path, "rb") as f, open(padded, "wb") as g:
        g.write(f.read() + b"\0" * 8)
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_load(a.ctx, padded)
    assert e.value.status == "IO"
    truncated = os.path.join(tmp_path, "truncated.mclbm")
    with open(path, "rb") as f, open(truncated, "wb") as g:
        g.write(f.read()[:-4])
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_load(a.ctx, truncated)
    assert e.value.status == "IO"
    # the D3Q27 library's checkpoint (same N, M, units) does not load into the D3Q19 library
    mclbm.load(lattice=27, build_if_missing=True)
    b27 = Ensemble(16, 2, Re=300.0, Ma=0.1, precision="fp32", lattice=27).init().step(3)
    p27 = os.path.join(tmp_path, "b27.mclbm")
    mclbm.mclbm_save(b27.ctx, p27)
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_load(a.ctx, p27)
    assert e.value.status == "SHAPE"
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_load(b27.ctx, path)
    assert e.value.status == "SHAPE"
    mclbm.mclbm_load(a.ctx, path)  # its own file still loads
    assert a.steps_taken == 3
