"""C-ABI checks that need no GPU: the library loads and exports every entry point
include/*.h declares; host-side logic (units, validation, sizes, the Philox draw,
the velocity set) agrees with the oracle and the paper's tables."""
import glob
import os
import re

import numpy as np
import pytest

import ensemble_inputs as gen
import oracle
from paper_2608_23786_gb300 import mclbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return mclbm.load(build_if_missing=True)


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"MCLBM_API\s+[\w\s\*]+?\b(mclbm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared entry points
    assert set(mclbm.declared_symbols()) == declared


def test_lattice_matches_oracle_set(lib):
    c, w = mclbm.mclbm_lattice()
    co, wo, _ = oracle.lattice()
    lib_set = {tuple(v): wi for v, wi in zip(c.tolist(), w)}
    orc_set = {tuple(v): wi for v, wi in zip(co.tolist(), wo)}
    assert lib_set == orc_set
    # storage order: rest, then opposite pairs
    for i in range(1, 19, 2):
        assert (c[i] == -c[i + 1]).all()


def _cfg(N=64, M=4, Re=800.0, Ma=0.025, precision=mclbm.FP32, pattern=mclbm.PULL, dt=0.0):
    return mclbm.Config(N=N, M=M, precision=precision, pattern=pattern, nu=1.0 / Re, Ma=Ma, dt=dt, U_c=1.0,
                        width=0.025, seed=1, init_density=0, options=0)


@pytest.mark.parametrize("N,Re,Ma", [(32, 1280, 0.05), (64, 2560, 0.025), (512, 20480, 0.003125), (64, 800, 0.025)])
def test_units_match_oracle(lib, N, Re, Ma):
    u = mclbm.mclbm_compute_units(_cfg(N=N, Re=Re, Ma=Ma)).as_dict()
    o = oracle.units(N, Re, Ma)
    for k_lib, k_orc in (("dx", "dx"), ("U_lat", "ulat"), ("dt", "dt"), ("nu_lat", "nu_lat"), ("tau", "tau"),
                         ("omega", "omega")):
        assert abs(u[k_lib] - o[k_orc]) <= 1e-14 * abs(o[k_orc]), k_lib


def test_units_from_dt(lib):
    """dt given instead of Ma: U_lat = dt U_c / dx."""
    o = oracle.units(64, 2560, 0.025)
    u = mclbm.mclbm_compute_units(_cfg(N=64, Re=2560, Ma=0.0, dt=o["dt"])).as_dict()
    assert abs(u["U_lat"] - o["ulat"]) <= 1e-15 and abs(u["tau"] - o["tau"]) <= 1e-15


def test_validation_errors(lib):
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_compute_units(_cfg(N=48))
    assert e.value.status == "SHAPE"
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_compute_units(mclbm.Config(N=32, M=1, precision=1, pattern=0, nu=-1e-3, Ma=0.1, dt=0, U_c=1,
                                               width=0.025, seed=0, init_density=0, options=0))
    assert e.value.status == "UNSTABLE_TAU"
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_compute_units(_cfg(precision=7))
    assert e.value.status == "INVALID_ARG"
    assert "precision" in mclbm.mclbm_last_error()


@pytest.mark.parametrize("prec,b", [(mclbm.FP64, 8), (mclbm.FP32, 4), (mclbm.FP16, 2)])
@pytest.mark.parametrize("pattern,k", [(mclbm.PULL, 2), (mclbm.AA, 1)])
def test_required_bytes(lib, prec, b, pattern, k):
    pop, work = mclbm.mclbm_required_bytes(_cfg(N=64, M=64, precision=prec, pattern=pattern))
    assert pop == k * 19 * b * 64**3 * 64
    # statistics of two samples at a time: two velocity fields (one sample's u_z kept beside the
    # other's field) + complex FFT buffer + two power spectra
    assert work >= 64**3 * (32 + 16 + 16)
    # 512^3 x 4 FP16 AA: 38 bytes per node
    pop, _ = mclbm.mclbm_required_bytes(_cfg(N=512, M=4, Re=6400, Ma=0.003125, precision=mclbm.FP16,
                                             pattern=mclbm.AA))
    assert pop == 38 * 512**3 * 4


def test_philox_draw_matches_numpy_philox(lib):
    """The library's Philox4x64-10 parameter draw is bit-identical to numpy's Philox with the
    counter convention (b, m, 0, 0)."""
    for seed in (0, 1, 12345, 2**63 + 7):
        A = mclbm.mclbm_draw_params(seed, 0, 9)
        B = gen.draw_params(seed, 9)
        np.testing.assert_array_equal(A, B)
        np.testing.assert_array_equal(mclbm.mclbm_draw_params(seed, 4, 3), B[4:7])


def test_d3q27_library_exports_the_same_abi(lib):
    """libmclbm_d3q27.so: the same entry points, the D3Q27 set (matching the oracle's), and
    27 populations per node in the sizes."""
    lib27 = mclbm.load(lattice=27)
    for name in _declared():
        assert hasattr(lib27, name), name
    c, w = mclbm.mclbm_lattice(27)
    co, wo, _ = oracle.lattice(27)
    assert {tuple(v): wi for v, wi in zip(c.tolist(), w)} == {tuple(v): wi for v, wi in zip(co.tolist(), wo)}
    for i in range(1, 27, 2):
        assert (c[i] == -c[i + 1]).all()
    pop, _ = mclbm.mclbm_required_bytes(_cfg(N=64, M=8, precision=mclbm.FP32, pattern=mclbm.PULL), lattice=27)
    assert pop == 2 * 27 * 4 * 64**3 * 8
    assert "D3Q27" in mclbm.mclbm_version(27) and "D3Q19" in mclbm.mclbm_version()


def test_leray_coefficient_map_against_fft_projection(lib):
    """mclbm_leray_params (host) maps the 24 coefficients of the perturbation to those of its
    Leray projection: evaluated on a 16^3 grid, L X reproduces the oracle's FFT projection of s;
    the transpose option is the matrix transpose; the map is a projection (L L = L)."""
    X = gen.draw_params(5, 3)
    Y = mclbm.mclbm_leray_params(X)
    _, s = oracle.rtgv_fields(16, X)
    _, s_y = oracle.rtgv_fields(16, Y)
    np.testing.assert_allclose(s_y, oracle.leray_project(s), rtol=0, atol=1e-15)
    np.testing.assert_allclose(mclbm.mclbm_leray_params(Y), Y, rtol=0, atol=1e-16)
    E = np.eye(24)
    L = mclbm.mclbm_leray_params(E).T  # column q = L e_q
    np.testing.assert_allclose(mclbm.mclbm_leray_params(E, transpose=True).T, L.T, atol=0)


def _cuda_present():
    import torch
    return torch.cuda.is_available()


@pytest.mark.skipif(_cuda_present(), reason="checks the failure without a GPU")
def test_no_gpu_fails_loudly(lib):
    """There is no CPU path: without a device, context creation reports the CUDA error (after the
    host-side checks, before any buffer is touched) and Ensemble refuses to start."""
    cfg = _cfg(N=16, M=2)
    pop, work = mclbm.mclbm_required_bytes(cfg)
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_create(cfg, 256, pop, 512, work)  # aligned stand-in addresses, never dereferenced
    assert e.value.status == "CUDA"
    assert "cudaGetDevice" in mclbm.mclbm_last_error()
    with pytest.raises(mclbm.MclbmError) as e:  # the host checks come first: a short buffer is OOM
        mclbm.mclbm_create(cfg, 256, pop - 1, 512, work)
    assert e.value.status == "OOM"
    from paper_2608_23786_gb300 import Ensemble
    with pytest.raises(RuntimeError, match="CUDA"):
        Ensemble(16, 2, Re=400.0, Ma=0.1)
