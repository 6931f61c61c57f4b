"""Initialisation with the Leray-projected perturbation (option MCLBM_OPT_LERAY, Sec.
"Discretization and well-prepared initial data") against the oracle (FFT projection), the
divergence of the initial velocity, and the FP64 gradient with respect to the 24 parameters
against the oracle's complex step through the projected initialisation."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_populations
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


@pytest.mark.parametrize("steps", [0, 5])
def test_fp64_leray_init_and_steps_match_oracle(steps):
    N, M, Re, Ma = 16, 3, 400.0, 0.1
    X = gen.draw_params(21, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", leray=True).init(X).step(steps)
    un = oracle.units(N, Re, Ma)
    f = oracle.init_ensemble_leray(N, X, un["ulat"])
    oracle.run(f, un["omega"], steps)
    assert np.max(np.abs(lib_populations(ens) - f) / np.abs(f)) <= 1e-12
    np.testing.assert_array_equal(ens.params(), X)  # the parameters stay the coefficients of s


def test_initial_velocity_is_divergence_free_with_the_option():
    N, M = 32, 2
    X = gen.draw_params(22, M)
    k = np.fft.fftfreq(N, d=1.0 / N)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    divs = []
    for leray in (False, True):
        ens = Ensemble(N, M, Re=400.0, Ma=0.05, precision="fp64", leray=leray).init(X)
        u = ens.moments(1)[1].cpu().numpy()
        h = np.fft.fftn(u, axes=(-3, -2, -1))
        divs.append(np.abs(KX * h[0] + KY * h[1] + KZ * h[2]).max() / np.abs(h).max())
    assert divs[1] <= 1e-12 < divs[0]


def test_fp64_gradient_with_leray_matches_oracle_complex_step():
    N, M, Re, Ma, T, K = 16, 2, 200.0, 0.1, 10, 4
    X = gen.draw_params(23, M)
    un = oracle.units(N, Re, Ma)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", leray=True).init(X)
    need = mclbm.mclbm_grad_required_bytes(ens.ctx, T, K)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    J, G = mclbm.mclbm_grad(ens.ctx, 0, T, K, (buf.data_ptr() + 255) // 256 * 256, need, M)
    h = 1e-30
    ref = np.zeros((M, 24))
    for k in range(24):
        p = X.astype(np.complex128)
        p[:, k] += 1j * h
        f = oracle.init_ensemble_leray(N, p, un["ulat"], cplx=True)
        oracle.run(f, un["omega"], T)
        _, u = oracle.moments(f)
        E, _ = oracle.energy(u, un["ulat"])
        ref[:, k] = E.imag / h
    assert np.max(np.abs(G - ref)) <= 1e-8 * np.abs(ref).max()
