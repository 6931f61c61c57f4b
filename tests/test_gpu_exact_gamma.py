"""The exact entropic gamma (option MCLBM_OPT_EXACT_GAMMA, Eq. (kbc_entropy)) on the GPU
(safeguarded Newton / Halley) against the oracle's exact gamma (bisection): FP64 per population,
FP32 and FP16 velocity error, D3Q27, and the option's launch and adjoint rules."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_populations, rel_l2
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)
    mclbm.load(build_if_missing=True, lattice=27)


def _oracle_exact(N, X, Re, Ma, steps, lattice=19):
    un = oracle.units(N, Re, Ma)
    f = oracle.init_ensemble(N, X, un["ulat"], lattice=lattice)
    with oracle.exact_gamma():
        oracle.run(f, un["omega"], steps)
    return f, un


@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("steps", [1, 5, 20])
def test_fp64_exact_gamma_parity(pattern, steps):
    N, M, Re, Ma = 16, 3, 400.0, 0.1
    X = gen.draw_params(61, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", pattern=pattern, exact_gamma=True).init(X).step(steps)
    assert mclbm.mclbm_get_launch(ens.ctx)[0] == 6
    f, _ = _oracle_exact(N, X, Re, Ma, steps)
    assert np.max(np.abs(lib_populations(ens) - f) / np.abs(f)) <= 1e-12


def test_exact_gamma_changes_the_dynamics():
    """The exact and closed-form gamma give states that differ beyond rounding (second order in
    the non-equilibrium), while both conserve mass."""
    N, M, Re, Ma, steps = 16, 2, 400.0, 0.1, 20
    X = gen.draw_params(62, M)
    a = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", exact_gamma=True).init(X).step(steps)
    b = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64").init(X).step(steps)
    fa, fb = a.populations(0), b.populations(0)
    assert (fa - fb).abs().max().item() > 1e-10
    assert abs(fa.sum().item() - fb.sum().item()) <= 1e-12 * fb.sum().item()


def test_fp32_exact_gamma_velocity_error():
    N, M, Re, Ma, steps = 32, 2, 800.0, 0.025, 100
    X = gen.draw_params(63, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", exact_gamma=True).init(X).step(steps)
    f, un = _oracle_exact(N, X, Re, Ma, steps)
    _, u = oracle.moments(f)
    got = np.stack([ens.moments(m)[1].cpu().numpy() for m in range(M)])
    assert rel_l2(got, u / un["ulat"]) <= 1e-5


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_fp32_exact_gamma_velocity_error_ma01(pattern):
    """Larger deviations (Ma 0.1: |f*/w - 1| up to a few tenths) and both streaming patterns."""
    N, M, Re, Ma, steps = 16, 2, 400.0, 0.1, 40
    X = gen.draw_params(65, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", pattern=pattern, exact_gamma=True).init(X).step(steps)
    f, un = _oracle_exact(N, X, Re, Ma, steps)
    _, u = oracle.moments(f)
    got = np.stack([ens.moments(m)[1].cpu().numpy() for m in range(M)])
    assert rel_l2(got, u / un["ulat"]) <= 1e-5


def test_fp16_exact_gamma_velocity_error():
    """FP16 storage with the exact gamma (collided in FP32): the storage rounding's bound."""
    N, M, Re, Ma, steps = 32, 2, 800.0, 0.025, 100
    X = gen.draw_params(66, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp16", exact_gamma=True).init(X).step(steps)
    assert mclbm.mclbm_get_launch(ens.ctx)[0] == 6
    f, un = _oracle_exact(N, X, Re, Ma, steps)
    _, u = oracle.moments(f)
    got = np.stack([ens.moments(m)[1].cpu().numpy() for m in range(M)])
    assert rel_l2(got, u / un["ulat"]) <= 1e-3


def test_d3q27_fp32_exact_gamma_velocity_error():
    N, M, Re, Ma, steps = 16, 2, 400.0, 0.1, 20
    X = gen.draw_params(67, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", exact_gamma=True, lattice=27).init(X).step(steps)
    f, un = _oracle_exact(N, X, Re, Ma, steps, lattice=27)
    _, u = oracle.moments(f)
    got = np.stack([ens.moments(m)[1].cpu().numpy() for m in range(M)])
    assert rel_l2(got, u / un["ulat"]) <= 1e-5


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_d3q27_fp16_exact_gamma_velocity_error(pattern):
    """FP16 storage on D3Q27: four nodes per thread through the exact-gamma solver in turn."""
    N, M, Re, Ma, steps = 16, 2, 400.0, 0.1, 20
    X = gen.draw_params(68, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp16", pattern=pattern, exact_gamma=True, lattice=27).init(X)
    ens.step(steps)
    assert mclbm.mclbm_get_launch(ens.ctx)[0] == 6
    f, un = _oracle_exact(N, X, Re, Ma, steps, lattice=27)
    _, u = oracle.moments(f)
    got = np.stack([ens.moments(m)[1].cpu().numpy() for m in range(M)])
    assert rel_l2(got, u / un["ulat"]) <= 1e-3


def test_d3q27_fp64_exact_gamma_parity():
    N, M, Re, Ma, steps = 16, 2, 400.0, 0.1, 6
    X = gen.draw_params(64, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", exact_gamma=True, lattice=27).init(X).step(steps)
    f, _ = _oracle_exact(N, X, Re, Ma, steps, lattice=27)
    assert np.max(np.abs(lib_populations(ens) - f) / np.abs(f)) <= 1e-12


def test_launch_and_adjoint_rules():
    ens = Ensemble(16, 1, Re=400.0, Ma=0.1, precision="fp32", exact_gamma=True).init()
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_set_launch(ens.ctx, 2, 128, 3)  # only kind 6 with the option
    plain = Ensemble(16, 1, Re=400.0, Ma=0.1, precision="fp32").init()
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_set_launch(plain.ctx, 1, 128, 6)  # and kind 6 only with it
    assert mclbm.mclbm_autotune(ens.ctx, 1)[0] == 6
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_grad(ens.ctx, 0, 2, 1, buf.data_ptr(), 1 << 20, 1)
    assert e.value.status == "INVALID_ARG"
