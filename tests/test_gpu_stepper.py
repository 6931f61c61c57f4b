"""GPU parity of the fused stream + KBC collide stepper against the FP64 oracle,
through the C ABI (libmclbm)."""
import math

import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_populations, lib_to_oracle_perm, oracle_to_lib, rel_l2
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu

# Deterministic Taylor-Green sample at 32^3: U_lat = 0.05 (Ma = 0.05 sqrt(3)), Re = 100,
# density from the TGV pressure field, FP64.
CFG1 = dict(N=32, M=1, Re=100.0, Ma=0.05 * math.sqrt(3.0), init_density=1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _oracle_run(N, X, Re, Ma, steps, density_mode=0, M=None):
    un = oracle.units(N, Re, Ma)
    f = oracle.init_ensemble(N, X, un["ulat"], density_mode=density_mode, M=M)
    oracle.run(f, un["omega"], steps)
    return f, un


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_fp64_tgv_32_parity_1_10_200_steps(pattern):
    """FP64 GPU populations equal the oracle's to <= 1e-12 relative, per population,
    after 1, 10 and 200 steps of the deterministic TGV (32^3, Re = 100)."""
    ens = Ensemble(CFG1["N"], 1, Re=CFG1["Re"], Ma=CFG1["Ma"], precision="fp64", pattern=pattern,
                   init_density=1).init_tgv()
    un = oracle.units(32, CFG1["Re"], CFG1["Ma"])
    f = oracle.init_ensemble(32, None, un["ulat"], density_mode=1, M=1)
    done = 0
    for target in (0, 1, 10, 200):
        oracle.run(f, un["omega"], target - done)
        ens.step(target - done)
        done = target
        got = lib_populations(ens)
        err = np.max(np.abs(got - f) / np.abs(f))
        assert err <= 1e-12, (target, err)


@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("steps", [1, 7, 40])
def test_fp64_rtgv_ensemble_parity(pattern, steps):
    """A 3-sample RTGV ensemble at 16^3 (tile tail: 16^3 * 3 is not a multiple of the grid
    stride) matches per population, including odd step counts of the AA pattern."""
    N, M, Re, Ma = 16, 3, 400.0, 0.1
    X = gen.draw_params(11, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", pattern=pattern).init(X).step(steps)
    f, _ = _oracle_run(N, X, Re, Ma, steps)
    got = lib_populations(ens)
    assert np.max(np.abs(got - f) / np.abs(f)) <= 1e-12


def test_fp64_smallest_lattice_and_single_sample():
    """N = 8 (the smallest lattice), M = 1."""
    X = gen.draw_params(3, 1)
    ens = Ensemble(8, 1, Re=50.0, Ma=0.2, precision="fp64").init(X).step(25)
    f, _ = _oracle_run(8, X, 50.0, 0.2, 25)
    assert np.max(np.abs(lib_populations(ens) - f) / np.abs(f)) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("steps", [1, 2, 9])
def test_aa_equals_pull_bitwise(precision, steps):
    """In-place AA streaming and two-lattice pull streaming give bit-identical states
    (each node does the same arithmetic; a race or a wrong slot would break equality)."""
    X = gen.draw_params(5, 2)
    a = Ensemble(16, 2, Re=200.0, Ma=0.1, precision=precision, pattern="pull").init(X).step(steps)
    b = Ensemble(16, 2, Re=200.0, Ma=0.1, precision=precision, pattern="aa").init(X).step(steps)
    for m in range(2):
        assert torch.equal(a.populations(m), b.populations(m))


def test_params_and_philox_draw_through_context():
    """mclbm_init_ensemble(NULL) draws the Philox parameters; mclbm_get_params returns them."""
    ens = Ensemble(8, 5, Re=100.0, Ma=0.1, precision="fp32", seed=77).init()
    np.testing.assert_array_equal(ens.params(), gen.draw_params(77, 5))
    assert ens.steps_taken == 0
    ens.step(3)
    assert ens.steps_taken == 3


def _velocity(ens):
    return np.stack([ens.moments(m)[1].cpu().numpy() for m in range(ens.M)])


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_fp32_shifted_velocity_error_after_100_steps(pattern):
    """Shifted FP32 storage with FP32 collision: velocity within 1e-5 relative L2 of the FP64
    oracle after 100 steps (RTGV, 32^3 x 4, Re = 800, Ma = 0.025)."""
    N, M, Re, Ma, steps = 32, 4, 800.0, 0.025, 100
    X = gen.draw_params(2, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", pattern=pattern).init(X).step(steps)
    f, un = _oracle_run(N, X, Re, Ma, steps)
    _, u = oracle.moments(f)
    u_phys = u / un["ulat"]
    err = rel_l2(_velocity(ens), u_phys)
    assert err <= 1e-5, err


def test_fp16_shifted_velocity_error_after_100_steps():
    """Shifted FP16 storage (FP32 collision): velocity within 1e-3 relative L2 of the FP64
    oracle after 100 steps (same case as the FP32 test)."""
    N, M, Re, Ma, steps = 32, 4, 800.0, 0.025, 100
    X = gen.draw_params(2, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp16", pattern="aa").init(X).step(steps)
    f, un = _oracle_run(N, X, Re, Ma, steps)
    _, u = oracle.moments(f)
    err = rel_l2(_velocity(ens), u / un["ulat"])
    assert err <= 1e-3, err


def test_full_size_one_step_sampled_parity_fp32():
    """64^3 x 64 shifted FP32 ensemble (the benchmark's workload and launch): after 20 steps,
    one more GPU step is compared, for samples 0, 31 and 63, with one oracle step taken from
    the GPU's own pre-step state (converted to FP64)."""
    N, M, Re, Ma = 64, 64, 800.0, 0.025
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", pattern="pull", seed=1).init().step(20)
    un = oracle.units(N, Re, Ma)
    perm = lib_to_oracle_perm()
    inv = np.argsort(perm)
    picks = (0, 31, 63)
    before = {m: ens.populations(m).cpu().numpy()[inv][None].copy() for m in picks}
    ens.step(1)
    _, w, _ = oracle.lattice()
    for m in picks:
        f = before[m]
        oracle.step(f, un["omega"])
        got = ens.populations(m).cpu().numpy()[inv]
        dev = np.abs(got - f[0]) / w[:, None, None, None]
        # FP32 storage of h = f/w - 1 (|h| < 0.1): rounding 2^-24 * 0.1 per value, plus the
        # FP32 collision arithmetic
        assert dev.max() <= 5e-7, (m, dev.max())
        # mass and momentum of the step are conserved to FP32 rounding
        assert abs(got.sum() - f[0].sum()) <= 1e-6 * f[0].sum()


def test_full_size_conservation_fp32():
    """Global mass and momentum of every sample stay constant over 50 steps at 64^3 x 64
    (FP32 storage, collision conserves per node, streaming permutes)."""
    ens = Ensemble(64, 64, Re=800.0, Ma=0.025, precision="fp32", seed=1).init()
    c, _ = mclbm.mclbm_lattice()

    def totals(m):
        f = ens.populations(m)
        mass = f.sum().item()
        mom = [(f * torch.tensor(c[:, a], dtype=torch.float64, device=f.device)[:, None, None, None]).sum().item()
               for a in range(3)]
        return mass, mom

    t0 = {m: totals(m) for m in (0, 17, 63)}
    ens.step(50)
    for m in (0, 17, 63):
        mass, mom = totals(m)
        assert abs(mass - t0[m][0]) <= 2e-6 * t0[m][0]
        for a in range(3):
            assert abs(mom[a] - t0[m][1][a]) <= 2e-6 * t0[m][0]
    ens.check_finite()


def test_set_get_populations_roundtrip():
    """mclbm_set_populations then mclbm_get_populations returns the same FP64 state (pull and
    AA at odd parity)."""
    for pattern in ("pull", "aa"):
        ens = Ensemble(16, 2, Re=100.0, Ma=0.1, precision="fp64", pattern=pattern).init().step(3)
        f = ens.populations(1)
        g = f * (1 + 1e-3 * torch.as_tensor(gen.uniform(8, tuple(f.shape)), device=f.device))
        ens.set_populations(g, 1)
        assert torch.equal(ens.populations(1), g)
