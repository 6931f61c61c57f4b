"""GPU parity of the ensemble reductions (FP64) against the NumPy oracle, through the
C ABI: kinetic energy, enstrophy, mean/variance fields, shell spectrum, trace S2,
axis S_p, restriction and the one-point W1."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_populations
from oracle import stats
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _pair(N=16, M=3, steps=30, precision="fp64", Re=300.0, Ma=0.1, seed=21, pattern="pull"):
    """A GPU ensemble and the oracle velocity field computed from the GPU's own state (so the
    statistics are compared on identical input)."""
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=precision, pattern=pattern, seed=seed).init().step(steps)
    f = lib_populations(ens)
    _, u = oracle.moments(f)
    return ens, stats.to_physical(u, ens.units["U_lat"])


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


@pytest.mark.parametrize("steps", [0, 1, 30])
def test_energy_enstrophy(steps):
    ens, u = _pair(steps=steps, pattern="aa")
    E, Z = ens.energy(enstrophy=True)
    assert _rel(E, stats.kinetic_energy(u)) <= 1e-12
    assert _rel(Z, stats.enstrophy(u)) <= 1e-12
    # the fused population-side reduction agrees with the field route
    assert _rel(ens.energy(), E) <= 1e-12


def test_energy_fp32_storage_reduction_is_fp64():
    """With FP32 storage the velocity comes from the stored FP32 deviations (FP32 arithmetic);
    the squares and sums are FP64."""
    ens, u = _pair(precision="fp32", M=4)
    assert _rel(ens.energy(), stats.kinetic_energy(u)) <= 2e-6


def test_initial_energy_closed_form_on_gpu():
    """E_0 = U_c^2/8 + sum X^2 / 1024 per sample (equilibrium init, rho = 1)."""
    X = gen.draw_params(8, 6)
    ens = Ensemble(16, 6, Re=100.0, Ma=0.05, precision="fp64").init(X)
    np.testing.assert_allclose(ens.energy(), 1 / 8 + (X**2).sum(1) / 1024, rtol=1e-12)


def test_mean_var():
    ens, u = _pair(M=5)
    mean, var = ens.mean_var()
    om, ov = stats.mean_var(u)
    np.testing.assert_allclose(mean.cpu().numpy(), om, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(var.cpu().numpy(), ov, rtol=1e-9, atol=1e-18)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_mean_var_reduced_precision_storage_chunks(precision):
    """FP32/FP16 storage: the per-node differences to sample 0 and their squares summed in FP32
    over chunks of 8 samples, the chunks accumulated in FP64.  M = 11 spans a full chunk and a
    partial one; against NumPy's FP64 mean and variance of the library's own velocity field (whose
    FP32 velocities divide where the pass multiplies by a reciprocal: a few ulp apart, about 1e-5
    of the sample-to-sample differences): mean within 1e-6 of the velocity scale, variance within
    2e-4 relative where it holds at least 1e-3 of its maximum; E against the library's own FP64
    energy reduction within 2e-6.  A chunk flushed twice or not at all would be off by O(1/M)."""
    ens = Ensemble(16, 11, Re=300.0, Ma=0.1, precision=precision, seed=21).init().step(12)
    u = _gpu_field(ens)
    E, mean, var = ens.energy_mean_var()
    rm, rv = stats.mean_var(u)
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    assert np.max(np.abs(mean - rm)) <= 1e-6 * np.max(np.abs(u))
    big = rv >= 1e-3 * rv.max()
    assert np.max(np.abs(var - rv)[big] / rv[big]) <= 2e-4
    assert _rel(E, ens.energy()) <= 2e-6


def test_mean_var_needs_two_samples():
    ens = Ensemble(8, 1, Re=100.0, Ma=0.1, precision="fp32").init()
    with pytest.raises(mclbm.MclbmError) as e:
        ens.mean_var()
    assert e.value.status == "SHAPE"


def _bins_close(got, ref, rel, floor):
    """Relative agreement on bins holding at least `floor` of the total."""
    tot = np.abs(ref).sum(axis=-1, keepdims=True)
    mask = np.abs(ref) >= floor * tot
    assert mask.any()
    err = np.abs(got - ref)[mask] / np.abs(ref)[mask]
    assert err.max() <= rel, err.max()
    # bins below the floor still agree in absolute terms
    assert np.max(np.abs(got - ref)) <= rel * tot.max()


# M = 3: one pair of samples sharing transforms (u_z of both in one transform, both
# autocorrelations from one inverse) and an odd last sample with transforms of its own
@pytest.mark.parametrize("N,M", [(8, 2), (16, 3), (32, 2)])
def test_spectrum(N, M):
    ens, u = _pair(N=N, M=M)
    _bins_close(ens.spectrum(), stats.energy_spectrum(u), 1e-10, 1e-12)


@pytest.mark.parametrize("M", [1, 2])
def test_spectrum_tgv_closed_form(M):
    """Deterministic TGV at t = 0: E(2) = 3 pi U^2 / 124 (U = U_c = 1), zero elsewhere; with
    M = 2 both samples come out of the paired transforms."""
    ens = Ensemble(16, M, Re=100.0, Ma=0.05, precision="fp64").init_tgv()
    for E in ens.spectrum():
        assert abs(E[2] - 3 * np.pi / 124) <= 1e-12
        assert np.all(np.abs(np.delete(E, 2)) <= 1e-14)


@pytest.mark.parametrize("N,M", [(8, 2), (16, 3), (32, 2)])
def test_sf_trace(N, M):
    ens, u = _pair(N=N, M=M)
    _bins_close(ens.sf_trace(), stats.structure_function_trace(u), 1e-10, 1e-12)


def test_paired_spectra_match_single_sample_contexts():
    """A sample's spectrum and trace S2 do not depend on the sample it is paired with: the
    samples of a 3-sample ensemble (a pair and a single) against three one-sample contexts
    holding the same parameters: within 1e-12 relative on bins holding at least 1e-6 of the
    total, and 1e-12 of the total on every bin (the transforms' rounding differs between the
    two)."""
    X = gen.draw_params(29, 3)
    ens = Ensemble(16, 3, Re=300.0, Ma=0.1, precision="fp64").init(X).step(12)
    E, S = ens.spectrum(), ens.sf_trace()
    for m in range(3):
        one = Ensemble(16, 1, Re=300.0, Ma=0.1, precision="fp64").init(X[m:m + 1]).step(12)
        _bins_close(E[m:m + 1], one.spectrum(), 1e-12, 1e-6)
        _bins_close(S[m:m + 1], one.sf_trace(), 1e-12, 1e-6)


@pytest.mark.parametrize("N,pmax", [(8, 6), (16, 6), (32, 3), (8, 8)])
def test_sf_axes(N, pmax):
    ens, u = _pair(N=N, M=2)
    got = ens.sf_axes(pmax)
    ref = stats.structure_function_axes(u, pmax)
    assert _rel(got, ref) <= 1e-10


@pytest.mark.parametrize("N", [64, 128])
def test_reductions_at_large_kernel_shapes(N):
    """FP64 parity of the spectrum, trace S2 and axis S_p where the kernels take the shapes of
    the large lattices: the S_p kernel stages 256 / (N/2) lines per block (8 at N = 64, 4 at
    N = 128, against 16 at N = 32), and the shell kernel spreads 16 blocks over the rows of
    disks of up to N/2 rows.  Same bounds as at small N: 1e-10 relative on bins holding at
    least 1e-12 of the total."""
    ens, u = _pair(N=N, M=2, steps=10)
    _bins_close(ens.spectrum(), stats.energy_spectrum(u), 1e-10, 1e-12)
    _bins_close(ens.sf_trace(), stats.structure_function_trace(u), 1e-10, 1e-12)
    assert _rel(ens.sf_axes(6), stats.structure_function_axes(u, 6)) <= 1e-10


def test_reductions_at_256():
    """N = 256 (two lines per block in the S_p kernel, shells of up to 128 disk rows), one FP64
    sample on the library's own velocity field (its moments are checked against the oracle at
    the smaller sizes): spectrum and trace S2 on every bin, S_p at the lags 1, 37, 128."""
    ens = Ensemble(256, 1, Re=1600.0, Ma=0.05, precision="fp64", seed=23).init().step(4)
    u = _gpu_field(ens)
    _bins_close(ens.spectrum(), stats.energy_spectrum(u), 1e-10, 1e-12)
    _bins_close(ens.sf_trace(), stats.structure_function_trace(u), 1e-10, 1e-12)
    lags = [1, 37, 128]
    got = ens.sf_axes(6)[:, :, [r - 1 for r in lags]]
    ref = stats.structure_function_axes(u, 6, lags=lags)[:, :, [r - 1 for r in lags]]
    assert _rel(got, ref) <= 1e-10


def _gpu_field(ens):
    """The library's own physical velocity of every sample, [M][3][N][N][N] (for FP32/FP16
    storage formed in FP32 from the stored deviations, like the stepper's moments)."""
    return np.stack([ens.moments(m)[1].cpu().numpy() for m in range(ens.M)])


def test_sf_axes_fp32_line_sums_at_256():
    """FP32 storage at N = 256 (eight 32-point chunks per line summed in FP32 before the FP64
    accumulation): S_p, p = 2..6, at the lags 1, 37 and 128 against the oracle's FP64 evaluation
    of the library's own velocity field, within 1e-5 relative."""
    ens = Ensemble(256, 1, Re=1600.0, Ma=0.05, precision="fp32", seed=23).init().step(4)
    u = _gpu_field(ens)
    lags = [1, 37, 128]
    got = ens.sf_axes(6)[:, :, [r - 1 for r in lags]]
    ref = stats.structure_function_axes(u, 6, lags=lags)[:, :, [r - 1 for r in lags]]
    assert _rel(got, ref) <= 1e-5


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_sf_axes_reduced_precision_storage(precision):
    """FP32/FP16 storage: differences and powers in FP32, FP32 line sums (of 32-point chunks)
    accumulated in FP64, against the oracle's FP64 evaluation on the library's own velocity
    field (N = 64 spans two 32-point chunks per line; p = 2..6 within 1e-5 relative); pmax = 8
    takes the FP64 path (1e-10).  The field itself matches the oracle's FP64 moments of the same
    populations to FP32 rounding."""
    ens, u = _pair(N=64, M=2, steps=20, precision=precision)
    ug = _gpu_field(ens)
    assert np.max(np.abs(ug - u)) <= 1e-6 * np.max(np.abs(u))
    got = ens.sf_axes(6)
    assert _rel(got, stats.structure_function_axes(ug, 6)) <= 1e-5
    ens8, _ = _pair(N=8, M=2, precision=precision)
    assert _rel(ens8.sf_axes(8), stats.structure_function_axes(_gpu_field(ens8), 8)) <= 1e-10


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("fp16", 2e-6)])
@pytest.mark.parametrize("pattern,steps", [("pull", 7), ("aa", 6), ("aa", 7)])
def test_energy_mean_var_one_pass(precision, tol, pattern, steps):
    """The one-pass E_m + mean/var: energies as mclbm_energy (FP64 storage 1e-12; FP32/FP16
    storage, whose moments are FP32, within 2e-6), mean and variance bit-identical to
    mclbm_mean_var, and FP64 storage against the oracle; AA at even and odd parity."""
    ens, u = _pair(N=16, M=5, steps=steps, precision=precision, pattern=pattern)
    E, mean, var = ens.energy_mean_var()
    assert _rel(E, ens.energy()) <= tol
    m2, v2 = ens.mean_var()
    assert torch.equal(mean, m2) and torch.equal(var, v2)
    if precision == "fp64":
        rm, rv = stats.mean_var(u)
        np.testing.assert_allclose(mean.cpu().numpy(), rm, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(var.cpu().numpy(), rv, rtol=1e-9, atol=1e-18)
        assert _rel(E, stats.kinetic_energy(u)) <= 1e-12


def test_energy_mean_var_one_pass_full_warp_rows():
    """64^3 x 4 (a row spans a full warp and more), FP32 pull: the same agreement."""
    ens = Ensemble(64, 4, Re=800.0, Ma=0.025, precision="fp32", seed=3).init().step(5)
    E, mean, var = ens.energy_mean_var()
    assert _rel(E, ens.energy()) <= 2e-6
    m2, v2 = ens.mean_var()
    assert torch.equal(mean, m2) and torch.equal(var, v2)


def test_restrict():
    ens, u = _pair(N=16, M=3)
    ref = stats.restrict(u, 8)
    # components near zero come from sums of +-f ~ 0.03: compare against the velocity scale
    np.testing.assert_allclose(ens.restrict(8).cpu().numpy(), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("MA,MB", [(4, 4), (3, 7)])
def test_w1_between_levels(MA, MB):
    """W_{1,1} between a 16^3 and a 32^3 ensemble (different N and M)."""
    A, ua = _pair(N=16, M=MA, seed=3)
    B, ub = _pair(N=32, M=MB, seed=4, Re=600.0, Ma=0.05)
    W, pp = A.w1(B, per_point=True)
    Wo, Do = stats.w1_one_point(stats.restrict(ua), stats.restrict(ub), per_point=True)
    assert abs(W - Wo) <= 1e-12 * Wo
    np.testing.assert_allclose(pp, Do, rtol=1e-12, atol=1e-18)


def test_w1_restricted_equal_sizes_and_shift():
    """Raw entry point on device arrays: shifting every value by c gives W = 3 c (three
    components, each shifted by c)."""
    import torch
    M, G = 33, 512
    a = torch.as_tensor(gen.normal(60, (M, G, 3)), device="cuda")
    b = a + 0.125
    work = torch.empty(mclbm.mclbm_w1_work_bytes(M, M, G), dtype=torch.uint8, device="cuda")
    W = mclbm.mclbm_w1_restricted(a.data_ptr(), M, b.data_ptr(), M, G, work.data_ptr(), work.numel())
    assert abs(W - 3 * 0.125) <= 1e-14
    c = torch.as_tensor(gen.normal(61, (M, G, 3)), device="cuda")
    W2 = mclbm.mclbm_w1_restricted(a.data_ptr(), M, c.data_ptr(), M, G, work.data_ptr(), work.numel())
    ref = stats.w1_one_point(a.cpu().numpy(), c.cpu().numpy())
    assert abs(W2 - ref) <= 1e-13 * ref
