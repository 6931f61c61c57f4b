"""Statistics of the reduced-precision paths against the FP64 oracle's own run: after 100 steps of
an RTGV ensemble (32^3 x 4, Re = 800, Ma = 0.025) the kinetic energy, shell spectrum, trace S2,
S_p along the axes and the one-point W1 between two ensembles computed by the library on its FP32
(or FP16) storage run are compared with the same statistics of the oracle's FP64 run.  The FP32
bounds are those the hot-path scope fixes for the shifted FP32 path (KE 2e-5, E(kappa) 1e-4 on bins
holding >= 1e-6 of the total, S2 and S_p 1e-4, W1 1e-4 relative); FP16 storage is held to the
measured errors with a margin."""
import numpy as np
import pytest

import ensemble_inputs as gen
import oracle
from oracle import stats
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu

N, M, RE, MA, STEPS = 32, 4, 800.0, 0.025, 100


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


@pytest.fixture(scope="module")
def oracle_fields():
    """The oracle's physical velocity of two independent ensembles after STEPS steps."""
    out = []
    for seed in (71, 72):
        X = gen.draw_params(seed, M)
        un = oracle.units(N, RE, MA)
        f = oracle.init_ensemble(N, X, un["ulat"])
        oracle.run(f, un["omega"], STEPS)
        _, u = oracle.moments(f)
        out.append((X, stats.to_physical(u, un["ulat"])))
    return out


def _errors(precision, pattern, oracle_fields):
    (Xa, ua), (Xb, ub) = oracle_fields
    a = Ensemble(N, M, Re=RE, Ma=MA, precision=precision, pattern=pattern).init(Xa).step(STEPS)
    b = Ensemble(N, M, Re=RE, Ma=MA, precision=precision, pattern=pattern).init(Xb).step(STEPS)
    err = {}
    Eo = stats.kinetic_energy(ua)
    err["ke"] = np.max(np.abs(a.energy() - Eo) / Eo)
    Sp, So = a.spectrum(), stats.energy_spectrum(ua)
    tot = So.sum(axis=1, keepdims=True)
    for key, floor in (("spectrum", 1e-6), ("spectrum_1e-4", 1e-4), ("spectrum_1e-2", 1e-2)):
        big = So >= floor * tot
        err[key] = np.max(np.abs(Sp - So)[big] / So[big])
    err["spectrum_abs"] = np.max(np.abs(Sp - So) / tot)
    T, To = a.sf_trace(), stats.structure_function_trace(ua)
    err["s2"] = np.max(np.abs(T - To)[:, 1:] / To[:, 1:])
    P, Po = a.sf_axes(6), stats.structure_function_axes(ua, 6)
    err["sp"] = np.max(np.abs(P - Po) / Po)
    W, Wo = a.w1(b), stats.w1_one_point(stats.restrict(ua), stats.restrict(ub))
    err["w1"] = abs(W - Wo) / Wo
    return err


@pytest.mark.parametrize("pattern", ["pull", "aa"])
def test_fp32_statistics_against_the_fp64_oracle_run(pattern, oracle_fields):
    """Measured: KE 2.8e-6, E(kappa) 5.5e-5, S2 2.9e-6, S_p 8.9e-6, W1 8.0e-6."""
    err = _errors("fp32", pattern, oracle_fields)
    bounds = {"ke": 2e-5, "spectrum": 1e-4, "s2": 1e-4, "sp": 1e-4, "w1": 1e-4}
    for k, tol in bounds.items():
        assert err[k] <= tol, (k, err[k])


def test_fp16_statistics_against_the_fp64_oracle_run(oracle_fields):
    """Measured: KE 2.5e-5; E(kappa) 2.5e-5 on bins holding >= 1e-2 of the energy, 1.9e-4 on bins
    >= 1e-4, and at most 2.5e-5 of the total energy on any bin; S2 2.6e-5, S_p 1.5e-4, W1 4.6e-3.
    On the bins near 1e-6 of the total the relative error reaches 3.6e-2: there the FP16
    rounding of the stored deviations (2^-11 of |h|, about 1e-5 of the velocity scale, spread
    over all wavenumbers) is comparable to the bin itself, so those bins are held to the
    absolute bound instead."""
    err = _errors("fp16", "aa", oracle_fields)
    bounds = {"ke": 1e-4, "spectrum_1e-2": 1e-4, "spectrum_1e-4": 1e-3, "spectrum_abs": 1e-4, "s2": 1e-4,
              "sp": 1e-3, "w1": 2e-2}
    for k, tol in bounds.items():
        assert err[k] <= tol, (k, err[k])
