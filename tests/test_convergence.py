"""Host-side convergence pipeline against closed forms: power laws give their exponents and
K41 plateaus, exponential decay gives its dissipation rate, the trapezoidal rule is exact on
linear data."""
import numpy as np

from paper_2608_23786_gb300 import convergence as cv


def test_eoc_slope_of_power_laws():
    Ns = [32, 64, 128, 256]
    assert abs(cv.eoc_slope(Ns, [3.0 * N ** -0.45 for N in Ns]) + 0.45) <= 1e-13
    assert abs(cv.eoc_slope(Ns, [N ** 2.0 for N in Ns]) - 2.0) <= 1e-13


def test_dissipation_of_exponential_decay():
    """E(t) = E0 exp(-2 nu k^2 t): -dE/dt = 2 nu k^2 E (second-order differences: error O(dt^2))."""
    t = np.linspace(0.0, 1.0, 201)
    rate = np.array([0.3, 1.1])
    E = 0.125 * np.exp(-np.outer(t, rate))
    d = cv.dissipation_rate(t, E)
    assert np.allclose(d, E * rate[None, :], rtol=2e-4)


def test_k41_spectrum_and_structure_function_plateaus():
    """E_m(kappa) = C_Kol d_m^(2/3) kappa^(-5/3) compensates to 1 in every sample (std 0);
    S2_m(r) = C (d_m r)^(2/3) compensates to C."""
    d = np.array([0.5, 0.8, 1.3])
    kappa = np.arange(33, dtype=np.float64)
    E = cv.C_KOL * d[:, None] ** (2 / 3) * np.where(kappa > 0, kappa, 1.0)[None, :] ** (-5 / 3)
    keta, mean, std = cv.compensated_spectrum(E, d, nu=1e-3)
    assert np.allclose(mean, 1.0, rtol=1e-13) and np.all(std <= 1e-13)
    assert np.allclose(keta, kappa[1:] * (1e-9 / d.mean()) ** 0.25, rtol=1e-14)
    r = np.linspace(0.1, np.pi, 16)
    S2 = 7.7 * (d[:, None] * r[None, :]) ** (2 / 3)
    _, mean, std = cv.compensated_structure_function(S2, r, d, nu=1e-3)
    assert np.allclose(mean, 7.7, rtol=1e-13) and np.all(std <= 1e-12)


def test_time_integrals_exact_on_linear_data():
    t = np.array([0.0, 0.5, 1.5, 3.0])
    E = np.stack([np.full((2, 5), 2.0 + 3.0 * tk) for tk in t])  # [T][M][K], linear in t
    assert np.allclose(cv.time_integrated_spectrum(t, E), 2.0 * 3.0 + 1.5 * 9.0, rtol=1e-14)
    S = np.stack([np.full(4, 1.0 + tk) for tk in t])
    assert np.allclose(cv.time_integrated_structure_function(t, S, p=2), np.sqrt(3.0 + 4.5), rtol=1e-14)
