"""Convergence pipeline on the statistics the GPU path computes (host-side post-processing).

- ``eoc_slope``: least-squares slope of log D over log N, the experimental order of convergence
  of Algorithm "ComputeSlopes" (EOSC from ``Ensemble.sample_error`` values, EOWC from W1 values).
- ``dissipation_rate``: per-sample d_m(t) ~ -dE_m/dt from the kinetic energy over time (the
  paper's numerical approximation of nu |grad u|^2 / |Omega|, Sec. "Energy spectra").
- ``kolmogorov_scale``: eta(t) = (nu^3 / E[d(t)])^(1/4), Eq. (kolmogorov_microscale).
- ``compensated_spectrum``: E^c_m = C_Kol^-1 d_m^(-2/3) kappa^(5/3) E_m(kappa), Eq. (compensatedE),
  compensated per sample, then mean and standard deviation over the samples.
- ``compensated_structure_function``: S^{2,c}_m = S^2_m(r) / (d_m r)^(2/3), Eq. (compensatedSF).
- ``time_integrated_spectrum`` / ``time_integrated_structure_function``: E_T(kappa) = int_0^T
  E[E(kappa, t)] dt and S^p(T, r) = (int_0^T S^p(r, t) dt)^(1/p) (Eqs. (energyScaling),
  (structures)) by the trapezoidal rule over the sampled times.

Means and standard deviations over samples use the unbiased (M - 1) variance.
"""
import numpy as np

C_KOL = 1.5  # K41 constant (Sec. "Energy spectra")


def eoc_slope(Ns, Ds):
    """Slope alpha of the least-squares line log D = alpha log N + b over the resolutions Ns."""
    x = np.log(np.asarray(Ns, dtype=np.float64))
    y = np.log(np.asarray(Ds, dtype=np.float64))
    xm, ym = x.mean(), y.mean()
    return float(((x - xm) * (y - ym)).sum() / ((x - xm) ** 2).sum())


def dissipation_rate(t, E):
    """d_m(t_k) = -dE_m/dt at the sample times t [T] from the per-sample energy E [T][M]
    (second-order differences: central inside, one-sided at the ends)."""
    t = np.asarray(t, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    return -np.gradient(E, t, axis=0, edge_order=2)


def kolmogorov_scale(nu, d_mean):
    """eta = (nu^3 / E[d])^(1/4), Eq. (kolmogorov_microscale)."""
    return (nu**3 / np.asarray(d_mean, dtype=np.float64)) ** 0.25


def _mean_std(X):
    X = np.asarray(X, dtype=np.float64)
    return X.mean(axis=0), (X.std(axis=0, ddof=1) if X.shape[0] > 1 else np.zeros(X.shape[1:]))


def compensated_spectrum(E, d, nu):
    """E [M][K] per-sample shell spectra at one time (kappa = 0..K-1), d [M] per-sample
    dissipation rates.  Returns (kappa eta, mean E^c, std E^c) over kappa >= 1."""
    E = np.asarray(E, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    kappa = np.arange(E.shape[1], dtype=np.float64)[1:]
    Ec = E[:, 1:] * kappa[None, :] ** (5.0 / 3.0) / (C_KOL * d[:, None] ** (2.0 / 3.0))
    mean, std = _mean_std(Ec)
    return kappa * kolmogorov_scale(nu, d.mean()), mean, std


def compensated_structure_function(S2, r, d, nu):
    """S2 [M][R] per-sample second-order structure functions at the physical separations
    r [R] (r <= pi), d [M].  Returns (r / eta, mean S^{2,c}, std S^{2,c})."""
    S2 = np.asarray(S2, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    Sc = S2 / (d[:, None] * r[None, :]) ** (2.0 / 3.0)
    mean, std = _mean_std(Sc)
    return r / kolmogorov_scale(nu, d.mean()), mean, std


def _trapezoid(t, y):
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    dt = np.diff(t).reshape((-1,) + (1,) * (y.ndim - 1))
    return (0.5 * (y[1:] + y[:-1]) * dt).sum(axis=0)


def time_integrated_spectrum(t, E):
    """E_T(kappa) = int_0^T E[E(kappa, t)] dt from per-sample spectra E [T][M][K] at times t [T]."""
    return _trapezoid(t, np.asarray(E, dtype=np.float64).mean(axis=1))


def time_integrated_structure_function(t, S, p=2):
    """S^p(T, r) = (int_0^T S^p(r, t) dt)^(1/p) from ensemble S^p [T][R] (or [T][M][R], averaged
    over the samples first) at times t [T]."""
    S = np.asarray(S, dtype=np.float64)
    if S.ndim == 3:
        S = S.mean(axis=1)
    return _trapezoid(t, S) ** (1.0 / p)
