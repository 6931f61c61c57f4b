"""Pins of the C oracle's kinetic energy and enstrophy (the objective behind every adjoint
parity test), of its relative entropy H_rel, and of how its exact entropic gamma is decided.
Each pin is a closed form or an independent evaluation chosen so that a plausible mistake
(a dropped term, a wrong sign of a curl term, a wrong grid spacing, a dropped volume factor,
a constrained minimiser where the unconstrained one exists) fails it."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import ensemble_inputs as gen
import oracle
from oracle import stats


def _grid(N):
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def _lattice_units(u_phys, ulat, uc=1.0):
    """The C oracle takes lattice-unit velocities and returns physical E and Z."""
    return np.ascontiguousarray(u_phys * (ulat / uc))


@pytest.mark.parametrize("N", [8, 16])
def test_c_energy_enstrophy_of_taylor_green(N):
    """TGV: E = U^2/8 and, with second-order central differences on dx = 2 pi / N (each
    derivative of a unit Fourier mode carries s = sin(dx)/dx), Z = (3/8) U^2 s^2.  The z
    vorticity is d_x u_y - d_y u_x = 2 U s sin x sin y cos z; the other sign would make it
    vanish."""
    U, ulat = 0.9, 0.05
    X, Y, Z = _grid(N)
    u = np.zeros((1, 3, N, N, N))
    u[0, 0] = U * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[0, 1] = -U * np.cos(X) * np.sin(Y) * np.cos(Z)
    E, Zs = oracle.energy(_lattice_units(u, ulat), ulat)
    dx = 2 * np.pi / N
    s = np.sin(dx) / dx
    assert abs(E[0] - U**2 / 8) <= 1e-15
    assert abs(Zs[0] - 3 / 8 * U**2 * s**2) <= 1e-14


def _sheared(N, comp, a, b):
    """A field with one nonzero vorticity component, whose two curl terms both act:
    comp 0: u_y = b sin(y + z), u_z = a sin(y + z)  ->  w_x = s (a - b) cos(y + z)
    comp 1: u_z = b sin(z + x), u_x = a sin(z + x)  ->  w_y = s (a - b) cos(z + x)
    comp 2: u_x = b sin(x + y), u_y = a sin(x + y)  ->  w_z = s (a - b) cos(x + y)
    (w = curl u: w_x = d_y u_z - d_z u_y, w_y = d_z u_x - d_x u_z, w_z = d_x u_y - d_y u_x)."""
    X, Y, Z = _grid(N)
    u = np.zeros((1, 3, N, N, N), dtype=np.result_type(a, b, np.float64))
    arg = {0: Y + Z, 1: Z + X, 2: X + Y}[comp]
    first, second = {0: (1, 2), 1: (2, 0), 2: (0, 1)}[comp]  # (b-component, a-component)
    u[0, first] = b * np.sin(arg)
    u[0, second] = a * np.sin(arg)
    return u


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("N", [8, 16])
def test_c_enstrophy_signs_of_every_curl_term(comp, N):
    """Each vorticity component is the difference of two derivatives: for the sheared fields
    Z = s^2 (a - b)^2 / 4 (mean of cos^2 over the grid is 1/2) and E = (a^2 + b^2) / 4; a sign
    error in either curl term gives (a + b)^2, a spacing of 2 pi / (N - 1) another s."""
    a, b, ulat = 1.0, 0.3, 0.02
    E, Zs = oracle.energy(_lattice_units(_sheared(N, comp, a, b), ulat), ulat)
    dx = 2 * np.pi / N
    s = np.sin(dx) / dx
    assert abs(E[0] - (a * a + b * b) / 4) <= 1e-14
    assert abs(Zs[0] - s * s * (a - b) ** 2 / 4) <= 1e-14


def test_c_energy_complex_twin_derivative():
    """The complex-step twin (behind every complex-step gradient): with the amplitude a + i h,
    Im Z / h = dZ/da = s^2 (a - b) / 2 and Im E / h = a / 2, and the real parts are the real
    oracle's values."""
    N, a, b, h, ulat = 8, 1.0, 0.3, 1e-30, 0.02
    for comp in range(3):
        u = _sheared(N, comp, a + 1j * h, b)
        E, Zs = oracle.energy(np.ascontiguousarray(u * ulat), ulat)
        dx = 2 * np.pi / N
        s = np.sin(dx) / dx
        assert abs(Zs[0].imag / h - s * s * (a - b) / 2) <= 1e-14
        assert abs(E[0].imag / h - a / 2) <= 1e-15
        Er, Zr = oracle.energy(_lattice_units(_sheared(N, comp, a, b), ulat), ulat)
        assert E[0].real == Er[0] and Zs[0].real == Zr[0]


def test_c_energy_equals_numpy_statistics_on_a_random_field():
    """The C and NumPy statements of E and Z (written separately) agree on a random field of
    three samples, to rounding."""
    N, M, ulat = 16, 3, 0.05
    u_phys = gen.normal(90, (M, 3, N, N, N))
    E, Zs = oracle.energy(_lattice_units(u_phys, ulat), ulat)
    np.testing.assert_allclose(E, stats.kinetic_energy(u_phys), rtol=1e-13)
    np.testing.assert_allclose(Zs, stats.enstrophy(u_phys), rtol=1e-13)


def test_hrel_closed_forms():
    """H_rel = eps^3 sum_x sum_i [f_i ln(f_i / w_i) - f_i + w_i], eps = 2 pi / N (Eqs.
    (relEntropy1), (relEntropy2)).  With f_i = e w_i the bracket is w_i (e - e + 1) = w_i, so
    every node contributes sum w = 1 and H_rel = M (2 pi)^3 (dropping -f + w gives e times
    that, dropping eps^3 gives M N^3).  With f = w, H_rel = 0.  With f_i = e w_i on the six
    face velocities only (weight 1/18 each) and f_i = w_i elsewhere, every node contributes
    1/3 (D3Q19 weights).  With f_i = 2 w_i: 2 ln 2 - 1 per node."""
    c, w, _ = oracle.lattice()
    N, M = 4, 2
    ones = np.ones((M, 19, N, N, N))
    W = w[None, :, None, None, None] * ones
    vol = (2 * np.pi) ** 3
    assert abs(oracle.hrel(np.e * W) - M * vol) <= 1e-13 * M * vol
    assert abs(oracle.hrel(W)) <= 1e-15
    face = (np.abs(c).sum(1) == 1)
    f = W.copy()
    f[:, face] *= np.e
    assert abs(oracle.hrel(f) - M * vol / 3) <= 1e-13 * M * vol
    assert abs(oracle.hrel(2 * W) - M * vol * (2 * np.log(2) - 1)) <= 1e-13 * M * vol


def _node(seed, amp, u_scale=0.05):
    c, w, _ = oracle.lattice()
    r = gen.uniform(seed, 23)
    return oracle.equilibrium(1.0 + 0.02 * r[0], u_scale * r[1:4]) + amp * w * r[4:23]


def _positivity_interval(f, ds, dh, omega):
    """The g for which every f*(g) = f - omega Ds - (omega g / 2) Dh is positive."""
    A, B = f - omega * ds, 0.5 * omega * dh
    hi = np.min(A[B > 0] / B[B > 0]) if np.any(B > 0) else np.inf
    lo = np.max(A[B < 0] / B[B < 0]) if np.any(B < 0) else -np.inf
    return lo, hi


@pytest.mark.parametrize("seed", [80, 81, 82, 83, 84])
def test_exact_gamma_equals_unconstrained_argmin_where_it_is_interior(seed):
    """Away from equilibrium (amplitude 2e-2) the unconstrained minimiser of H(f*(g)) =
    sum f* ln(f* / w) (Eq. (kbc_entropy)) lies inside 0 <= g <= 4 / omega: the oracle reports
    the node as decided by an interior root and returns the minimiser that a derivative-free
    Brent search of H over the whole positivity interval (no constraint) finds."""
    _, w, _ = oracle.lattice()
    omega = 1.9
    f = _node(seed, 2e-2)
    _, _, ds, dh = oracle.collide(f, omega)
    with oracle.exact_gamma() as ex:
        _, ge, _, _ = oracle.collide(f, omega)
        counts = ex.counts()
    assert counts["interior"] == 1 and sum(counts.values()) == 1, counts
    lo, hi = _positivity_interval(f, ds, dh, omega)

    def H(g):
        x = f - omega * ds - 0.5 * omega * g * dh
        return np.sum(x * np.log(x / w))

    span = min(hi, 1e3) - max(lo, -1e3)
    res = minimize_scalar(H, bounds=(max(lo, -1e3) + 1e-9 * span, min(hi, 1e3) - 1e-9 * span), method="bounded",
                          options={"xatol": 1e-12, "maxiter": 2000})
    assert 0.0 < ge < 4.0 / omega
    # a derivative-free search locates a smooth minimum to about sqrt(machine epsilon)
    assert abs(res.x - ge) <= 2e-6 * abs(ge), (res.x, ge)
    assert H(ge) <= res.fun + 1e-15
    assert H(ge - 1e-5) > H(ge) and H(ge + 1e-5) > H(ge)


def test_exact_gamma_counts_report_where_the_constraint_binds():
    """Close to equilibrium (amplitude 1e-7) the unconstrained minimiser lies outside
    0 <= g <= 4 / omega (it grows like 1 / |Dh| with the polynomial equilibrium): the oracle
    reports an end point for such nodes and returns it, and an ensemble step counts every node
    once."""
    omega = 1.95
    with oracle.exact_gamma() as ex:
        for seed in (60, 61, 62):
            _, ge, _, _ = oracle.collide(_node(seed, 1e-7), omega)
            assert ge == 0.0 or ge == 4.0 / omega
        counts = ex.counts()
    assert counts["upper_end"] + counts["lower_end"] == 3 and sum(counts.values()) == 3, counts
    N, M = 8, 2
    un = oracle.units(N, 200.0, 0.1)
    f = oracle.init_ensemble(N, gen.draw_params(5, M), un["ulat"])
    oracle.run(f, un["omega"], 3)
    with oracle.exact_gamma() as ex:
        oracle.step(f, un["omega"])
        counts = ex.counts()
    assert sum(counts.values()) == M * N**3, counts
