"""Pins of the oracle's diffusive-scaling units and RTGV initialisation."""
import math
import os

import numpy as np
import pytest

import ensemble_inputs as gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        M, N, dt, Ma, Re, tau = line.split()
        rows.append((int(M), int(N), float(dt), float(Ma), float(Re), float(tau)))
    return rows


def _sig(x, digits):
    return float(f"{x:.{digits - 1}e}")


@pytest.mark.parametrize("row", [r for r in _table("params2_table.txt") if r[1] >= 32], ids=lambda r: f"N{r[1]}")
def test_units_reproduce_table_params2(row):
    """Table "params2", rows N = 32..512: dt to its 3 printed digits, tau_rel to its 6 decimals."""
    M, N, dt, Ma, Re, tau = row
    u = oracle.units(N, Re, Ma)
    assert _sig(u["dt"], 3) == dt
    assert round(u["tau"], 6) == tau
    assert abs(u["omega"] * u["tau"] - 1) < 1e-15
    # Table "frequencySummary": omega_nu = 2 c_s^2 / (2 nu + c_s^2)
    assert abs(u["omega"] - (2 / 3) / (2 * u["nu_lat"] + 1 / 3)) < 1e-15


def test_small_n_rows_follow_the_other_grid_convention():
    """Reading of the unit convention: rows N = 8, 16 of Table "params2" and every row of
    Table "params1" are reproduced by dx = 2 pi / (N - 1), not by the periodic 2 pi / N the
    library uses (Sec. "Numerical validation": eps = 2 pi / N).  Recorded, not adopted."""
    rows = [r for r in _table("params2_table.txt") if r[1] < 32] + _table("params1_table.txt")
    for M, N, dt, Ma, Re, tau in rows:
        u = oracle.units(N - 1, Re, Ma)  # dx = 2 pi / (N - 1)
        assert abs(u["tau"] - tau) <= 1e-6
        assert abs(u["dt"] - dt) <= 0.02 * dt
        assert abs(oracle.units(N, Re, Ma)["tau"] - tau) > 1e-6 or N >= 256


def _physical_u(f, ulat):
    rho, u = oracle.moments(f)
    return rho, u / ulat


@pytest.mark.parametrize("N", [8, 16])
def test_initial_energy_closed_form(N):
    """Per-sample E_0 = U_c^2/8 + (1/1024) sum X^2 exactly for N >= 8: the TGV modes
    (+-1,+-1,+-1) and the perturbation modes (+-2,+-2,+-2) are orthogonal on the grid and
    each product a_i(2x) a_j(2y) a_k(2z) has mean square 1/8 (Eqs. (tgv_init_velo),
    (alpha_perturbation))."""
    X = gen.draw_params(seed=5, M=3)
    ulat = 0.02
    f = oracle.init_ensemble(N, X, ulat)
    rho, u = _physical_u(f, ulat)
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-15)
    E = 0.5 * np.mean(np.sum(u * u, axis=1), axis=(1, 2, 3))
    expect = 1.0 / 8 + (X**2).sum(axis=1) / 1024
    np.testing.assert_allclose(E, expect, rtol=1e-13)


def test_parameter_index_order():
    """Parameter index 8 alpha + 4 i + 2 j + k: projecting component alpha of the initial
    velocity on a_i(2x) a_j(2y) a_k(2z) returns X_{alpha,ijk} / 8 times the mode's mean
    square 1/8 (a_0 = sin, a_1 = cos)."""
    N = 16
    X = gen.draw_params(seed=9, M=1)
    ulat = 0.01
    f = oracle.init_ensemble(N, X, ulat)
    _, u = _physical_u(f, ulat)
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, Xg = np.meshgrid(x, x, x, indexing="ij")
    a = [np.sin, np.cos]
    for al in range(3):
        for i in range(2):
            for j in range(2):
                for k in range(2):
                    mode = a[i](2 * Xg) * a[j](2 * Y) * a[k](2 * Z)
                    proj = np.mean(u[0, al] * mode)
                    assert abs(proj - X[0, 8 * al + 4 * i + 2 * j + k] / 64) < 1e-14


def test_tgv_density_option_mean_is_one():
    """Density option 1: rho = 1 + p / c_s^2 with the TGV pressure; its grid mean is 1 and
    its extremes are 1 + 3 (U^2/16) (+-2)(3) = 1 +- 9 U^2 / 8."""
    N, ulat = 16, 0.05
    f = oracle.init_ensemble(N, None, ulat, density_mode=1, M=1)
    rho, _ = oracle.moments(f)
    assert abs(rho.mean() - 1.0) < 1e-15
    assert abs(rho.max() - (1 + 9 * ulat**2 / 8)) < 1e-15


def test_philox_parameter_draw_matches_definition():
    """The shared generator draws sample m's 24 values from Philox4x64-10 counters (b, m),
    b = 0..5: the values of sample m do not depend on how many samples are drawn, and lie in
    [-w, w] with the right scale."""
    A = gen.draw_params(seed=3, M=8)
    B = gen.draw_params(seed=3, M=3, first_sample=5)
    np.testing.assert_array_equal(A[5:8], B)
    assert np.all(np.abs(A) <= gen.RTGV_WIDTH)
    big = gen.draw_params(seed=1, M=400)
    assert abs(big.mean()) < 2e-3 and abs(big.var() - gen.RTGV_WIDTH**2 / 3) < 1e-5


def test_leray_projection_pins():
    """P v = v - grad Delta^-1 div v (Sec. "Discretization and well-prepared initial data"): the
    projected perturbation is divergence free (spectrally), P is idempotent, the TGV field
    (divergence free) is left unchanged, and the removed part is a gradient (its curl vanishes)."""
    N = 16
    X = gen.draw_params(8, 2)
    udet, s = oracle.rtgv_fields(N, X)
    ps = oracle.leray_project(s)
    k = np.fft.fftfreq(N, d=1.0 / N)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    h = np.fft.fftn(ps, axes=(-3, -2, -1))
    assert np.abs(KX * h[:, 0] + KY * h[:, 1] + KZ * h[:, 2]).max() <= 1e-12 * np.abs(h).max()
    np.testing.assert_allclose(oracle.leray_project(ps), ps, rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.leray_project(udet[None]), udet[None], rtol=0, atol=1e-14)
    g = np.fft.fftn(s - ps, axes=(-3, -2, -1))
    curl = [KY * g[:, 2] - KZ * g[:, 1], KZ * g[:, 0] - KX * g[:, 2], KX * g[:, 1] - KY * g[:, 0]]
    assert max(np.abs(c).max() for c in curl) <= 1e-12 * np.abs(g).max()
    # the projected perturbation keeps about 2/3 of the energy of a mode with k = (2, 2, 2)
    assert 0.3 < np.sum(ps**2) / np.sum(s**2) < 1.0
