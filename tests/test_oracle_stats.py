"""Pins of the oracle's ensemble statistics: closed forms, brute force on tiny grids,
independent library routines and invariants."""
from itertools import permutations

import numpy as np
import pytest

import ensemble_inputs as gen
from oracle import stats


def _grid(N):
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def _tgv(N, U=1.0):
    X, Y, Z = _grid(N)
    u = np.zeros((1, 3, N, N, N))
    u[0, 0] = U * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[0, 1] = -U * np.cos(X) * np.sin(Y) * np.cos(Z)
    return u


def test_shell_counts():
    """|S_1| = 18, |S_2| = 62, |S_3| = 98 (integer points with round(|k|) = kappa)."""
    cnt = stats.shell_counts(16)
    assert cnt[0] == 1 and cnt[1] == 18 and cnt[2] == 62 and cnt[3] == 98


@pytest.mark.parametrize("N", [8, 16])
def test_spectrum_of_tgv(N):
    """TGV (Eq. (tgv_init_velo)) puts all energy in the 8 modes (+-1,+-1,+-1), |k|^2 = 3,
    shell kappa = 2: E(2) = 4 pi / 62 * (1/2) * 3 * (U^2/4) = 3 pi U^2 / 124."""
    U = 0.7
    E = stats.energy_spectrum(_tgv(N, U))[0]
    assert abs(E[2] - 3 * np.pi * U**2 / 124) < 1e-14
    assert np.all(np.abs(np.delete(E, 2)) < 1e-15)


def test_spectrum_of_single_mode_and_perturbation_shell():
    """A sin x: E(1) = pi A^2 / 18.  A product a_i(2x)a_j(2y)a_k(2z) lands in kappa = 3
    (|k|^2 = 12) with E(3) = 4 pi / 98 * (1/2) * 12 * mean(u^2)."""
    N, A = 16, 0.3
    X, Y, Z = _grid(N)
    u = np.zeros((1, 3, N, N, N))
    u[0, 1] = A * np.sin(X)
    E = stats.energy_spectrum(u)[0]
    assert abs(E[1] - np.pi * A**2 / 18) < 1e-15
    u = np.zeros((1, 3, N, N, N))
    u[0, 2] = A * np.cos(2 * X) * np.sin(2 * Y) * np.cos(2 * Z)
    E = stats.energy_spectrum(u)[0]
    assert abs(E[3] - 4 * np.pi / 98 * 0.5 * 12 * A**2 / 8) < 1e-15


def test_spectrum_parseval_on_random_field():
    """Parseval with the /N^3 normalisation of Eq. (dftCoeff): a field of four plane-wave
    terms of known |k|^2 has energy N^-3 sum |u|^2 / 2 equal to the sum of the terms'
    mean squares / 2, and each shell of Eq. (energySpecDisc) holds 4 pi / |S| |k|^2 times
    the energy of the terms that fall in it."""
    N = 16
    X, Y, Z = _grid(N)
    r = gen.uniform(7, 8)
    u = np.zeros((1, 3, N, N, N))
    u[0, 0] = r[0] * np.sin(X + r[1]) + r[2] * np.cos(2 * Y + 3 * Z)
    u[0, 1] = r[3] * np.cos(3 * X - Y)
    u[0, 2] = r[4] * np.sin(X + Y + Z + r[5])
    E = stats.energy_spectrum(u)[0]
    direct = 0.5 * np.mean(np.sum(u[0] ** 2, axis=0))
    # energies per term (mean square / 2) with their |k|^2 and shell
    terms = [(0.5 * r[0] ** 2 / 2, 1), (0.5 * r[2] ** 2 / 2, 13), (0.5 * r[3] ** 2 / 2, 10), (0.5 * r[4] ** 2 / 2, 3)]
    assert abs(sum(t for t, _ in terms) - direct) < 1e-14
    cnt = stats.shell_counts(N)
    by_shell = {}
    for e, k2 in terms:
        kap = int(np.rint(np.sqrt(k2)))
        by_shell[kap] = by_shell.get(kap, 0) + 4 * np.pi / cnt[kap] * k2 * e
    for kap, val in by_shell.items():
        assert abs(E[kap] - val) < 1e-14


def _brute_autocorr(u_m):
    N = u_m.shape[-1]
    R = np.zeros((N, N, N))
    for hz in range(N):
        for hy in range(N):
            for hx in range(N):
                sh = np.roll(u_m, shift=(-hz, -hy, -hx), axis=(1, 2, 3))
                R[hz, hy, hx] = np.mean(np.sum(u_m * sh, axis=0))
    return R


def test_autocorrelation_wiener_khinchin_matches_brute_force():
    """Eq. (SF_approx_spec3) evaluated directly (O(N^6)) equals the FFT route of Eq.
    (SF_approx_spec5) on an 8^3 random field; R_0 = mean |u|^2."""
    u = gen.normal(3, (3, 8, 8, 8))
    R = stats.autocorrelation(u)
    Rb = _brute_autocorr(u)
    np.testing.assert_allclose(R, Rb, rtol=0, atol=1e-13)
    assert abs(R[0, 0, 0] - np.mean(np.sum(u * u, axis=0))) < 1e-13


def test_sf_trace_brute_force_and_single_mode():
    """S2 of Algorithm "SF_spectral" from a brute-force R_h with lags h in {-N/2+1..N/2}^3
    binned by round(|h|); and for u = (A sin x, 0, 0): R_h = (A^2/2) cos(2 pi h_x / N)."""
    N = 8
    u = gen.normal(4, (1, 3, N, N, N))
    S = stats.structure_function_trace(u)[0]
    Rb = _brute_autocorr(u[0])
    h = np.arange(N)
    h = np.where(h > N // 2, h - N, h)
    hz, hy, hx = np.meshgrid(h, h, h, indexing="ij")
    shell = np.rint(np.sqrt(hx**2 + hy**2 + hz**2)).astype(int)
    for r in range(N // 2 + 1):
        sel = shell == r
        assert abs(S[r] - np.mean(2 * (Rb[0, 0, 0] - Rb[sel]))) < 1e-13
    A = 0.4
    X, Y, Z = _grid(N)
    u = np.zeros((1, 3, N, N, N))
    u[0, 0] = A * np.sin(X)
    S = stats.structure_function_trace(u)[0]
    for r in range(N // 2 + 1):
        sel = shell == r
        expect = np.mean(2 * (A**2 / 2) * (1 - np.cos(2 * np.pi * hx[sel] / N)))
        assert abs(S[r] - expect) < 1e-15


def test_sf_axes_brute_force_and_closed_form():
    """S_p along axes by explicit loops on 8^3, and for u = (A sin x, 0, 0):
    S_2(r) = (1/3) A^2 (1 - cos(r dx))."""
    N, pmax = 8, 6
    u = gen.normal(5, (2, 3, N, N, N))
    S = stats.structure_function_axes(u, pmax)
    for m in range(2):
        for r in (1, 2, 4):
            for p in (2, 3, 6):
                acc = 0.0
                for z in range(N):
                    for y in range(N):
                        for x in range(N):
                            acc += abs(u[m, 0, z, y, (x + r) % N] - u[m, 0, z, y, x]) ** p
                            acc += abs(u[m, 1, z, (y + r) % N, x] - u[m, 1, z, y, x]) ** p
                            acc += abs(u[m, 2, (z + r) % N, y, x] - u[m, 2, z, y, x]) ** p
                assert abs(S[m, p - 2, r - 1] - acc / (3 * N**3)) < 1e-12 * max(1.0, acc / (3 * N**3))
    A = 0.5
    X, Y, Z = _grid(N)
    u = np.zeros((1, 3, N, N, N))
    u[0, 0] = A * np.sin(X)
    S = stats.structure_function_axes(u, 2)
    for r in range(1, N // 2 + 1):
        assert abs(S[0, 0, r - 1] - A**2 * (1 - np.cos(2 * np.pi * r / N)) / 3) < 1e-15


@pytest.mark.parametrize("M", [2, 3, 5, 7])
def test_w1_equals_min_over_permutations(M):
    """Eq. (wassersteinPermutations): brute-force minimum over S_M equals the CDF form."""
    a = gen.normal(10 + M, M)
    b = gen.normal(20 + M, M) + 0.3
    best = min(np.mean(np.abs(a - b[list(p)])) for p in permutations(range(M)))
    assert abs(stats.w1_empirical(a, b) - best) < 1e-14


def test_w1_invariants_and_unequal_sizes():
    a = gen.normal(1, 40)
    assert abs(stats.w1_empirical(a, a + 0.25) - 0.25) < 1e-14  # shift invariance
    assert stats.w1_empirical(a, a) == 0.0
    scipy_stats = pytest.importorskip("scipy.stats")
    for ma, mb in [(7, 13), (64, 32), (5, 5)]:
        x = gen.normal(ma, ma)
        y = gen.uniform(mb, mb)
        assert abs(stats.w1_empirical(x, y) - scipy_stats.wasserstein_distance(x, y)) < 1e-14


def test_w1_one_point_restriction_and_sum():
    """Algorithm "WassersteinDistance1": restriction to the 8^3 nodes n = j N / 8 and
    (1/Q^3) sum_points sum_components W1."""
    N = 16
    ua = gen.normal(30, (4, 3, N, N, N))
    ub = gen.normal(31, (6, 3, N, N, N))
    ra, rb = stats.restrict(ua), stats.restrict(ub)
    assert ra.shape == (4, 512, 3)
    # node (jz, jy, jx) = (1, 2, 3) -> index (1*8 + 2)*8 + 3, lattice node (2, 4, 6)
    np.testing.assert_array_equal(ra[:, (1 * 8 + 2) * 8 + 3, 1], ua[:, 1, 2, 4, 6])
    W, D = stats.w1_one_point(ra, rb, per_point=True)
    assert abs(W - D.sum() / 512) < 1e-15
    assert abs(D[77, 2] - stats.w1_empirical(ra[:, 77, 2], rb[:, 77, 2])) == 0.0


def test_energy_enstrophy_closed_forms():
    """KE of the TGV is U^2/8; its central-difference enstrophy is (3/8) U^2 s^2 with
    s = sin(dx)/dx (each discrete derivative of a unit mode carries the factor s)."""
    N, U = 16, 0.9
    u = _tgv(N, U)
    assert abs(stats.kinetic_energy(u)[0] - U**2 / 8) < 1e-15
    dx = 2 * np.pi / N
    s = np.sin(dx) / dx
    assert abs(stats.enstrophy(u)[0] - 3 / 8 * U**2 * s**2) < 1e-14


def test_mean_var_two_samples_closed_form():
    a = gen.normal(40, (1, 3, 4, 4, 4))
    b = gen.normal(41, (1, 3, 4, 4, 4))
    mean, var = stats.mean_var(np.concatenate([a, b]))
    np.testing.assert_allclose(mean, 0.5 * (a[0] + b[0]), rtol=1e-15)
    np.testing.assert_allclose(var, 0.5 * (a[0] - b[0]) ** 2, rtol=1e-13)


def test_sample_error_closed_forms():
    """Eq. (sample_error): a field scaled by (1 + s) has relative L1 error |s| in every component
    and in the vector norm; identical fields have error 0; the error is the mean of the
    per-sample ratios."""
    from oracle import stats as st
    uref = gen.uniform(61, (5, 64, 3)) + 0.2
    s = np.array([0.1, -0.3, 0.02, 0.5, -0.05])[:, None, None]
    e = st.sample_error(uref * (1 + s), uref)
    assert np.allclose(e, np.mean(np.abs(s)), rtol=1e-14)
    assert np.all(st.sample_error(uref, uref) == 0.0)
    u = uref.copy()
    u[0, 3, 1] += 0.25  # one node of one sample in the y component
    e = st.sample_error(u, uref)
    assert abs(e[1] - 0.25 / np.abs(uref[0, :, 1]).sum() / 5) <= 1e-15
    assert e[0] == 0.0 and e[2] == 0.0
