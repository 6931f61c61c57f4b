"""Pins of the oracle's D3Q27 variant (the same KBC method on the 27-velocity set): lattice,
equilibrium, shear part as the moment-space projection in the full 27-monomial basis,
collision invariants and special cases, the closed-form gamma as the root of the linearised
stationarity condition, streaming and conservation, and second-order viscous decay."""
from fractions import Fraction

import numpy as np
import pytest

import ensemble_inputs as gen
import oracle

Q = 27
WF = {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)}


def test_velocity_set_is_d3q27():
    c, w, opp = oracle.lattice(Q)
    assert len({tuple(v) for v in c}) == 27 and np.all(np.abs(c) <= 1)
    n2 = (c * c).sum(1)
    for i in range(Q):
        assert (c[opp[i]] == -c[i]).all()
        assert w[i] == float(WF[int(n2[i])])


def test_weight_moments_isotropic_exact():
    c, w, _ = oracle.lattice(Q)
    wf = [WF[int((v * v).sum())] for v in c]
    assert sum(wf) == 1
    for a in range(3):
        assert sum(wf[i] * c[i, a] for i in range(Q)) == 0
        assert sum(wf[i] * c[i, a] ** 4 for i in range(Q)) == Fraction(1, 3)
        for b in range(3):
            assert sum(wf[i] * c[i, a] * c[i, b] for i in range(Q)) == (Fraction(1, 3) if a == b else 0)
            for g in range(3):
                assert sum(wf[i] * c[i, a] * c[i, b] * c[i, g] for i in range(Q)) == 0
            if a != b:
                assert sum(wf[i] * c[i, a] ** 2 * c[i, b] ** 2 for i in range(Q)) == Fraction(1, 9)
    assert sum(wf[i] * c[i, 0] ** 2 * c[i, 1] ** 2 * c[i, 2] ** 2 for i in range(Q)) == Fraction(1, 27)


def test_equilibrium_moments():
    c, w, _ = oracle.lattice(Q)
    rho, u = 1.03, np.array([0.04, -0.03, 0.02])
    feq = oracle.equilibrium(rho, u, lattice=Q)
    assert abs(feq.sum() - rho) <= 1e-15 * rho
    np.testing.assert_allclose(c.T @ feq, rho * u, rtol=0, atol=1e-16)
    P = np.einsum("ia,ib,i->ab", c, c, feq)
    np.testing.assert_allclose(P, rho * (np.eye(3) / 3 + np.outer(u, u)), rtol=0, atol=2e-16)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_shear_part_is_the_moment_space_projection(seed):
    """Ds = M^-1 m_s for the invertible matrix of the 27 raw monomials c_x^a c_y^b c_z^c
    (a, b, c <= 2), m_s carrying only the deviatoric second moments of f^neq."""
    c, w, _ = oracle.lattice(Q)
    expo = [(a, b, g) for a in range(3) for b in range(3) for g in range(3)]
    Mm = np.array([c[:, 0] ** a * c[:, 1] ** b * c[:, 2] ** g for a, b, g in expo], dtype=float)
    assert np.linalg.matrix_rank(Mm) == Q
    fneq = 1e-3 * gen.uniform(seed, Q)
    ds = oracle.shear_part(fneq)
    P = np.einsum("ia,ib,i->ab", c, c, fneq)
    D = P - np.eye(3) * np.trace(P) / 3
    m_s = np.zeros(Q)
    for k, e in enumerate(expo):
        if sum(e) == 2:
            a, b = [d for d in range(3) for _ in range(e[d])]
            m_s[k] = D[a, b]
    np.testing.assert_allclose(ds, np.linalg.solve(Mm, m_s), rtol=0, atol=1e-17)


def _random_node(seed, amp=1e-2):
    c, w, _ = oracle.lattice(Q)
    r = gen.uniform(seed, 4 + Q)
    f = oracle.equilibrium(1.0 + 0.02 * r[0], 0.05 * r[1:4], lattice=Q) + amp * w * r[4:]
    return f


@pytest.mark.parametrize("seed", [10, 11])
def test_collision_invariants_and_bgk_cases(seed):
    c, w, _ = oracle.lattice(Q)
    f = _random_node(seed)
    rho = f.sum()
    feq = oracle.equilibrium(rho, (c.T @ f) / rho, lattice=Q)
    fs, g, ds, dh = oracle.collide(f, omega=1.7)
    assert abs(fs.sum() - f.sum()) <= 1e-15
    np.testing.assert_allclose(c.T @ fs, c.T @ f, rtol=0, atol=1e-16)
    np.testing.assert_allclose(ds + dh, f - feq, rtol=0, atol=1e-16)  # an ulp of f ~ 0.3
    fs1, g1, *_ = oracle.collide(f, omega=1.0)  # omega = 1: gamma = 2, BGK
    assert g1 == 2.0
    np.testing.assert_allclose(fs1, feq, rtol=2e-15, atol=1e-17)
    fe, *_ = oracle.collide(feq, omega=1.9)  # equilibrium is a fixed point
    np.testing.assert_allclose(fe, feq, rtol=1e-15, atol=0)


@pytest.mark.parametrize("seed", range(30, 46))
def test_closed_form_gamma_is_root_of_linearised_stationarity(seed):
    c, w, _ = oracle.lattice(Q)
    f = _random_node(seed, amp=5e-3)
    omega = 1.95
    fs, g, ds, dh = oracle.collide(f, omega)
    rho = f.sum()
    feq = oracle.equilibrium(rho, (c.T @ f) / rho, lattice=Q)

    def cond(gp):
        return np.sum(dh * (f - omega * ds - 0.5 * omega * gp * dh - feq) / feq)

    lo, hi = -50.0, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (cond(mid) > 0) == (cond(lo) > 0):
            lo = mid
        else:
            hi = mid
    assert abs(0.5 * (lo + hi) - g) <= 1e-12 * abs(g)


def test_streaming_and_conservation():
    c, w, _ = oracle.lattice(Q)
    un = oracle.units(8, 100.0, 0.1)
    f = oracle.init_ensemble(8, gen.draw_params(0, 1), un["ulat"], lattice=Q)
    f = f + 1e-4 * w[None, :, None, None, None] * gen.uniform(1, f.shape)
    before = f.copy()
    mass0 = f.sum()
    mom0 = np.einsum("ia,mizyx->a", c, f)
    oracle.step(f, un["omega"])
    for z, y, x in [(0, 0, 0), (3, 5, 7), (7, 7, 7)]:
        fs, *_ = oracle.collide(before[0, :, z, y, x], un["omega"])
        for i in range(Q):
            assert f[0, i, (z + c[i, 2]) % 8, (y + c[i, 1]) % 8, (x + c[i, 0]) % 8] == fs[i]
    oracle.run(f, un["omega"], 50)
    assert abs(f.sum() - mass0) <= 1e-13 * mass0
    np.testing.assert_allclose(np.einsum("ia,mizyx->a", c, f), mom0, rtol=0, atol=1e-13 * mass0)


def _shear_wave_error(N):
    un = oracle.units(N, 20.0, 0.05)
    ulat, nu, om = un["ulat"], un["nu_lat"], un["omega"]
    x = 2 * np.pi * np.arange(N) / N
    f = np.zeros((1, Q, N, N, N))
    for iy in range(N):
        f[0, :, :, iy, :] = oracle.equilibrium(1.0, np.array([0.5 * ulat * np.sin(x[iy]), 0.0, 0.0]),
                                               lattice=Q)[:, None, None]
    k = 2 * np.pi / N
    nsteps = int(round(0.5 / (nu * k * k)))
    oracle.run(f, om, nsteps)
    _, u = oracle.moments(f)
    s = np.sin(x)[None, :, None]
    amp = np.sum(u[0, 0] * s) / np.sum(np.broadcast_to(s, u[0, 0].shape) ** 2)
    return amp / (0.5 * ulat * np.exp(-nu * k * k * nsteps)) - 1.0


def test_shear_wave_decays_at_the_viscous_rate():
    e16, e32 = _shear_wave_error(16), _shear_wave_error(32)
    assert abs(e32) < 6e-3
    assert 3.0 < e16 / e32 < 5.0
