"""NumPy front end of the C oracle stepper (test infrastructure only).

Arrays are C-contiguous float64 (or complex128 for the complex-step twin).
Population fields are [M][Q][N][N][N] (x fastest, Q = 19 for D3Q19, the paper's
velocity set, or 27 for D3Q27) in the oracle's own velocity order, which
``lattice(Q)`` reports.  Functions taking a population field infer Q from it;
the others take ``lattice=19`` or ``27``.
"""
import ctypes

import numpy as np

from .build import load_oracle

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _ptr(a, dtype):
    assert a.dtype == dtype and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_dp)


def _arr(a, cplx=False):
    dt = np.complex128 if cplx else np.float64
    return np.ascontiguousarray(a, dtype=dt)


def _fn(name, cplx=False, lattice=19):
    assert lattice in (19, 27)
    lib = load_oracle()
    return getattr(lib, ("orcz" if cplx else "orc") + ("27_" if lattice == 27 else "_") + name)


def lattice(lattice=19):
    """(c [Q,3] int, w [Q] float64, opp [Q] int) of the oracle's D3Q19 or D3Q27 set."""
    c = np.zeros((lattice, 3), dtype=np.int32)
    w = np.zeros(lattice)
    opp = np.zeros(lattice, dtype=np.int32)
    _fn("lattice", lattice=lattice)(c.ctypes.data_as(_ip), _ptr(w, np.float64), opp.ctypes.data_as(_ip))
    return c.astype(np.int64), w, opp.astype(np.int64)


def units(N, Re, Ma, Uc=1.0):
    """Diffusive-scaling units: dict dx, ulat, dt, nu_lat, tau, omega."""
    out = np.zeros(6)
    fn = load_oracle().orc_units
    fn.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
    fn(int(N), float(Re), float(Ma), float(Uc), _ptr(out, np.float64))
    return dict(zip(("dx", "ulat", "dt", "nu_lat", "tau", "omega"), out.tolist()))


def equilibrium(rho, u, lattice=19):
    """f^eq(rho, u) of Eq. (equilibrium), real arguments."""
    u = _arr(u)
    feq = np.zeros(lattice)
    fn = _fn("equilibrium", lattice=lattice)
    fn.argtypes = [ctypes.c_double, _dp, _dp]
    fn(float(rho), _ptr(u, np.float64), _ptr(feq, np.float64))
    return feq


def shear_part(fneq):
    fneq = _arr(fneq)
    ds = np.zeros(len(fneq))
    _fn("shear_part", lattice=len(fneq))(_ptr(fneq, np.float64), _ptr(ds, np.float64))
    return ds


class exact_gamma:
    """Context manager: within it the real oracle (both velocity sets) takes the exact entropic
    gamma of Eq. (kbc_entropy) (bisection) instead of the closed form, Eq. (entropyControl)."""

    def __enter__(self):
        for q in (19, 27):
            _fn("set_exact_gamma", lattice=q)(1)
        return self

    def __exit__(self, *exc):
        for q in (19, 27):
            _fn("set_exact_gamma", lattice=q)(0)
        return False

    @staticmethod
    def counts(lattice=19):
        """How the nodes collided since the context was entered were decided: a dict of counts
        'dh_zero' (gamma = 2), 'empty' (no g keeps every f* positive: closed form kept),
        'lower_end', 'upper_end' (the constraint binds) and 'interior' (the unconstrained
        root of Eq. (kbc_entropy) lies inside the interval and is taken)."""
        out = (ctypes.c_longlong * 5)()
        fn = _fn("exact_gamma_counts", lattice=lattice)
        fn.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        fn(out)
        return dict(zip(("dh_zero", "empty", "lower_end", "upper_end", "interior"), list(out)))


def collide(f, omega, cplx=False):
    """One-node KBC collision: returns (f*, gamma, Ds, Dh)."""
    f = _arr(f, cplx)
    dt = f.dtype
    q = len(f)
    fs = np.zeros(q, dtype=dt)
    ds = np.zeros(q, dtype=dt)
    dh = np.zeros(q, dtype=dt)
    g = np.zeros(1, dtype=dt)
    fn = _fn("collide", cplx, q)
    fn.argtypes = [_dp, ctypes.c_double, _dp, _dp, _dp, _dp]
    fn(_ptr(f, dt), float(omega), _ptr(fs, dt), _ptr(g, dt), _ptr(ds, dt), _ptr(dh, dt))
    return fs, g[0], ds, dh


def init_ensemble(N, params, ulat, uc=1.0, density_mode=0, M=None, cplx=False, lattice=19):
    """Equilibrium-initialised RTGV ensemble [M][Q][N][N][N]; params [M][24] or None."""
    dt = np.complex128 if cplx else np.float64
    if params is not None:
        params = _arr(params, cplx).reshape(-1, 24)
        M = params.shape[0]
    assert M is not None
    f = np.zeros((M, lattice, N, N, N), dtype=dt)
    fn = _fn("init", cplx, lattice)
    fn.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp]
    fn(int(N), int(M), None if params is None else _ptr(params, dt), float(ulat), float(uc), int(density_mode),
       _ptr(f, dt))
    return f


def rtgv_fields(N, params, uc=1.0):
    """(u_det [3][N][N][N], s [M][3][N][N][N]) of Eqs. (tgv_init_velo) and
    (alpha_perturbation) on the nodes x_n = 2 pi n / N (array axes z, y, x), physical units."""
    params = np.asarray(params).reshape(-1, 24)
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    udet = np.stack([uc * np.sin(X) * np.cos(Y) * np.cos(Z), -uc * np.cos(X) * np.sin(Y) * np.cos(Z),
                     np.zeros_like(X)])
    a = [[np.sin(2 * X), np.cos(2 * X)], [np.sin(2 * Y), np.cos(2 * Y)], [np.sin(2 * Z), np.cos(2 * Z)]]
    s = np.zeros((params.shape[0], 3, N, N, N), dtype=np.result_type(params.dtype, np.float64))
    for m in range(params.shape[0]):
        for al in range(3):
            for i in range(2):
                for j in range(2):
                    for k in range(2):
                        s[m, al] += params[m, 8 * al + 4 * i + 2 * j + k] * a[0][i] * a[1][j] * a[2][k]
    return udet, s / 8.0


def leray_project(v):
    """Leray projection P v = v - grad Delta^-1 div v of periodic fields v [..][3][N][N][N]
    (array axes z, y, x; domain [0, 2 pi)^3): per Fourier mode k, (I - k k^T / |k|^2) v_k,
    the mean (k = 0) kept.  numpy.fft serves as the transform."""
    v = np.asarray(v)
    N = v.shape[-1]
    k1 = np.fft.fftfreq(N, d=1.0 / N)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    K = [KX, KY, KZ]
    K2 = KX**2 + KY**2 + KZ**2
    K2[0, 0, 0] = 1.0
    vh = np.fft.fftn(v, axes=(-3, -2, -1))
    kdotv = sum(K[a] * vh[..., a, :, :, :] for a in range(3))
    out = np.empty_like(vh)
    for a in range(3):
        out[..., a, :, :, :] = vh[..., a, :, :, :] - K[a] * kdotv / K2
    res = np.fft.ifftn(out, axes=(-3, -2, -1))
    return res.real if not np.iscomplexobj(v) else res


def init_ensemble_leray(N, params, ulat, uc=1.0, cplx=False, lattice=19):
    """RTGV ensemble initialised with the Leray-projected perturbation, u_0 = (U_lat / U_c)
    (u_det + P s) (Sec. "Discretization and well-prepared initial data"), f_0 = f^eq(1, u_0)."""
    dt = np.complex128 if cplx else np.float64
    params = np.asarray(params, dtype=dt).reshape(-1, 24)
    M = params.shape[0]
    udet, s = rtgv_fields(N, params, uc)
    if cplx:  # the projection of the real and imaginary parts separately (P is a real operator)
        ps = leray_project(s.real) + 1j * leray_project(s.imag)
    else:
        ps = leray_project(s)
    u = np.ascontiguousarray(((udet[None] + ps) * (ulat / uc)).reshape(M, 3, N * N * N), dtype=dt)
    f = np.zeros((M, lattice, N, N, N), dtype=dt)
    fn = _fn("init_velocity", cplx, lattice)
    fn.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
    fn(int(N), int(M), _ptr(u, dt), _ptr(f, dt))
    return f


def step(f, omega, with_gamma=False):
    """Advance f (modified in place) by one stream+collide step; optionally return gamma [M][N^3]."""
    cplx = f.dtype == np.complex128
    M, q, N = f.shape[0], f.shape[1], f.shape[2]
    assert q in (19, 27) and f.flags["C_CONTIGUOUS"]
    scratch = np.empty_like(f)
    g = np.zeros((M, N * N * N), dtype=f.dtype) if with_gamma else None
    fn = _fn("step", cplx, q)
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
    fn(int(N), int(M), float(omega), _ptr(f, f.dtype), _ptr(scratch, f.dtype),
       None if g is None else _ptr(g, f.dtype))
    return g


def run(f, omega, nsteps):
    """Advance f (in place) by nsteps steps."""
    cplx = f.dtype == np.complex128
    M, N = f.shape[0], f.shape[2]
    scratch = np.empty_like(f)
    fn = _fn("run", cplx, f.shape[1])
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
    fn(int(N), int(M), float(omega), int(nsteps), _ptr(f, f.dtype), _ptr(scratch, f.dtype))
    return f


def moments(f):
    """(rho [M][N][N][N], u [M][3][N][N][N]) in lattice units."""
    cplx = f.dtype == np.complex128
    M, N = f.shape[0], f.shape[2]
    rho = np.zeros((M, N, N, N), dtype=f.dtype)
    u = np.zeros((M, 3, N, N, N), dtype=f.dtype)
    fn = _fn("moments", cplx, f.shape[1])
    fn.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    fn(int(N), int(M), _ptr(f, f.dtype), _ptr(rho, f.dtype), _ptr(u, f.dtype))
    return rho, u


def energy(u, ulat, uc=1.0):
    """(E [M], Z [M]): kinetic energy and enstrophy per sample, physical units."""
    cplx = u.dtype == np.complex128
    u = np.ascontiguousarray(u)
    M, N = u.shape[0], u.shape[2]
    E = np.zeros(M, dtype=u.dtype)
    Z = np.zeros(M, dtype=u.dtype)
    fn = _fn("energy", cplx)
    fn.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
    fn(int(N), int(M), _ptr(u, u.dtype), float(ulat), float(uc), _ptr(E, u.dtype), _ptr(Z, u.dtype))
    return E, Z


def hrel(f):
    """Global relative entropy H_rel, Eq. (relEntropy2)."""
    f = _arr(f)
    M, N = f.shape[0], f.shape[2]
    fn = _fn("hrel", lattice=f.shape[1])
    fn.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
    fn.restype = ctypes.c_double
    return fn(int(N), int(M), _ptr(f, np.float64))


def complex_step_grad(N, params, ulat, omega, nsteps, objective="energy", h=1e-30, uc=1.0, lattice=19):
    """d J / d X (J = mean kinetic energy or enstrophy of each sample at step nsteps)
    by complex-step differentiation of the whole oracle: J(X + i h e_k) has imaginary
    part h dJ/dX_k to machine precision.  Returns [M][24]."""
    params = np.asarray(params, dtype=np.float64).reshape(-1, 24)
    M = params.shape[0]
    grad = np.zeros((M, 24))
    for k in range(24):
        p = params.astype(np.complex128)
        p[:, k] += 1j * h
        f = init_ensemble(N, p, ulat, uc, cplx=True, lattice=lattice)
        run(f, omega, nsteps)
        _, u = moments(f)
        E, Z = energy(u, ulat, uc)
        J = E if objective == "energy" else Z
        grad[:, k] = J.imag / h
    return grad
