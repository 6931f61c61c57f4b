"""FP64 NumPy oracle of the ensemble statistics (test infrastructure only).

Each function states the passage it follows.  Library primitives (numpy.fft,
numpy.sort) serve as single steps; nothing is blocked, fused or reordered
beyond the written definition.  Velocity fields are u [M][3][N][N][N]
(components x, y, z; array axes z, y, x) in physical units unless noted.
"""
import numpy as np


def to_physical(u_lat, ulat, uc=1.0):
    """u_phys = u_lat U_c / U_lat (lattice -> physical velocity)."""
    return np.asarray(u_lat, dtype=np.float64) * (uc / ulat)


def kinetic_energy(u):
    """E_m = (1/N^3) sum_x |u|^2 / 2 (energy per unit volume, Appendix
    "Computation of the energy spectrum": N^-d sum |u|^2 = sum Phi)."""
    u = np.asarray(u, dtype=np.float64)
    return 0.5 * np.mean(np.sum(u * u, axis=1), axis=(1, 2, 3))


def enstrophy(u):
    """Z_m = (1/N^3) sum_x |curl u|^2 / 2 with second-order central differences,
    dx = 2 pi / N (enstrophy is not defined in the paper; this is the reading
    used throughout the library)."""
    u = np.asarray(u, dtype=np.float64)
    N = u.shape[-1]
    dx = 2 * np.pi / N

    def d(field, axis):  # axis: 0 = x, 1 = y, 2 = z in physical terms
        ax = {0: -1, 1: -2, 2: -3}[axis]
        return (np.roll(field, -1, axis=ax) - np.roll(field, 1, axis=ax)) / (2 * dx)

    ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
    wx = d(uz, 1) - d(uy, 2)
    wy = d(ux, 2) - d(uz, 0)
    wz = d(uy, 0) - d(ux, 1)
    return 0.5 * np.mean(wx * wx + wy * wy + wz * wz, axis=(1, 2, 3))


def mean_var(u):
    """Ensemble mean and unbiased (M - 1) variance of every velocity component at
    every node, Eqs. (spectrum_mean), (spectrum_var) applied pointwise."""
    u = np.asarray(u, dtype=np.float64)
    M = u.shape[0]
    mean = u.sum(axis=0) / M
    var = ((u - mean) ** 2).sum(axis=0) / (M - 1)
    return mean, var


def _wavenumbers(N):
    """Signed integer wavenumber of every FFT index, in K_N = {-N/2+1, ..., N/2}."""
    k = np.fft.fftfreq(N, d=1.0 / N).astype(np.int64)
    k[k == -N // 2] = N // 2
    return k


def energy_spectrum(u):
    """Shell spectrum E_m(kappa), kappa = 0..N/2, Eqs. (dftCoeff), (energySpecDisc):
    u~ = DFT / N^3, Phi = |u~|^2, S_kappa = {k in K_N : round(|k|) = kappa},
    E_m(kappa) = 4 pi / |S_kappa| sum_{S_kappa} |k|^2 Phi / 2.  Returns [M][N/2+1]."""
    u = np.asarray(u, dtype=np.float64)
    M, N = u.shape[0], u.shape[-1]
    k = _wavenumbers(N)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    k2 = (kx * kx + ky * ky + kz * kz).astype(np.float64)
    shell = np.rint(np.sqrt(k2)).astype(np.int64)
    out = np.zeros((M, N // 2 + 1))
    for m in range(M):
        phi = np.zeros((N, N, N))
        for a in range(3):
            uh = np.fft.fftn(u[m, a]) / N**3
            phi += (uh * np.conj(uh)).real
        for kappa in range(N // 2 + 1):
            sel = shell == kappa
            cnt = int(sel.sum())
            out[m, kappa] = 4 * np.pi / cnt * np.sum(0.5 * k2[sel] * phi[sel])
    return out


def shell_counts(N):
    """|S_kappa| for kappa = 0..N/2 over K_N."""
    k = _wavenumbers(N)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    shell = np.rint(np.sqrt((kx * kx + ky * ky + kz * kz).astype(np.float64))).astype(np.int64)
    return np.array([(shell == r).sum() for r in range(N // 2 + 1)])


def autocorrelation(u_m):
    """R_h = N^-3 F^-1(sum_i |F(u_i)|^2)_h, Eq. (PSD_def) (F unnormalised forward,
    F^-1 with the factor N^-3, as numpy's ifftn)."""
    N = u_m.shape[-1]
    psi = np.zeros((N, N, N))
    for a in range(3):
        fh = np.fft.fftn(u_m[a])
        psi += (fh * np.conj(fh)).real
    return np.fft.ifftn(psi).real / N**3


def structure_function_trace(u):
    """S2_m(r), r = 0..N/2, Algorithm "SF_spectral": S2_m(r) = 1/|C_r| sum_{h in C_r}
    2 (R_0 - R_h), C_r = {h in {-N/2+1..N/2}^3 : round(|h|) = r}.  Returns [M][N/2+1]."""
    u = np.asarray(u, dtype=np.float64)
    M, N = u.shape[0], u.shape[-1]
    h = _wavenumbers(N)
    hz, hy, hx = np.meshgrid(h, h, h, indexing="ij")
    shell = np.rint(np.sqrt((hx * hx + hy * hy + hz * hz).astype(np.float64))).astype(np.int64)
    out = np.zeros((M, N // 2 + 1))
    for m in range(M):
        R = autocorrelation(u[m])
        for r in range(N // 2 + 1):
            sel = shell == r
            out[m, r] = np.sum(2.0 * (R[0, 0, 0] - R[sel])) / sel.sum()
    return out


def structure_function_axes(u, pmax=6, lags=None):
    """Longitudinal structure functions along the lattice axes, Eq. (structuresLocal)
    restricted to n in {e_x, e_y, e_z} with the modulus of Eq. (structures):
    S_p,m(r) = 1/(3 N^3) sum_x sum_a |u_a(x + r e_a) - u_a(x)|^p, r = 1..N/2,
    p = 2..pmax.  Returns [M][pmax-1][N/2] (index r-1); with `lags` (a list of r), only those
    entries are evaluated and the others stay zero (large lattices)."""
    u = np.asarray(u, dtype=np.float64)
    M, N = u.shape[0], u.shape[-1]
    out = np.zeros((M, pmax - 1, N // 2))
    axis_of = {0: -1, 1: -2, 2: -3}
    for m in range(M):
        for r in (range(1, N // 2 + 1) if lags is None else lags):
            incs = [np.abs(np.roll(u[m, a], -r, axis=axis_of[a]) - u[m, a]) for a in range(3)]
            for p in range(2, pmax + 1):
                out[m, p - 2, r - 1] = sum(np.sum(d**p) for d in incs) / (3 * N**3)
    return out


def restrict(u, Q=8):
    """Exact restriction to the common Q^3 grid (node n = j N / Q), Appendix
    "Computation of the Wasserstein distance".  Returns [M][Q^3][3]."""
    u = np.asarray(u, dtype=np.float64)
    N = u.shape[-1]
    assert N % Q == 0
    s = N // Q
    sub = u[:, :, ::s, ::s, ::s]  # [M][3][Q][Q][Q] (z, y, x)
    return np.ascontiguousarray(sub.reshape(u.shape[0], 3, Q**3).transpose(0, 2, 1))


def w1_empirical(a, b):
    """1-D W1 between the empirical laws of samples a and b (equal weights within
    each): the L1 distance of the two empirical CDFs over the merged support,
    which for equal sizes is the sorted-rearrangement cost (1/M) sum |a_(m) - b_(m)|."""
    a = np.sort(np.asarray(a, dtype=np.float64))
    b = np.sort(np.asarray(b, dtype=np.float64))
    allv = np.sort(np.concatenate([a, b]))
    deltas = np.diff(allv)
    Fa = np.searchsorted(a, allv[:-1], side="right") / a.size
    Fb = np.searchsorted(b, allv[:-1], side="right") / b.size
    return float(np.sum(np.abs(Fa - Fb) * deltas))


def w1_one_point(ua, ub, Q=8, per_point=False):
    """W_{1,1} of Algorithm "WassersteinDistance1": for each of the Q^3 points and each
    component the 1-D W1 between the two ensembles' values, summed over components and
    averaged over points.  ua [M_A][Q^3][3], ub [M_B][Q^3][3] (restricted fields)."""
    G = Q**3
    D = np.zeros((G, 3))
    for i in range(G):
        for c in range(3):
            D[i, c] = w1_empirical(ua[:, i, c], ub[:, i, c])
    total = D.sum() / G
    return (total, D) if per_point else total


def ot_w1_lp(X, Y):
    """W1 between the empirical laws of the rows of X [M_A][k] and Y [M_B][k] (atoms weighted
    1/M_A and 1/M_B) with the Euclidean ground metric: the transport linear program that the
    paper solves with an exact network-simplex call (Algorithms "WassersteinDistance2" and
    "WassersteinDistance2_vector"), min sum_ij pi_ij |X_i - Y_j| over pi >= 0 with row sums
    1/M_A and column sums 1/M_B, solved by scipy.optimize.linprog (HiGHS)."""
    from scipy.optimize import linprog
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    MA, MB = X.shape[0], Y.shape[0]
    C = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2))
    A_eq = np.zeros((MA + MB, MA * MB))
    for i in range(MA):
        A_eq[i, i * MB:(i + 1) * MB] = 1.0
    for j in range(MB):
        A_eq[MA + j, j::MB] = 1.0
    b_eq = np.concatenate([np.full(MA, 1.0 / MA), np.full(MB, 1.0 / MB)])
    # the solver's tolerances are absolute: solve with costs scaled to a unit maximum and
    # tightened tolerances, then scale the optimum back
    cmax = C.max()
    if cmax == 0.0:
        return 0.0
    res = linprog(C.ravel() / cmax, A_eq=A_eq, b_eq=b_eq, bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert res.status == 0
    return float(res.fun) * cmax


def ot_w1_assignment(X, Y):
    """Equal sizes M: the optimal plan of ot_w1_lp is a permutation matrix / M (the extreme points
    of the doubly stochastic matrices), so W1 = (1/M) min over permutations s of
    sum_m |X_m - Y_s(m)|; the assignment is solved by scipy.optimize.linear_sum_assignment."""
    from scipy.optimize import linear_sum_assignment
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    assert X.shape == Y.shape
    C = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2))
    r, c = linear_sum_assignment(C)
    return float(C[r, c].sum() / X.shape[0])


def ot_w1(X, Y):
    """ot_w1_assignment for equal sizes, ot_w1_lp otherwise."""
    return ot_w1_assignment(X, Y) if len(X) == len(Y) else ot_w1_lp(X, Y)


def pair_index(i, j, G):
    """Position of the point pair (i, j), i <= j, in the row-major upper triangle of G x G."""
    return i * G - i * (i - 1) // 2 + (j - i)


def w1_two_point(ua, ub, vector=True, per_pair=False):
    """Two-point W1 between the laws of two ensembles on the G restriction points.
    vector: W_{1,2}^v of Eq. (W1_vector) / Algorithm "WassersteinDistance2_vector", the W1 of
    the joint laws of (u(x_i), u(x_j)) in R^6 for every pair i <= j; otherwise W_{1,2} of
    Algorithm "WassersteinDistance2", the W1 of (u_c(x_i), u_c(x_j)) in R^2 for every pair and
    component c, summed over c.  Pairs with i != j count twice (the symmetric lower triangle);
    the sum is divided by G^2.  ua [M_A][G][3], ub [M_B][G][3] (restricted fields).
    per_pair: also return [G (G + 1) / 2] (vector) or [G (G + 1) / 2][3] values in pair_index
    order."""
    ua = np.asarray(ua, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    G = ua.shape[1]
    npairs = G * (G + 1) // 2
    D = np.zeros(npairs) if vector else np.zeros((npairs, 3))
    total = 0.0
    for i in range(G):
        for j in range(i, G):
            w = 1.0 if i == j else 2.0
            k = pair_index(i, j, G)
            if vector:
                D[k] = ot_w1(np.concatenate([ua[:, i, :], ua[:, j, :]], axis=1),
                             np.concatenate([ub[:, i, :], ub[:, j, :]], axis=1))
                total += w * D[k]
            else:
                for c in range(3):
                    D[k, c] = ot_w1(np.stack([ua[:, i, c], ua[:, j, c]], axis=1),
                                    np.stack([ub[:, i, c], ub[:, j, c]], axis=1))
                    total += w * D[k, c]
    total /= G * G
    return (total, D) if per_pair else total


def sample_error(u, uref):
    """Ensemble-averaged relative L1 error between paired samples on the restriction grid,
    Eq. (sample_error): (1/M) sum_m sum_k |u_m(x_k) - uref_m(x_k)| / sum_k |uref_m(x_k)|, for
    each velocity component (|.| the absolute value) and for the velocity vector (|.| the
    Euclidean norm).  u, uref [M][G][3] (the same samples m at two resolutions).  Returns
    [4]: x, y, z, vector."""
    u = np.asarray(u, dtype=np.float64)
    uref = np.asarray(uref, dtype=np.float64)
    out = np.zeros(4)
    for c in range(3):
        out[c] = np.mean(np.abs(u[:, :, c] - uref[:, :, c]).sum(axis=1) / np.abs(uref[:, :, c]).sum(axis=1))
    out[3] = np.mean(np.linalg.norm(u - uref, axis=2).sum(axis=1) / np.linalg.norm(uref, axis=2).sum(axis=1))
    return out
