/*
 * FP64 CPU oracle of the Monte Carlo KBC lattice Boltzmann scheme.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the timed CPU baseline
 * of the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library: the velocity set is enumerated here from its definition
 * and every formula is written out in the paper's notation.
 *
 * The file is compiled for two velocity sets (-DORC_Q=19: D3Q19, the paper's;
 * -DORC_Q=27: D3Q27) and twice for each: once with real_t = double (symbols
 * orc_* / orc27_*) and once with real_t = double complex (symbols orcz_* /
 * orcz27_*, -DORC_COMPLEX) so that the complex-step derivative of any scalar
 * of the whole simulation with respect to the 24 uncertainty parameters can be
 * taken through exactly the same code.  Only +, -, *, / act on real_t values,
 * so the complex build is the analytic continuation of the real one.
 *
 * Parity status: every function below is pinned by a CPU test (lattice
 * moments, equilibrium moments, shear part vs. the moment-space definition,
 * fixed points, conservation, closed-form gamma vs. a bisection root,
 * units vs. Table "params2", initial energy closed form, shear-wave decay).
 *
 * Layout of a population field: f[m][i][z][y][x], m < M samples, i < Q
 * velocities in this file's own enumeration order, n = N*N*N nodes with x
 * fastest.  The stored state at integer time t is the pre-collision one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifndef ORC_Q
#define ORC_Q 19
#endif
#if ORC_Q == 19
#define PFX_R orc_
#define PFX_C orcz_
#elif ORC_Q == 27
#define PFX_R orc27_
#define PFX_C orcz27_
#else
#error "ORC_Q must be 19 or 27"
#endif
#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)
/* RSYM: real-only entry points; SYM: entry points of both arithmetic twins */
#define RSYM(name) CAT(PFX_R, name)
#ifdef ORC_COMPLEX
#include <complex.h>
typedef double complex real_t;
#define SYM(name) CAT(PFX_C, name)
#define RE(v) creal(v)
#else
typedef double real_t;
#define SYM(name) CAT(PFX_R, name)
#define RE(v) (v)
#endif

#define Q ORC_Q

/* ---- Velocity set.  D3Q19 (Sec. "Entropic multi-relaxation lattice Boltzmann
 * scheme"): the 19 vectors of {-1,0,1}^3 with |c|^2 <= 2, weights 1/3, 1/18, 1/36
 * for |c|^2 = 0, 1, 2.  D3Q27: all 27 vectors of {-1,0,1}^3, weights 8/27, 2/27,
 * 1/54, 1/216 for |c|^2 = 0, 1, 2, 3 (the tensor product of the D1Q3 weights
 * 2/3, 1/6).  c_s^2 = 1/3 for both. ---- */
static int C[Q][3];
static double W[Q];
static int OPP[Q];
static int lattice_ready = 0;

static double shell_weight(int shell)
{
#if ORC_Q == 19
    static const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
#else
    static const double w[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
#endif
    return w[shell];
}

static void build_lattice(void)
{
    if (lattice_ready) return;
    int q = 0;
    const int max_shell = Q == 19 ? 2 : 3;
    /* rest, then faces, edges (and corners); within each shell a fixed scan order */
    for (int shell = 0; shell <= max_shell; ++shell)
        for (int cz = -1; cz <= 1; ++cz)
            for (int cy = -1; cy <= 1; ++cy)
                for (int cx = -1; cx <= 1; ++cx) {
                    int n2 = cx * cx + cy * cy + cz * cz;
                    if (n2 != shell) continue;
                    C[q][0] = cx; C[q][1] = cy; C[q][2] = cz;
                    W[q] = shell_weight(shell);
                    ++q;
                }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2]) OPP[i] = j;
    lattice_ready = 1;
}

static const double CS2 = 1.0 / 3.0;

#ifndef ORC_COMPLEX
void RSYM(lattice)(int *c, double *w, int *opp)
{
    build_lattice();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = C[i][a];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

/* Units under diffusive scaling (Sec. "Numerical validation of convergence
 * rates", Tables "params1/params2", Table "frequencySummary"):
 *   dx = 2 pi / N,  U_lat = Ma * c_s,  dt = U_lat dx / U_c,
 *   nu_phys = U_c l_c / Re (l_c = 1),  nu_lat = nu_phys dt / dx^2,
 *   omega_nu = 2 c_s^2 / (2 nu_lat + c_s^2),  tau = 1 / omega_nu.
 * out = {dx, U_lat, dt, nu_lat, tau, omega_nu}. */
void RSYM(units)(int N, double Re, double Ma, double Uc, double *out)
{
    const double pi = 3.14159265358979323846;
    double dx = 2.0 * pi / N;
    double ulat = Ma * sqrt(CS2);
    double dt = ulat * dx / Uc;
    double nu = Uc * 1.0 / Re;
    double nu_lat = nu * dt / (dx * dx);
    double omega = 2.0 * CS2 / (2.0 * nu_lat + CS2);
    out[0] = dx; out[1] = ulat; out[2] = dt; out[3] = nu_lat; out[4] = 1.0 / omega; out[5] = omega;
}
#endif

/* Second-order truncated equilibrium, Eq. (equilibrium):
 * f_i^eq = rho w_i [1 + c.u / c_s^2 + ((c.u)^2 - c_s^2 |u|^2) / (2 c_s^4)]. */
void SYM(equilibrium)(real_t rho, const real_t *u, real_t *feq)
{
    build_lattice();
    real_t uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        real_t cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        feq[i] = rho * W[i] * (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
    }
}

/* Conserved moments: rho = sum f, rho u = sum c f. */
void SYM(node_moments)(const real_t *f, real_t *rho, real_t *u)
{
    build_lattice();
    real_t r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += C[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* Shear part of the non-equilibrium populations (Sec. "Entropic
 * multi-relaxation", Table "frequencySummary"): the populations that carry
 * exactly the deviatoric raw second moments D_ab = P_ab - delta_ab tr(P)/3 of
 * f^neq (the shear tensors N and Pi) and nothing else of the lattice's raw
 * moment basis (for D3Q27 the 27 products c_x^a c_y^b c_z^c, a, b, c <= 2).
 * Written out per velocity class:
 *   rest:                      0
 *   face  +-e_a:               D_aa / 2
 *   edge  s e_a + l e_b:       s l P_ab / 4
 *   corner (D3Q27):            0.                                            */
void SYM(shear_part)(const real_t *fneq, real_t *ds)
{
    build_lattice();
    real_t P[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            P[a][b] = 0;
            for (int i = 0; i < Q; ++i) P[a][b] += C[i][a] * C[i][b] * fneq[i];
        }
    real_t tr = P[0][0] + P[1][1] + P[2][2];
    for (int i = 0; i < Q; ++i) {
        int n2 = C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2];
        if (n2 == 0) {
            ds[i] = 0;
        } else if (n2 == 1) {
            int a = C[i][0] ? 0 : (C[i][1] ? 1 : 2);
            ds[i] = 0.5 * (P[a][a] - tr / 3.0);
        } else if (n2 == 2) {
            int a = -1, b = -1;
            for (int k = 0; k < 3; ++k)
                if (C[i][k]) { if (a < 0) a = k; else b = k; }
            ds[i] = 0.25 * C[i][a] * C[i][b] * P[a][b];
        } else {
            ds[i] = 0;
        }
    }
}

/* KBC collision at one node, Eq. (kbcCollision) with the closed-form
 * stabiliser Eq. (entropyControl):
 *   f^neq = f - f^eq(rho, u),  Ds = shear part,  Dh = f^neq - Ds,
 *   <X|Y> = sum X_i Y_i / f_i^eq,
 *   gamma = 2/omega - (2 - 2/omega) <Ds|Dh> / <Dh|Dh>   (gamma = 2 if <Dh|Dh> = 0),
 *   f* = f - omega Ds - (omega gamma / 2) Dh.
 * Optional outputs gamma, ds, dh may be NULL. */
#ifndef ORC_COMPLEX
/* Exact entropic gamma of Eq. (kbc_entropy): the minimiser of H(f*(g)) = sum f*_i ln(f*_i / w_i)
 * over g, f*(g) = f - omega Ds - (omega g / 2) Dh, taken over 0 <= g <= 4 / omega (the range in
 * which the relaxation factor omega g / 2 of Dh stays in the stable [0, 2]; with the polynomial
 * equilibrium the unconstrained minimiser grows like 1 / |Dh| near equilibrium).
 * dH/dg = -(omega / 2) sum Dh_i (ln(f*_i / w_i) + 1) and sum Dh_i = 0, so the stationary point
 * is the root of G(g) = sum Dh_i ln(f*_i(g) / w_i); G decreases (G' = -(omega / 2)
 * sum Dh_i^2 / f*_i) where every f*_i > 0, so H is convex along the line and the constrained
 * minimiser is the root if it lies inside the interval, else the nearer end point.  The root is
 * found by bisection.  Dh = 0: gamma = 2 (the paper's BGK value). */
static int exact_gamma_mode = 0;

/* How each exact-gamma node was decided since the mode was last switched on, so that a run can
 * report how often the constraint binds: [0] Dh = 0 (gamma = 2), [1] empty positivity interval
 * (closed form kept), [2] minimiser at the lower end, [3] at the upper end, [4] interior root. */
static long long exact_gamma_counts[5];

void RSYM(set_exact_gamma)(int on)
{
    exact_gamma_mode = on;
    if (on)
        for (int k = 0; k < 5; ++k) exact_gamma_counts[k] = 0;
}

void RSYM(exact_gamma_counts)(long long *out)
{
    for (int k = 0; k < 5; ++k) out[k] = exact_gamma_counts[k];
}

static void count_exact_gamma(int k)
{
#pragma omp atomic
    exact_gamma_counts[k] += 1;
}

static double exact_gamma(const double *f, const double *ds, const double *dh, double omega, double g_closed)
{
    double A[Q], B[Q], lo = 0.0, hi = 4.0 / omega;
    for (int i = 0; i < Q; ++i) {
        A[i] = f[i] - omega * ds[i];
        B[i] = 0.5 * omega * dh[i];
        if (B[i] > 0) { double r = A[i] / B[i]; if (r < hi) hi = r; }
        if (B[i] < 0) { double r = A[i] / B[i]; if (r > lo) lo = r; }
    }
    if (!(lo < hi)) {
        count_exact_gamma(1);
        return g_closed;
    }
    /* H is convex along the line: the minimiser over [lo, hi] is an end point where G does not
     * change sign inside, else the root */
    double G_lo = 0, G_hi = 0;
    for (int i = 0; i < Q; ++i) {
        G_lo += dh[i] * log((A[i] - lo * B[i]) / W[i]);
        G_hi += dh[i] * log((A[i] - hi * B[i]) / W[i]);
    }
    if (!(G_lo > 0)) {
        count_exact_gamma(2);
        return lo;
    }
    if (!(G_hi < 0)) {
        count_exact_gamma(3);
        return hi;
    }
    count_exact_gamma(4);
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double G = 0;
        for (int i = 0; i < Q; ++i) G += dh[i] * log((A[i] - mid * B[i]) / W[i]);
        if (G > 0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}
#endif

void SYM(collide)(const real_t *f, double omega, real_t *fstar, real_t *gamma_out, real_t *ds_out,
                  real_t *dh_out)
{
    build_lattice();
    real_t rho, u[3], feq[Q], fneq[Q], ds[Q], dh[Q];
    SYM(node_moments)(f, &rho, u);
    SYM(equilibrium)(rho, u, feq);
    for (int i = 0; i < Q; ++i) fneq[i] = f[i] - feq[i];
    SYM(shear_part)(fneq, ds);
    for (int i = 0; i < Q; ++i) dh[i] = fneq[i] - ds[i];
    real_t sh = 0, hh = 0;
    for (int i = 0; i < Q; ++i) {
        sh += ds[i] * dh[i] / feq[i];
        hh += dh[i] * dh[i] / feq[i];
    }
    real_t gamma;
    if (RE(hh) == 0.0)
        gamma = 2.0;
    else
        gamma = 2.0 / omega - (2.0 - 2.0 / omega) * sh / hh;
#ifndef ORC_COMPLEX
    if (exact_gamma_mode) {
        if (hh != 0.0)
            gamma = exact_gamma(f, ds, dh, omega, gamma);
        else
            count_exact_gamma(0);
    }
#endif
    for (int i = 0; i < Q; ++i) fstar[i] = f[i] - omega * ds[i] - 0.5 * omega * gamma * dh[i];
    if (gamma_out) *gamma_out = gamma;
    if (ds_out) memcpy(ds_out, ds, sizeof ds);
    if (dh_out) memcpy(dh_out, dh, sizeof dh);
}

/* Ensemble initialisation, Eqs. (tgv_init_velo), (alpha_perturbation),
 * (initialRTGV), (initialPopulations): nodes x_n = 2 pi n / N,
 *   u_det = U_c (sin x cos y cos z, -cos x sin y cos z, 0),
 *   s_alpha = 1/8 sum_{ijk in {0,1}^3} X_{alpha,ijk} a_i(2x) a_j(2y) a_k(2z),
 *   a_0 = sin, a_1 = cos, parameter index 8 alpha + 4 i + 2 j + k,
 *   u_0 (lattice) = (U_lat / U_c) (u_det + s),   f_0 = f^eq(rho_0, u_0).
 * rho_0 = 1 (density_mode 0, the paper's choice), or the Taylor-Green
 * pressure density 1 + p / c_s^2 with p = (U_lat^2/16)(cos 2x + cos 2y)(cos 2z + 2)
 * (density_mode 1).  params: [M][24] (may be NULL for the deterministic TGV). */
void SYM(init)(int N, int M, const real_t *params, double ulat, double uc, int density_mode, real_t *f)
{
    build_lattice();
    const double pi = 3.14159265358979323846;
    const size_t n = (size_t)N * N * N;
    for (int m = 0; m < M; ++m) {
        const real_t *X = params ? params + 24 * (size_t)m : NULL;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < N; ++z)
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) {
                    double px = 2.0 * pi * x / N, py = 2.0 * pi * y / N, pz = 2.0 * pi * z / N;
                    real_t u[3];
                    u[0] = uc * sin(px) * cos(py) * cos(pz);
                    u[1] = -uc * cos(px) * sin(py) * cos(pz);
                    u[2] = 0.0;
                    if (X) {
                        double ax[2] = {sin(2 * px), cos(2 * px)};
                        double ay[2] = {sin(2 * py), cos(2 * py)};
                        double az[2] = {sin(2 * pz), cos(2 * pz)};
                        for (int al = 0; al < 3; ++al) {
                            real_t s = 0;
                            for (int i = 0; i < 2; ++i)
                                for (int j = 0; j < 2; ++j)
                                    for (int k = 0; k < 2; ++k)
                                        s += X[8 * al + 4 * i + 2 * j + k] * (ax[i] * ay[j] * az[k]);
                            u[al] += s / 8.0;
                        }
                    }
                    for (int a = 0; a < 3; ++a) u[a] *= ulat / uc;
                    real_t rho = 1.0;
                    if (density_mode == 1) {
                        double p = ulat * ulat / 16.0 * (cos(2 * px) + cos(2 * py)) * (cos(2 * pz) + 2.0);
                        rho = 1.0 + p / CS2;
                    }
                    real_t feq[Q];
                    SYM(equilibrium)(rho, u, feq);
                    size_t node = ((size_t)z * N + y) * N + x;
                    for (int i = 0; i < Q; ++i) f[((size_t)m * Q + i) * n + node] = feq[i];
                }
    }
}

/* One time step of Eq. (lbIteration) for every sample: collide every node,
 * then stream f_i(x + c_i) = f*_i(x) with periodic wrap.  f holds the
 * pre-collision state at t on entry and at t + 1 on exit; scratch has the
 * same size as f.  gamma_out (may be NULL): [M][n] stabiliser values. */
/* Equilibrium populations f = f^eq(1, u) from a given lattice-unit velocity field
 * u [M][3][n] (x fastest): Eq. (initialPopulations) for initial velocities built outside
 * this file (the Leray-projected RTGV of Sec. "Discretization and well-prepared initial
 * data" is assembled in the NumPy front end). */
void SYM(init_velocity)(int N, int M, const real_t *u, real_t *f)
{
    build_lattice();
    const size_t n = (size_t)N * N * N;
    for (int m = 0; m < M; ++m) {
#pragma omp parallel for schedule(static)
        for (long long node = 0; node < (long long)n; ++node) {
            real_t v[3], feq[Q];
            for (int a = 0; a < 3; ++a) v[a] = u[((size_t)m * 3 + a) * n + node];
            SYM(equilibrium)(1.0, v, feq);
            for (int i = 0; i < Q; ++i) f[((size_t)m * Q + i) * n + node] = feq[i];
        }
    }
}

void SYM(step)(int N, int M, double omega, real_t *f, real_t *scratch, real_t *gamma_out)
{
    build_lattice();
    const size_t n = (size_t)N * N * N;
    for (int m = 0; m < M; ++m) {
        real_t *fm = f + (size_t)m * Q * n;
        real_t *sm = scratch + (size_t)m * Q * n;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < N; ++z)
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) {
                    size_t node = ((size_t)z * N + y) * N + x;
                    real_t fl[Q], fs[Q], g;
                    for (int i = 0; i < Q; ++i) fl[i] = fm[i * n + node];
                    SYM(collide)(fl, omega, fs, &g, NULL, NULL);
                    for (int i = 0; i < Q; ++i) sm[i * n + node] = fs[i];
                    if (gamma_out) gamma_out[(size_t)m * n + node] = g;
                }
#pragma omp parallel for schedule(static)
        for (int z = 0; z < N; ++z)
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) {
                    size_t node = ((size_t)z * N + y) * N + x;
                    for (int i = 0; i < Q; ++i) {
                        int xd = (x + C[i][0] + N) % N, yd = (y + C[i][1] + N) % N, zd = (z + C[i][2] + N) % N;
                        size_t dst = ((size_t)zd * N + yd) * N + xd;
                        fm[i * n + dst] = sm[i * n + node];
                    }
                }
    }
}

void SYM(run)(int N, int M, double omega, int nsteps, real_t *f, real_t *scratch)
{
    for (int t = 0; t < nsteps; ++t) SYM(step)(N, M, omega, f, scratch, NULL);
}

/* Macroscopic moments of every node: rho [M][n], u [M][3][n] in lattice
 * units (u = (1/rho) sum c f). */
void SYM(moments)(int N, int M, const real_t *f, real_t *rho, real_t *u)
{
    build_lattice();
    const size_t n = (size_t)N * N * N;
    for (int m = 0; m < M; ++m) {
#pragma omp parallel for schedule(static)
        for (long long node = 0; node < (long long)n; ++node) {
            real_t fl[Q], r, v[3];
            for (int i = 0; i < Q; ++i) fl[i] = f[((size_t)m * Q + i) * n + node];
            SYM(node_moments)(fl, &r, v);
            rho[(size_t)m * n + node] = r;
            for (int a = 0; a < 3; ++a) u[((size_t)m * 3 + a) * n + node] = v[a];
        }
    }
}

/* Kinetic energy and enstrophy per sample in physical units:
 *   u_phys = u_lat U_c / U_lat,  E_m = (1/N^3) sum_x |u_phys|^2 / 2,
 *   Z_m = (1/N^3) sum_x |curl u_phys|^2 / 2, curl by second-order central
 *   differences with dx = 2 pi / N.  u: [M][3][n] lattice units. */
void SYM(energy)(int N, int M, const real_t *u, double ulat, double uc, real_t *E, real_t *Z)
{
    const double pi = 3.14159265358979323846;
    const size_t n = (size_t)N * N * N;
    const double scale = uc / ulat;
    const double dx = 2.0 * pi / N;
    for (int m = 0; m < M; ++m) {
        const real_t *ux = u + ((size_t)m * 3 + 0) * n;
        const real_t *uy = u + ((size_t)m * 3 + 1) * n;
        const real_t *uz = u + ((size_t)m * 3 + 2) * n;
        real_t e = 0, zz = 0;
        for (int z = 0; z < N; ++z)
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) {
                    size_t c = ((size_t)z * N + y) * N + x;
                    real_t vx = ux[c] * scale, vy = uy[c] * scale, vz = uz[c] * scale;
                    e += 0.5 * (vx * vx + vy * vy + vz * vz);
                    size_t xp = ((size_t)z * N + y) * N + (x + 1) % N, xm = ((size_t)z * N + y) * N + (x + N - 1) % N;
                    size_t yp = ((size_t)z * N + (y + 1) % N) * N + x, ym = ((size_t)z * N + (y + N - 1) % N) * N + x;
                    size_t zp = ((size_t)((z + 1) % N) * N + y) * N + x, zm = ((size_t)((z + N - 1) % N) * N + y) * N + x;
                    real_t dyuz = (uz[yp] - uz[ym]) * scale / (2 * dx), dzuy = (uy[zp] - uy[zm]) * scale / (2 * dx);
                    real_t dzux = (ux[zp] - ux[zm]) * scale / (2 * dx), dxuz = (uz[xp] - uz[xm]) * scale / (2 * dx);
                    real_t dxuy = (uy[xp] - uy[xm]) * scale / (2 * dx), dyux = (ux[yp] - ux[ym]) * scale / (2 * dx);
                    real_t wx = dyuz - dzuy, wy = dzux - dxuz, wz = dxuy - dyux;
                    zz += 0.5 * (wx * wx + wy * wy + wz * wz);
                }
        E[m] = e / (double)n;
        if (Z) Z[m] = zz / (double)n;
    }
}

#ifndef ORC_COMPLEX
/* Global relative entropy, Eqs. (relEntropy1), (relEntropy2):
 * H_rel = eps^3 sum_x sum_i [f_i ln(f_i/w_i) - f_i + w_i], eps = 2 pi / N. */
double RSYM(hrel)(int N, int M, const double *f)
{
    build_lattice();
    const double pi = 3.14159265358979323846;
    const size_t n = (size_t)N * N * N;
    double eps = 2.0 * pi / N, acc = 0;
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < Q; ++i)
            for (size_t c = 0; c < n; ++c) {
                double v = f[((size_t)m * Q + i) * n + c];
                acc += v * log(v / W[i]) - v + W[i];
            }
    return acc * eps * eps * eps;
}
#endif
