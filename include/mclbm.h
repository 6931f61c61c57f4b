/*
 * mclbm.h - C ABI of the GB300 Monte Carlo KBC lattice Boltzmann library.
 *
 * The calls follow the paper's statement of the problem (Sec. "Discretization
 * and well-prepared initial data"): the statistical solution at time t is the
 * push-forward mu_t = (S(t) o I) # (U[-w, w]^24) of 24 uniform parameters per
 * sample through the equilibrium initialisation I (Eq. (initialPopulations))
 * and the KBC lattice Boltzmann solution operator S(t) (Eqs. (lbIteration),
 * (kbcCollision), (entropyControl)).  A context holds one ensemble of M
 * independent samples on an N^3 periodic lattice (D3Q19) at one viscosity.
 *
 * Conventions shared by every call:
 *  - Return value: MCLBM_OK (0) or a negative mclbm_status.  On error the
 *    thread-local message of mclbm_last_error() says what failed; no call ever
 *    aborts the process.
 *  - Device memory is allocated by the caller and borrowed: the library never
 *    calls cudaMalloc.  Sizes come from mclbm_required_bytes().  Buffers must be
 *    256-byte aligned and stay valid until mclbm_destroy().
 *  - Every device call is enqueued on the CUDA stream given at creation (NULL =
 *    legacy default stream).  Calls that return host data synchronise that
 *    stream before returning; the others return as soon as work is enqueued.
 *  - A context may be used by one host thread at a time; contexts on several
 *    devices may be used from one process.  A call on a context (or batch) runs on
 *    the context's device, the device current at mclbm_create: the call makes it
 *    current and restores the caller's current device before returning.
 *  - Arrays are C order.  A scalar field on the lattice is [z][y][x] (x fastest),
 *    node (x, y, z) at physical position 2 pi (x, y, z) / N.
 *  - Velocities returned by the library are physical: u_phys = u_lat U_c / U_lat.
 */
#ifndef MCLBM_H
#define MCLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MCLBM_API __attribute__((visibility("default")))
#else
#define MCLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCLBM_OK = 0,
    MCLBM_ERR_INVALID_ARG = -1, /* null pointer, out-of-range value               */
    MCLBM_ERR_UNSTABLE_TAU = -2, /* tau <= 1/2 (omega_nu outside (0, 2))         */
    MCLBM_ERR_OOM = -3,          /* a caller buffer is smaller than required      */
    MCLBM_ERR_CUDA = -4,         /* a CUDA runtime call failed                    */
    MCLBM_ERR_NONFINITE = -5,    /* a NaN/Inf was found in the state or a result  */
    MCLBM_ERR_TIMEOUT = -6,      /* a bounded device wait gave up                 */
    MCLBM_ERR_SHAPE = -7,        /* N not a power of two >= 8, N % Q != 0, M < 2  */
    MCLBM_ERR_IO = -8            /* checkpoint file could not be read or written  */
} mclbm_status;

/* Population storage (Assumption "Uniform low Mach regime" (i): f = w (1 + eps g)
 * motivates storing the small deviation h_i = f_i / w_i - 1). */
enum {
    MCLBM_FP64 = 0, /* raw f_i in FP64, FP64 arithmetic (the plain method)           */
    MCLBM_FP32 = 1, /* h_i in FP32, FP32 collision arithmetic                        */
    MCLBM_FP16 = 2  /* h_i in FP16 (round to nearest), FP32 collision arithmetic     */
};

/* Streaming pattern. */
enum {
    MCLBM_PULL = 0, /* two lattices, gather f_i(x - c_i): pop bytes = 2 Q b N^3 M    */
    MCLBM_AA = 1    /* one lattice updated in place, alternating even/odd access    */
};

/* Ensemble configuration; copied at mclbm_create, caller keeps ownership. */
typedef struct {
    int32_t N;            /* nodes per direction, power of two, 8 <= N <= 1024        */
    int32_t M;            /* samples, >= 1                                            */
    int32_t precision;    /* MCLBM_FP64 / MCLBM_FP32 / MCLBM_FP16                     */
    int32_t pattern;      /* MCLBM_PULL / MCLBM_AA                                    */
    double nu;            /* physical kinematic viscosity eps = U_c l_c / Re (l_c = 1) */
    double Ma;            /* Mach number: U_lat = Ma c_s.  Ignored when dt > 0         */
    double dt;            /* physical time step; 0 -> dt = U_lat dx / U_c             */
    double U_c;           /* reference velocity (1)                                   */
    double width;         /* support w of the uniform parameters (0.025)              */
    uint64_t seed;        /* key of the Philox4x64-10 parameter draw                  */
    int32_t init_density; /* 0: rho_0 = 1 (the paper); 1: TGV pressure density       */
    int32_t options;      /* bit flags MCLBM_OPT_*; 0 = the paper's computations      */
} mclbm_config;

/* Option bits of mclbm_config.options.
 * MCLBM_OPT_LERAY: initialise with the Leray-projected perturbation, u_0 = u_det + P s
 * (Sec. "Discretization and well-prepared initial data"; the paper's runs omit P).  The
 * parameters stay the 24 coefficients X of s; the gradient of mclbm_grad is with respect to
 * them (the projection's transpose is applied). */
#define MCLBM_OPT_LERAY 1
/* MCLBM_OPT_EXACT_GAMMA: gamma is the exact minimiser of Eq. (kbc_entropy) over
 * 0 <= gamma <= 4 / omega, the root of sum Dh ln(f* / w) = 0 (or the nearer end of that range)
 * by a safeguarded Newton (FP32) or Halley (FP64) iteration from the closed form (Eq.
 * (entropyControl)), in FP64 (FP64 storage) or FP32; the stepper then runs launch kind 6 (the
 * direct kernel).  mclbm_grad rejects contexts with this option. */
#define MCLBM_OPT_EXACT_GAMMA 2

/* Derived diffusive-scaling units (Table "frequencySummary", Tables "params1/2"). */
typedef struct {
    double dx;       /* 2 pi / N                                 */
    double U_lat;    /* lattice velocity scale, Ma c_s            */
    double dt;       /* U_lat dx / U_c                            */
    double nu_lat;   /* nu dt / dx^2                              */
    double tau;      /* 3 nu_lat + 1/2                            */
    double omega;    /* omega_nu = 2 c_s^2 / (2 nu_lat + c_s^2)   */
} mclbm_units;

typedef struct mclbm_ctx mclbm_ctx; /* opaque, library-owned */

/* Library version string (static storage). */
MCLBM_API const char* mclbm_version(void);

/* Thread-local message of the last failed call on this thread (library-owned,
 * valid until the next call on the same thread). */
MCLBM_API const char* mclbm_last_error(void);

/* D3Q19 velocity set in the library's storage order: c [19][3] and w [19]
 * (either may be NULL).  Host pointers. */
MCLBM_API int mclbm_lattice(int32_t* c, double* w);

/* Units of a configuration without creating a context (Sec. "Numerical validation
 * of convergence rates": eps = 2 pi / N, Re_N coupling; Table "frequencySummary").
 * Errors: INVALID_ARG, UNSTABLE_TAU. */
MCLBM_API int mclbm_compute_units(const mclbm_config* cfg, mclbm_units* out);

/* Bytes of caller-allocated device memory a configuration needs:
 * pop_bytes for the population lattice(s), work_bytes for reductions and
 * statistics (the velocity fields and power spectra of two samples at a time, the FFT
 * buffer, partial sums).
 * Errors: INVALID_ARG, SHAPE, UNSTABLE_TAU. */
MCLBM_API int mclbm_required_bytes(const mclbm_config* cfg, size_t* pop_bytes, size_t* work_bytes);

/* Create a context over caller-owned device buffers d_pop (>= pop_bytes) and
 * d_work (>= work_bytes), enqueuing on cuda_stream (a cudaStream_t, may be NULL).
 * The device current at this call is the context's device.  No kernel runs yet.
 * Errors: INVALID_ARG, SHAPE, UNSTABLE_TAU, OOM (buffers too small), CUDA. */
MCLBM_API int mclbm_create(const mclbm_config* cfg, void* d_pop, size_t pop_bytes, void* d_work, size_t work_bytes,
                 void* cuda_stream, mclbm_ctx** out);

/* Release the context (not the caller's buffers).  NULL is ignored. */
MCLBM_API void mclbm_destroy(mclbm_ctx* ctx);

/* Units of an existing context. */
MCLBM_API int mclbm_get_units(const mclbm_ctx* ctx, mclbm_units* out);

/* Ensemble initialisation I (Eqs. (tgv_init_velo), (alpha_perturbation),
 * (initialRTGV), (initialPopulations)): per sample m the 24 parameters
 * X[m][8 alpha + 4 i + 2 j + k] give u_0 = (U_lat / U_c)(u_det + s(X_m)) at every
 * node and f_0 = f^eq(rho_0, u_0).  params: host [M][24] or NULL; NULL draws
 * X ~ U[-w, w] from Philox4x64-10 keyed by (seed, 0), counters (b, m, 0, 0),
 * b = 0..5, U = (x >> 11) 2^-53, X = w (2U - 1).  Resets the step counter.
 * Errors: INVALID_ARG, CUDA. */
MCLBM_API int mclbm_init_ensemble(mclbm_ctx* ctx, const double* params);

/* The parameter draw on its own (host only, no GPU needed): samples
 * first_sample .. first_sample + M - 1 of the Philox4x64-10 stream described
 * above, out [M][24].  Errors: INVALID_ARG. */
MCLBM_API int mclbm_draw_params(uint64_t seed, int32_t first_sample, int32_t M, double width, double* out);

/* The deterministic Taylor-Green initial state (all 24 parameters zero). */
MCLBM_API int mclbm_init_tgv(mclbm_ctx* ctx);

/* Copy the ensemble's parameters to host params [M][24]. */
MCLBM_API int mclbm_get_params(const mclbm_ctx* ctx, double* params);

/* Advance every sample by nsteps fused stream+collide steps (Eq. (lbIteration)
 * with the KBC collision Eq. (kbcCollision) and the closed-form stabiliser
 * Eq. (entropyControl)).  Enqueued only.  Errors: INVALID_ARG, CUDA. */
MCLBM_API int mclbm_step(mclbm_ctx* ctx, int64_t nsteps);

/* Number of steps taken since the last initialisation. */
MCLBM_API int64_t mclbm_steps_taken(const mclbm_ctx* ctx);

/* Pre-collision populations f_i(x, t) of one sample as FP64 (not shifted), in the
 * library's velocity order: d_out device [19][N][N][N].  Enqueued only. */
MCLBM_API int mclbm_get_populations(const mclbm_ctx* ctx, int32_t sample, double* d_out);

/* Overwrite the pre-collision populations of one sample from device FP64
 * d_in [19][N][N][N] (rounded to the storage precision).  Enqueued only. */
MCLBM_API int mclbm_set_populations(mclbm_ctx* ctx, int32_t sample, const double* d_in);

/* Macroscopic moments at the current integer step, pre-collision (Definition of the
 * moments: rho = sum f, rho u = sum c f): d_rho [N^3] (may be NULL) and d_u [3][N^3]
 * physical velocity, FP64 device buffers, for one sample, formed in the arithmetic of the
 * stepper (FP64 for FP64 storage, FP32 from the stored deviations for FP32/FP16 storage), as
 * are the fields behind the spectra, structure functions and mean/variance.  Enqueued only. */
MCLBM_API int mclbm_moments(const mclbm_ctx* ctx, int32_t sample, double* d_rho, double* d_u);

/* Kinetic energy E_m = N^-3 sum |u|^2 / 2 and (if Z != NULL) enstrophy
 * Z_m = N^-3 sum |curl u|^2 / 2 (second-order central differences, dx = 2 pi / N)
 * of every sample, physical units, FP64 host arrays [M].  Synchronises.
 * Reductions are in a fixed order (run-to-run bitwise reproducible). */
MCLBM_API int mclbm_energy(mclbm_ctx* ctx, double* E, double* Z);

/* Ensemble mean and unbiased (M - 1) variance of the physical velocity at every
 * node (Eqs. (spectrum_mean), (spectrum_var) applied pointwise): d_mean, d_var
 * device FP64 [3][N^3], from one pass over the samples that accumulates, per node, the sums
 * of u_m - u_0 and of its square in FP64 (u_m formed as the stepper's moments; with FP32 or FP16
 * storage, whose velocity carries FP32 rounding at best, these sums are formed in FP32 over
 * chunks of 8 samples and the chunks accumulated in FP64).  Errors: SHAPE if M < 2.
 * Enqueued only. */
MCLBM_API int mclbm_mean_var(mclbm_ctx* ctx, double* d_mean, double* d_var);

/* mclbm_energy and mclbm_mean_var in one pass over the populations (each population is read
 * once for both): E [M] host FP64 (the kinetic energy of every sample, as mclbm_energy, the
 * sums taken in another fixed order; with FP32 or FP16 storage each warp's sum of |u|^2 is
 * formed in FP32 before its FP64 accumulation, within about 1e-6 relative of mclbm_energy),
 * d_mean / d_var as mclbm_mean_var.  Synchronises.  Errors: INVALID_ARG, SHAPE (M < 2). */
MCLBM_API int mclbm_energy_mean_var(mclbm_ctx* ctx, double* E, double* d_mean, double* d_var);

/* Shell energy spectrum (Eqs. (dftCoeff), (energySpecDisc)) of every sample:
 * E [M][N/2 + 1] host FP64, kappa = 0..N/2.  Synchronises. */
MCLBM_API int mclbm_spectrum(mclbm_ctx* ctx, double* E);

/* Trace second-order structure function of Algorithm "SF_spectral" (Lemma
 * "Spectral approximation of structure functions") of every sample:
 * S2 [M][N/2 + 1] host FP64, r = 0..N/2 (grid units).  Synchronises. */
MCLBM_API int mclbm_sf_trace(mclbm_ctx* ctx, double* S2);

/* Longitudinal structure functions along the lattice axes (Eq. (structuresLocal)
 * with n in {e_x, e_y, e_z}, modulus as in Eq. (structures)):
 * S [M][pmax - 1][N/2] host FP64, p = 2..pmax (2 <= pmax <= 8), r = 1..N/2.  FP64 contexts
 * (and pmax > 6) form the differences and powers in FP64; FP32 and FP16 storage contexts, whose
 * velocity carries FP32 precision at most, form them in FP32, sum each line (32-point chunks,
 * then the chunks) in FP32 and accumulate the line sums in FP64.  Synchronises. */
MCLBM_API int mclbm_sf_axes(mclbm_ctx* ctx, int32_t pmax, double* S);

/* Exact restriction of the physical velocity to the common Q^3 grid (node n = j N / Q,
 * Appendix "Computation of the Wasserstein distance"): d_out device FP64
 * [M][Q^3][3], point index (jz Q + jy) Q + jx.  Errors: SHAPE if N % Q != 0. */
MCLBM_API int mclbm_restrict(const mclbm_ctx* ctx, int32_t Q, double* d_out);

/* W_{1,1} of Algorithm "WassersteinDistance1" between the one-point laws of two
 * ensembles A and B (they may differ in N and M): restrict both to Q^3 points, for
 * every point and component the 1-D W1 of the two empirical laws (L1 distance of the
 * empirical CDFs, Eq. (wassersteinPermutations) for equal M), summed over components
 * and averaged over points.  W: host scalar.  per_point: host [Q^3][3] or NULL.
 * A and B are on one device.  Uses A's work buffer and stream; synchronises.
 * Errors: SHAPE; INVALID_ARG for contexts on different devices. */
MCLBM_API int mclbm_w1_1pt(mclbm_ctx* A, const mclbm_ctx* B, int32_t Q, double* W, double* per_point);

/* Same on restricted fields already on the device: d_a [MA][G][3], d_b [MB][G][3]
 * FP64; uses d_work (>= mclbm_w1_work_bytes(MA, MB, G)) on cuda_stream. */
MCLBM_API size_t mclbm_w1_work_bytes(int32_t MA, int32_t MB, int32_t G);
MCLBM_API int mclbm_w1_restricted(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G, void* d_work,
                        size_t work_bytes, void* cuda_stream, double* W, double* per_point);

/* Two-point W1 between the laws of two ensembles on restricted fields (d_a [MA][G][3],
 * d_b [MB][G][3] FP64 device, e.g. from mclbm_restrict).  vector = 1: W_{1,2}^v of
 * Eq. (W1_vector) / Algorithm "WassersteinDistance2_vector", the W1 of the joint laws of
 * (u(x_i), u(x_j)) in R^6; vector = 0: W_{1,2} of Algorithm "WassersteinDistance2", the W1
 * of (u_c(x_i), u_c(x_j)) in R^2 for each component c, summed over c.  Euclidean ground
 * metric, every point pair i <= j, off-diagonal pairs counted twice, divided by G^2.  Each
 * pair is an exact transport problem between uniform empirical measures (1 <= MA, MB <= 1024):
 * for L = lcm(MA, MB) <= 64 an assignment of L atoms per side (atoms repeated L/MA, L/MB
 * times), one warp per problem; otherwise the transportation problem with integer supply MB/g
 * per atom of A and demand MA/g per atom of B (g = gcd(MA, MB)) by successive shortest paths,
 * one block per problem.  Costs are fixed-point integers from FP32 atoms taken relative to
 * their mean; the plan is optimal for those costs and its cost is summed in FP64 (each pair's
 * value is within about 1e-7 of the spread of its atoms of the exact optimum).  W: host
 * scalar.  d_per_pair: device FP64 [G (G + 1) / 2][vector ? 1 : 3] in row-major upper-triangle
 * order (pair (i, j) at i G - i (i - 1) / 2 + j - i), or NULL.  d_work: >=
 * mclbm_w1_2pt_work_bytes(MA, MB, G, vector) bytes, 256-byte aligned (it includes, for unequal
 * MA and MB with lcm > 64, one 2 MA MB-byte flow matrix for each of 256 problems in flight).
 * Runs on cuda_stream and synchronises it.  Errors: INVALID_ARG, SHAPE (MA or MB > 1024),
 * OOM (work buffer too small), NONFINITE (a search failed, e.g. on non-finite atoms). */
MCLBM_API size_t mclbm_w1_2pt_work_bytes(int32_t MA, int32_t MB, int32_t G, int32_t vector);
MCLBM_API int mclbm_w1_2pt(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G, int32_t vector,
                           void* d_work, size_t work_bytes, void* cuda_stream, double* W, double* d_per_pair);

/* Sample convergence check, Eq. (sample_error): the ensemble-averaged relative L1 error
 * (1/M) sum_m sum_k |u_m(x_k) - ref_m(x_k)| / sum_k |ref_m(x_k)| between paired samples (the
 * same parameters at two resolutions) on the G restriction points.  d_u, d_ref: device FP64
 * [M][G][3] (e.g. from mclbm_restrict).  out: host [4], the x, y, z components (absolute
 * value) and the velocity vector (Euclidean norm).  d_work: >= mclbm_sample_error_work_bytes(M)
 * bytes.  Runs on cuda_stream and synchronises it.  FP64, fixed reduction order.  Errors:
 * INVALID_ARG, OOM (work buffer too small). */
MCLBM_API size_t mclbm_sample_error_work_bytes(int32_t M);
MCLBM_API int mclbm_sample_error(const double* d_u, const double* d_ref, int32_t M, int32_t G, void* d_work,
                                 size_t work_bytes, void* cuda_stream, double* out);

/* Coefficients of the Leray-projected perturbation: P s of Eq. (alpha_perturbation) is again
 * of that form (every term has wavenumbers (+-2, +-2, +-2), |k|^2 = 12, so
 * P s = s + grad(div s) / 12), with coefficients Y = L X.  X, Y: host [M][24] (index
 * 8 alpha + 4 i + 2 j + k as for the parameters).  transpose = 1 applies L^T instead.  Host
 * only; no device work.  Errors: INVALID_ARG.  The paper has no separate counterpart: this is
 * the map that MCLBM_OPT_LERAY applies at initialisation. */
MCLBM_API int mclbm_leray_params(const double* X, int32_t M, int32_t transpose, double* Y);

/* ---- launch shape and autotuning ------------------------------------------
 * kind 0: the direct stepper kernel updates `vec` consecutive nodes along x per
 * thread (vec-wide loads and stores, warp shuffles for the x-shifts) in blocks of
 * `block` threads on a persistent grid; vec in {1, 2} (FP64), {1, 2, 4} (FP32),
 * {2, 4, 8} (FP16), dividing N; block in {128, 256}.
 * kind 1: the staged kernel (one producer warp stages each tile's source rows in
 * shared memory with bulk asynchronous copies; eight consumer warps collide `vec`
 * in {1, 2} nodes per thread); `block` is ignored.
 * kind 2: the direct kernel with the next run's loads issued before the current
 * run's arithmetic (same vec and block values as kind 0).
 * kind 3: kind 2 with the FP32 collision of two nodes at a time in the packed FP32
 * instructions of sm_100 and later (FP32 and FP16 storage, even vec).
 * kinds 4 and 5: kind 3 with the runs ahead copied by cp.async into a shared-memory ring, one
 * or two runs deep (FP32 and FP16 storage, block 128).
 * kind 6: the direct kernel with the exact entropic gamma (contexts with
 * MCLBM_OPT_EXACT_GAMMA, and only they; vec = the first of the type's list, block 128).
 * Results do not depend on the shape (same arithmetic per node, every operation
 * rounded once in the same order).  mclbm_set_launch sets the shape of every step (under AA
 * streaming, of both parities); mclbm_get_launch reports the shape of pull steps and AA even
 * steps.  Errors: INVALID_ARG (unsupported shape, vec not dividing N, kind 6 on a context
 * without MCLBM_OPT_EXACT_GAMMA or another kind on one with it). */
MCLBM_API int mclbm_set_launch(mclbm_ctx* ctx, int32_t kind, int32_t vec, int32_t block);
MCLBM_API int mclbm_get_launch(const mclbm_ctx* ctx, int32_t* kind, int32_t* vec, int32_t* block);

/* Shape of one parity of an AA context: parity 0 the even steps (own node, no shifts),
 * parity 1 the odd steps (shifted loads and shifted stores, which favour other shapes).
 * Each AA step already runs as one launch per parity, so the two shapes never share a
 * launch.  Kind 1 (staged) serves both parities: setting it for one sets it for both, and
 * setting another kind for one parity while the other is staged replaces both.  The
 * defaults are measured per parity.  Pull contexts: parity 0 only.  Errors: INVALID_ARG as
 * for mclbm_set_launch, parity not 0 or 1, parity 1 on a pull context. */
MCLBM_API int mclbm_set_launch_parity(mclbm_ctx* ctx, int32_t parity, int32_t kind, int32_t vec, int32_t block);
MCLBM_API int mclbm_get_launch_parity(const mclbm_ctx* ctx, int32_t parity, int32_t* kind, int32_t* vec,
                                      int32_t* block);

/* Time every supported shape on this context for trial_steps steps each (CUDA events
 * on the context's stream; AA: trial_steps steps of each parity, timed per parity), keep the
 * fastest (AA: the fastest of each parity, or the staged kind for both where it is faster
 * over a pair of steps), and restore the initial state by re-running the initialisation from
 * the stored parameters.  Must directly follow mclbm_init_ensemble / mclbm_init_tgv
 * (INVALID_ARG otherwise).  Outputs may be NULL; kind, vec and block report the shape of
 * parity 0 (mclbm_get_launch_parity gives the other); best_ms is the time per step.
 * Synchronises. */
MCLBM_API int mclbm_autotune(mclbm_ctx* ctx, int32_t trial_steps, int32_t* kind, int32_t* vec, int32_t* block,
                             double* best_ms);

/* ---- batched levels of the viscosity sequence --------------------------------
 * Levels (contexts sharing device, stream, precision and pattern) advanced
 * together under diffusive scaling (Remark "Diffusive scaling": dt ~ dx^2): level l
 * takes substeps[l] steps per macro step; every substeps[l] divides the largest, S.
 * Sub-step s of a macro step advances each level with s % (S / substeps[l]) == 0, all
 * in one persistent launch.  With graphs enabled (default when the stream is not the
 * legacy default stream) one period of the schedule is captured into a CUDA graph
 * on first use and replayed.  The batch borrows the contexts; destroy it first. */
typedef struct mclbm_batch mclbm_batch;
MCLBM_API int mclbm_batch_create(mclbm_ctx* const* levels, int32_t nlev, const int32_t* substeps, mclbm_batch** out);
MCLBM_API void mclbm_batch_destroy(mclbm_batch* b);
MCLBM_API int mclbm_batch_set_graph(mclbm_batch* b, int32_t enable);
/* The batch's launch shape (initially that of levels[0]; an AA odd-step shape still at its
 * default becomes the default for the batch's largest level): mclbm_batch_set_launch for every
 * step, the _parity forms per parity of AA batches, with the rules of
 * mclbm_set_launch_parity; every level must accept the shape. */
MCLBM_API int mclbm_batch_set_launch(mclbm_batch* b, int32_t kind, int32_t vec, int32_t block);
MCLBM_API int mclbm_batch_set_launch_parity(mclbm_batch* b, int32_t parity, int32_t kind, int32_t vec, int32_t block);
MCLBM_API int mclbm_batch_get_launch_parity(const mclbm_batch* b, int32_t parity, int32_t* kind, int32_t* vec,
                                            int32_t* block);
/* Enqueue macro_steps macro steps.  Enqueued only. */
MCLBM_API int mclbm_batch_step(mclbm_batch* b, int64_t macro_steps);
MCLBM_API int64_t mclbm_batch_macro_steps(const mclbm_batch* b);
/* Autotune the batch's launch shape (one macro step per trial, trials trials per
 * shape): one shape for both parities first, then for AA batches the odd steps' shape with
 * that even shape (unless the staged kind won); then re-initialise every level.  Must
 * directly follow initialisation.  kind, vec and block report parity 0. */
MCLBM_API int mclbm_batch_autotune(mclbm_batch* b, int32_t trials, int32_t* kind, int32_t* vec, int32_t* block,
                                   double* best_ms);

/* ---- adjoint (gradients w.r.t. the 24 parameters) ------------------------------
 * Discrete adjoint of the time stepping: for J_m = E_m(T) (objective 0, kinetic
 * energy) or Z_m(T) (objective 1, enstrophy) of every sample m after nsteps steps,
 * dJ_m/dX_m [M][24] with X_m the sample's parameters (Eq. (alpha_perturbation)).
 * The reverse sweep applies the transpose of streaming and the hand-written
 * transpose of the KBC collision Jacobian, including the derivative of the closed-form
 * gamma of Eq. (entropyControl); states are checkpointed every ckpt_every steps and
 * each segment is recomputed from its checkpoint.  Pull streaming only.  The context
 * must directly follow an initialisation; on return it holds the state at step nsteps.
 * d_buf: caller device buffer of mclbm_grad_required_bytes() bytes (256-aligned).
 * J [M], dJdX [M][24]: host.  Synchronises.  Errors: INVALID_ARG, OOM, CUDA. */
MCLBM_API int mclbm_grad_required_bytes(const mclbm_ctx* ctx, int64_t nsteps, int32_t ckpt_every, size_t* bytes);
MCLBM_API int mclbm_grad(mclbm_ctx* ctx, int32_t objective, int64_t nsteps, int32_t ckpt_every, void* d_buf,
                         size_t buf_bytes, double* J, double* dJdX);

/* Device time (CUDA events on the context's stream) of the phases of the last
 * mclbm_grad on this context, ms[4]: forward with checkpoints, recomputation of the
 * segments, reverse sweep (adjoint kernels), parameter reduction.  Host array. */
MCLBM_API int mclbm_grad_timing(const mclbm_ctx* ctx, double* ms);

/* One transposed step on caller data, for checking the adjoint: given pre-collision
 * populations f^t (raw, FP64) and lambda^{t+1} = dJ/df^{t+1}, writes
 * lambda^t = dJ/df^t (all FP64 device [M][19][N][N][N], library velocity order),
 * computed in the context's arithmetic (FP64 or FP32).  Enqueued only. */
MCLBM_API int mclbm_adjoint_step(const mclbm_ctx* ctx, const double* d_f, const double* d_lambda_next, double* d_lambda);

/* Synchronise the context's stream and report a bounded device wait that gave up
 * since the last initialisation (MCLBM_ERR_TIMEOUT; the staged stepper's producer and
 * consumer waits are bounded and set this instead of hanging). */
MCLBM_API int mclbm_device_status(mclbm_ctx* ctx);

/* W_{1,1} on restricted fields like mclbm_w1_restricted, for callers that cannot
 * allocate device memory: code embedded where another allocator owns the GPU's memory
 * (a framework's caching pool or a fixed arena, whose accounting a cudaMalloc would
 * bypass), code that must not trigger the device-wide synchronisation of cudaFree, and
 * code running with no device memory to spare.  This call allocates nothing: its
 * scratch is a fixed array in the library's device image, holding at most 4096 points
 * (G <= 4096; larger G returns MCLBM_ERR_SHAPE), about 96 KiB that every GPU loading the
 * library keeps until the process exits.  The first call on a device looks up that
 * array's address (cudaGetSymbolAddress, with the device current), so make it before
 * any stream capture.  Calls share the array: nothing carries over from one call to the
 * next, but calls that overlap on the GPU race.  Same inputs, outputs and errors as
 * mclbm_w1_restricted otherwise; synchronises cuda_stream.  The paper has no
 * counterpart of this entry point. */
MCLBM_API int mclbm_w1_restricted_noalloc(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G,
                                          void* cuda_stream, double* W, double* per_point);

/* Arithmetic throughput of the current device, for setting kernels that are bound by
 * arithmetic rather than memory against a measured ceiling (the paper has no counterpart:
 * this is measurement support).  kind 0: FP64 fma; 1: FP32 fma; 2: packed FP32x2 fma (two
 * results per instruction); 3: packed half2 fma; 4: FP32 reciprocal approximation
 * (rcp.approx, the special-function unit).  One launch of 8 blocks of 256 threads per SM,
 * each thread running 8 independent chains of 16 * iters operations, timed with CUDA events
 * after one untimed launch on cuda_stream.  results_per_s: host, results (lane operations)
 * per second (an fma result is two floating-point operations); ms: host or NULL, the timed
 * launch.  d_sink: device, at least 8 bytes, written only if a chain reaches an impossible
 * value.  Synchronises.  Errors: INVALID_ARG, CUDA. */
MCLBM_API int mclbm_alu_rate(int32_t kind, int32_t iters, double* d_sink, void* cuda_stream, double* results_per_s,
                             double* ms);

/* Failure-path self-test: runs one bounded wait on a barrier that nothing completes, so
 * the wait runs out and records MCLBM_ERR_TIMEOUT exactly as a stepper wait would; the
 * next mclbm_device_status reports it and the next initialisation clears it.  No GPU
 * fault, trap or hang is involved.  Enqueued only. */
MCLBM_API int mclbm_selftest_timeout(mclbm_ctx* ctx);

/* Checkpoint of the current state to a host file (written after synchronising the stream):
 * a magic word, the format version (2), the velocity count Q of the library, the
 * configuration and its derived units, the step count, the parameters and the stored
 * populations, and nothing after them.  mclbm_load restores it only into a context of the
 * same lattice (Q), N, M, precision, pattern, options, viscosity, U_c and derived time step,
 * U_lat and omega (anything else would resume the state under other dynamics).
 * Errors: IO (cannot open, truncated, another format version, bytes after the lattice, not
 * a checkpoint), SHAPE (another lattice or configuration), CUDA. */
MCLBM_API int mclbm_save(const mclbm_ctx* ctx, const char* path);
MCLBM_API int mclbm_load(mclbm_ctx* ctx, const char* path);

/* Scan every stored population for NaN/Inf.  Returns MCLBM_OK or
 * MCLBM_ERR_NONFINITE.  Synchronises. */
MCLBM_API int mclbm_check_finite(mclbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MCLBM_H */
