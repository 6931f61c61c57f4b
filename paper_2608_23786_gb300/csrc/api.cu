// C ABI of libmclbm: argument checking, units, the Philox parameter draw,
// work-buffer layout and context bookkeeping.  Device work is delegated to the
// kernels of stepper.cu, fields.cu, spectral.cu, sfaxes.cu and w1.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"
#include "lattice.cuh"

namespace mclbm {

cudaError_t launch_twiddles(const mclbm_ctx* c);
size_t sf_axes_partial_bytes(int N);

namespace {
thread_local std::string g_last_error;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

size_t elem_bytes_of(int precision) { return precision == MCLBM_FP64 ? 8 : (precision == MCLBM_FP32 ? 4 : 2); }

// ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (hi, lo) = M0 * X0, (hi', lo') = M1 * X2, X <- (hi' ^ X1 ^ K0, lo', hi ^ X3 ^ K1, lo),
// with the key bumped by the Weyl constants between rounds.
void philox4x64_10(uint64_t ctr[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t X[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint64_t K0 = key_in[0], K1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        const unsigned __int128 p0 = (unsigned __int128)M0 * X[0];
        const unsigned __int128 p1 = (unsigned __int128)M1 * X[2];
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        const uint64_t n0 = hi1 ^ X[1] ^ K0, n1 = lo1, n2 = hi0 ^ X[3] ^ K1, n3 = lo0;
        X[0] = n0;
        X[1] = n1;
        X[2] = n2;
        X[3] = n3;
        K0 += W0;
        K1 += W1;
    }
    for (int k = 0; k < 4; ++k) out[k] = X[k];
}

void draw_params(uint64_t seed, int first, int M, double w, double* out)
{
    const uint64_t key[2] = {seed, 0};
    for (int m = 0; m < M; ++m)
        for (int b = 0; b < 6; ++b) {
            uint64_t ctr[4] = {(uint64_t)b, (uint64_t)(first + m), 0, 0}, r[4];
            philox4x64_10(ctr, key, r);
            for (int k = 0; k < 4; ++k) {
                const double U = (double)(r[k] >> 11) * 0x1.0p-53;
                out[24 * m + 4 * b + k] = w * (2.0 * U - 1.0);
            }
        }
}

int validate(const mclbm_config* cfg, mclbm_units* u)
{
    if (!cfg) return set_error(MCLBM_ERR_INVALID_ARG, "config is NULL");
    if (!is_pow2(cfg->N) || cfg->N < 8 || cfg->N > 1024)
        return set_error(MCLBM_ERR_SHAPE, "N must be a power of two in [8, 1024], got " + std::to_string(cfg->N));
    if (cfg->M < 1) return set_error(MCLBM_ERR_INVALID_ARG, "M must be >= 1");
    if (cfg->precision < 0 || cfg->precision > 2) return set_error(MCLBM_ERR_INVALID_ARG, "precision must be 0, 1 or 2");
    if (cfg->pattern < 0 || cfg->pattern > 1) return set_error(MCLBM_ERR_INVALID_ARG, "pattern must be 0 (pull) or 1 (AA)");
    if (!(cfg->U_c > 0) || !std::isfinite(cfg->U_c)) return set_error(MCLBM_ERR_INVALID_ARG, "U_c must be > 0");
    if (!(cfg->width >= 0) || !std::isfinite(cfg->width)) return set_error(MCLBM_ERR_INVALID_ARG, "width must be >= 0");
    if (cfg->init_density != 0 && cfg->init_density != 1)
        return set_error(MCLBM_ERR_INVALID_ARG, "init_density must be 0 or 1");
    if ((cfg->options & ~(MCLBM_OPT_LERAY | MCLBM_OPT_EXACT_GAMMA)) != 0)
        return set_error(MCLBM_ERR_INVALID_ARG, "unknown option bits");
    if (!std::isfinite(cfg->nu)) return set_error(MCLBM_ERR_INVALID_ARG, "nu must be finite");
    const double pi = 3.14159265358979323846;
    mclbm_units r;
    r.dx = 2.0 * pi / cfg->N;
    if (cfg->dt > 0) {
        r.dt = cfg->dt;
        r.U_lat = cfg->dt * cfg->U_c / r.dx;
    } else {
        if (!(cfg->Ma > 0) || !std::isfinite(cfg->Ma)) return set_error(MCLBM_ERR_INVALID_ARG, "Ma must be > 0 when dt = 0");
        r.U_lat = cfg->Ma * std::sqrt(1.0 / 3.0);
        r.dt = r.U_lat * r.dx / cfg->U_c;
    }
    r.nu_lat = cfg->nu * r.dt / (r.dx * r.dx);
    r.omega = (2.0 / 3.0) / (2.0 * r.nu_lat + 1.0 / 3.0);
    r.tau = 1.0 / r.omega;
    if (!(r.nu_lat > 0) || !(r.omega > 0 && r.omega < 2) || !(r.tau > 0.5))
        return set_error(MCLBM_ERR_UNSTABLE_TAU, "relaxation time tau = " + std::to_string(r.tau) + " is not > 1/2");
    if (u) *u = r;
    return MCLBM_OK;
}

}  // namespace

// Leray projection on the 24 coefficients of the perturbation (Sec. "Discretization and
// well-prepared initial data").  s_a = (1/8) sum_{ijk} X_{a,ijk} B_{ijk} with
// B_{ijk} = A_i(2x) A_j(2y) A_k(2z), A_0 = sin, A_1 = cos, so the derivative along axis b of
// B_{ijk} is 2 sg(t) B_{ijk with t flipped}, t the index of axis b, sg(0) = 1, sg(1) = -1.
// Every term has |k|^2 = 12, hence P s = s + grad(div s) / 12 and, on the coefficients,
//   Y_{b,lmn} = X_{b,lmn} + (1/3) sum_a sg(I_a(ijk)) sg(I_b(flip_a ijk)) X_{a,ijk},
//   ijk = flip_a flip_b (lmn).
void leray_matrix(double L[24][24])
{
    for (int r = 0; r < 24; ++r)
        for (int q = 0; q < 24; ++q) L[r][q] = r == q ? 1.0 : 0.0;
    for (int b = 0; b < 3; ++b)
        for (int lmn = 0; lmn < 8; ++lmn)
            for (int a = 0; a < 3; ++a) {
                int idx[3] = {(lmn >> 2) & 1, (lmn >> 1) & 1, lmn & 1};
                idx[b] ^= 1;
                idx[a] ^= 1;  // ijk = flip_a flip_b (lmn)
                const int ta = idx[a];
                int f[3] = {idx[0], idx[1], idx[2]};
                f[a] ^= 1;  // flip_a (ijk)
                const int tb = f[b];
                const double sg = (ta == 0 ? 1.0 : -1.0) * (tb == 0 ? 1.0 : -1.0);
                L[8 * b + lmn][8 * a + 4 * idx[0] + 2 * idx[1] + idx[2]] += sg / 3.0;
            }
}

void leray_map(const double* X, int M, bool transpose, double* Y)
{
    double L[24][24];
    leray_matrix(L);
    for (int m = 0; m < M; ++m) {
        double y[24];
        for (int r = 0; r < 24; ++r) {
            double acc = 0.0;
            for (int q = 0; q < 24; ++q) acc += (transpose ? L[q][r] : L[r][q]) * X[24 * m + q];
            y[r] = acc;
        }
        for (int r = 0; r < 24; ++r) Y[24 * m + r] = y[r];
    }
}

// Default launch shape: the fastest measured on a GB300 for the 64^3 x 64 and 128^3 x 32
// ensembles (the autotuner may pick another), for pull steps and AA even steps.  D3Q19: FP32
// packed collision, 2 nodes per thread; FP16 shared-memory prefetch ring, 8 nodes per thread;
// FP64 (bound by the FP64 units) the direct kernel.
LaunchConfig default_launch(int precision, int pattern, int options)
{
    if (options & MCLBM_OPT_EXACT_GAMMA) return LaunchConfig{exact_vec(precision), 128, 6};
#ifdef MCLBM_D3Q27
    // D3Q27 (measured at 128^3 x 32): FP32 prefetching kernel in blocks of 256; FP16 pull and AA
    // even steps the shared-memory ring (pull 85% with the row rotation and the single-level
    // kernel, against 67% for the direct kernel; AA even 89.0% against 87.7% for the packed
    // prefetching kernel)
    if (precision == MCLBM_FP64) return LaunchConfig{1, 128, 0};
    if (precision == MCLBM_FP32) return LaunchConfig{2, 256, 2};
    return LaunchConfig{4, 128, 4};
#else
    if (precision == MCLBM_FP64) return LaunchConfig{2, 128, 0};
    if (precision == MCLBM_FP32) return LaunchConfig{2, 128, 3};
    return LaunchConfig{8, 128, 4};
#endif
}

// AA odd steps read and write shifted rows and favour other shapes (measured per parity at
// 128^3 x 32 and 64^3 x 64): D3Q19 FP32 the two-stage cp.async ring with 4 nodes per thread,
// FP16 the packed prefetching kernel with 4; D3Q27 FP32 and FP16 the packed prefetching kernel in
// blocks of 256 (D3Q27 FP16 with the row rotation at 128^3: 83.2% of the copy bandwidth, against
// 80.7% for the ring and 52% for the one-node prefetching kernel without the rotation).
// Nmax: the largest lattice the shape serves (a context's N, a batch's largest level): D3Q19 FP16
// odd steps with Nmax <= 256 take the two-stage ring with 8 nodes per thread, whose rows of up to
// 256 nodes lie within one warp and rotate (128^3 x 32: 81.4% of the copy bandwidth against 80.7%
// for the packed prefetching kernel with 4; the three-level batch 64^3 x 64 + 128^3 x 32 + 256^3 x 8:
// 84.2% per macro step against 77.7% with rows of 256 nodes spanning warps).
LaunchConfig default_launch_odd(int precision, int pattern, int options, int Nmax)
{
    const LaunchConfig even = default_launch(precision, pattern, options);
    if (pattern != MCLBM_AA || even.kind == 6 || precision == MCLBM_FP64) return even;
#ifdef MCLBM_D3Q27
    (void)Nmax;
    return precision == MCLBM_FP32 ? LaunchConfig{2, 256, 3} : LaunchConfig{4, 256, 3};
#else
    if (precision == MCLBM_FP32) return LaunchConfig{4, 128, 5};
    if (Nmax <= 32 * 8) return LaunchConfig{8, 128, 4};
    return LaunchConfig{4, 128, 3};
#endif
}

int set_error(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_check(cudaError_t e, const char* what)
{
    return set_error(MCLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

WorkLayout work_layout(int N, int M)
{
    const size_t n = (size_t)N * N * N;
    WorkLayout wl;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    wl.params = take((size_t)M * 24 * sizeof(double));
    size_t part = (size_t)M * 2 * 1024 * sizeof(double);
    wl.partial = take(part > kPartialBytes ? part : kPartialBytes);
    wl.flag = take(16 * sizeof(int));
    wl.field = take(4 * n * sizeof(double));
    wl.cplx = take(n * 2 * sizeof(double));
    const size_t sfb = sf_axes_partial_bytes(N);
    wl.real = take(n * sizeof(double) > sfb ? n * sizeof(double) : sfb);
    wl.real2 = take(n * sizeof(double));
    wl.twiddle = take((size_t)N * 2 * sizeof(double));
    wl.trig = take((size_t)N * 4 * (sizeof(double) + sizeof(float)));  // FP64 table, then its FP32 copy
    size_t per = 2 * (size_t)(N / 2 + 1);
    if ((size_t)7 * (N / 2) > per) per = (size_t)7 * (N / 2);
    wl.bins = take((size_t)M * per * sizeof(double) + 2 * (size_t)M * sizeof(double));
    wl.total = off;
    return wl;
}

void* lattice_ptr(const mclbm_ctx* c, int which)
{
    const size_t one = c->elem_bytes * Q * (size_t)c->n * c->M;
    return (char*)c->pop + (size_t)which * one;
}

}  // namespace mclbm

using namespace mclbm;

// W1 region appended after the main layout: restricted fields of A and of up to
// kMaxW1Samples samples of B on the Q = 8 grid, plus the W1 kernel's own scratch.
static size_t w1_region_bytes(int M)
{
    const size_t G = 512;
    return ((size_t)(M + kMaxW1Samples) * G * 3 * sizeof(double) + 255) / 256 * 256 + w1_work_bytes(M, kMaxW1Samples, 512) +
           256;
}

extern "C" {

const char* mclbm_version(void) { return "mclbm 0.2.0 (" MCLBM_LATTICE_NAME " KBC, sm_103a)"; }

const char* mclbm_last_error(void) { return g_last_error.c_str(); }

int mclbm_lattice(int32_t* c, double* w)
{
    for (int i = 0; i < Q; ++i) {
        if (c) {
            c[3 * i + 0] = cx(i);
            c[3 * i + 1] = cy(i);
            c[3 * i + 2] = cz(i);
        }
        if (w) w[i] = weight<double>(i);
    }
    return MCLBM_OK;
}

int mclbm_compute_units(const mclbm_config* cfg, mclbm_units* out)
{
    if (!out) return set_error(MCLBM_ERR_INVALID_ARG, "out is NULL");
    return validate(cfg, out);
}

int mclbm_required_bytes(const mclbm_config* cfg, size_t* pop_bytes, size_t* work_bytes)
{
    int st = validate(cfg, nullptr);
    if (st != MCLBM_OK) return st;
    const size_t n = (size_t)cfg->N * cfg->N * cfg->N;
    const size_t one = elem_bytes_of(cfg->precision) * Q * n * (size_t)cfg->M;
    if (pop_bytes) *pop_bytes = one * (cfg->pattern == MCLBM_PULL ? 2 : 1);
    if (work_bytes) *work_bytes = work_layout(cfg->N, cfg->M).total + w1_region_bytes(cfg->M);
    return MCLBM_OK;
}

int mclbm_create(const mclbm_config* cfg, void* d_pop, size_t pop_bytes, void* d_work, size_t work_bytes,
                 void* cuda_stream, mclbm_ctx** out)
{
    if (!out) return set_error(MCLBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mclbm_units u;
    int st = validate(cfg, &u);
    if (st != MCLBM_OK) return st;
    size_t need_pop = 0, need_work = 0;
    mclbm_required_bytes(cfg, &need_pop, &need_work);
    if (!d_pop || !d_work) return set_error(MCLBM_ERR_INVALID_ARG, "device buffers must not be NULL");
    if (((uintptr_t)d_pop & 255) || ((uintptr_t)d_work & 255))
        return set_error(MCLBM_ERR_INVALID_ARG, "device buffers must be 256-byte aligned");
    if (pop_bytes < need_pop)
        return set_error(MCLBM_ERR_OOM, "population buffer has " + std::to_string(pop_bytes) + " bytes, needs " +
                                            std::to_string(need_pop));
    if (work_bytes < need_work)
        return set_error(MCLBM_ERR_OOM,
                         "work buffer has " + std::to_string(work_bytes) + " bytes, needs " + std::to_string(need_work));
    int dev = 0;
    MCLBM_CUDA(cudaGetDevice(&dev));
    mclbm_ctx* c = new (std::nothrow) mclbm_ctx();
    if (!c) return set_error(MCLBM_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->units = u;
    c->N = cfg->N;
    c->logN = ilog2(cfg->N);
    c->M = cfg->M;
    c->n = (int64_t)cfg->N * cfg->N * cfg->N;
    c->pop = d_pop;
    c->pop_bytes = pop_bytes;
    c->work = (char*)d_work;
    c->work_bytes = work_bytes;
    c->wl = work_layout(cfg->N, cfg->M);
    c->stream = (cudaStream_t)cuda_stream;
    c->device = dev;
    c->cur = 0;
    c->steps = 0;
    c->params.assign((size_t)cfg->M * 24, 0.0);
    c->elem_bytes = elem_bytes_of(cfg->precision);
    c->twiddles_ready = false;
    c->launch = default_launch(cfg->precision, cfg->pattern, cfg->options);
    c->launch_odd = default_launch_odd(cfg->precision, cfg->pattern, cfg->options, cfg->N);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    c->num_sms = sms;
    *out = c;
    return MCLBM_OK;
}

void mclbm_destroy(mclbm_ctx* ctx) { delete ctx; }

int mclbm_get_units(const mclbm_ctx* ctx, mclbm_units* out)
{
    if (!ctx || !out) return set_error(MCLBM_ERR_INVALID_ARG, "NULL argument");
    *out = ctx->units;
    return MCLBM_OK;
}

static int do_init(mclbm_ctx* c)
{
    double* d_params = (double*)(c->work + c->wl.params);
    // the coefficients of the perturbation the initialisation evaluates: X, or L X with the
    // Leray projection
    c->init_coeffs = c->params;
    if (c->cfg.options & MCLBM_OPT_LERAY) leray_map(c->params.data(), c->M, false, c->init_coeffs.data());
    MCLBM_CUDA(cudaMemcpyAsync(d_params, c->init_coeffs.data(), sizeof(double) * 24 * c->M, cudaMemcpyHostToDevice,
                               c->stream));
    c->cur = 0;
    c->steps = 0;
    MCLBM_CUDA(cudaMemsetAsync(c->work + c->wl.flag, 0, 16 * sizeof(int), c->stream));
    MCLBM_CUDA(launch_init(c, d_params));
    return MCLBM_OK;
}

int mclbm_init_ensemble(mclbm_ctx* ctx, const double* params)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    MCLBM_ON_DEVICE(ctx->device);
    if (params) {
        for (size_t k = 0; k < ctx->params.size(); ++k) {
            if (!std::isfinite(params[k])) return set_error(MCLBM_ERR_INVALID_ARG, "params must be finite");
            ctx->params[k] = params[k];
        }
    } else {
        draw_params(ctx->cfg.seed, 0, ctx->M, ctx->cfg.width, ctx->params.data());
    }
    return do_init(ctx);
}

int mclbm_draw_params(uint64_t seed, int32_t first_sample, int32_t M, double width, double* out)
{
    if (!out || M < 0 || first_sample < 0 || !(width >= 0) || !std::isfinite(width))
        return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    draw_params(seed, first_sample, M, width, out);
    return MCLBM_OK;
}

int mclbm_init_tgv(mclbm_ctx* ctx)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    MCLBM_ON_DEVICE(ctx->device);
    std::fill(ctx->params.begin(), ctx->params.end(), 0.0);
    return do_init(ctx);
}

int mclbm_leray_params(const double* X, int32_t M, int32_t transpose, double* Y)
{
    if (!X || !Y || M < 1 || (transpose != 0 && transpose != 1)) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    leray_map(X, M, transpose == 1, Y);
    return MCLBM_OK;
}

int mclbm_get_params(const mclbm_ctx* ctx, double* params)
{
    if (!ctx || !params) return set_error(MCLBM_ERR_INVALID_ARG, "NULL argument");
    std::memcpy(params, ctx->params.data(), sizeof(double) * ctx->params.size());
    return MCLBM_OK;
}

int mclbm_step(mclbm_ctx* ctx, int64_t nsteps)
{
    if (!ctx || nsteps < 0) return set_error(MCLBM_ERR_INVALID_ARG, "bad ctx or nsteps < 0");
    MCLBM_ON_DEVICE(ctx->device);
    for (int64_t s = 0; s < nsteps; ++s) MCLBM_CUDA(launch_step(ctx));
    return MCLBM_OK;
}

int64_t mclbm_steps_taken(const mclbm_ctx* ctx) { return ctx ? ctx->steps : -1; }

int mclbm_get_populations(const mclbm_ctx* ctx, int32_t sample, double* d_out)
{
    if (!ctx || !d_out || sample < 0 || sample >= ctx->M) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    MCLBM_CUDA(launch_get_populations(ctx, sample, d_out));
    return MCLBM_OK;
}

int mclbm_set_populations(mclbm_ctx* ctx, int32_t sample, const double* d_in)
{
    if (!ctx || !d_in || sample < 0 || sample >= ctx->M) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    MCLBM_CUDA(launch_set_populations(ctx, sample, d_in));
    return MCLBM_OK;
}

int mclbm_moments(const mclbm_ctx* ctx, int32_t sample, double* d_rho, double* d_u)
{
    if (!ctx || !d_u || sample < 0 || sample >= ctx->M) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    MCLBM_CUDA(launch_moments(ctx, sample, d_rho, d_u));
    return MCLBM_OK;
}

int mclbm_energy(mclbm_ctx* ctx, double* E, double* Z)
{
    if (!ctx || !E) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    MCLBM_CUDA(launch_energy(ctx, Z != nullptr, E, Z));
    return MCLBM_OK;
}

int mclbm_mean_var(mclbm_ctx* ctx, double* d_mean, double* d_var)
{
    if (!ctx || !d_mean || !d_var) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    if (ctx->M < 2) return set_error(MCLBM_ERR_SHAPE, "variance needs M >= 2");
    MCLBM_CUDA(launch_mean_var(ctx, d_mean, d_var));
    return MCLBM_OK;
}

int mclbm_energy_mean_var(mclbm_ctx* ctx, double* E, double* d_mean, double* d_var)
{
    if (!ctx || !E || !d_mean || !d_var) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    if (ctx->M < 2) return set_error(MCLBM_ERR_SHAPE, "variance needs M >= 2");
    if (ctx->M > 1024) {  // the one-pass kernel reduces up to 1024 energies in shared memory
        MCLBM_CUDA(launch_mean_var(ctx, d_mean, d_var));
        MCLBM_CUDA(launch_energy(ctx, false, E, nullptr));
        return MCLBM_OK;
    }
    MCLBM_CUDA(launch_energy_mean_var(ctx, E, d_mean, d_var));
    return MCLBM_OK;
}

static int ensure_twiddles(mclbm_ctx* ctx)
{
    if (!ctx->twiddles_ready) {
        MCLBM_CUDA(launch_twiddles(ctx));
        ctx->twiddles_ready = true;
    }
    return MCLBM_OK;
}

int mclbm_spectrum(mclbm_ctx* ctx, double* E)
{
    if (!ctx || !E) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    int st = ensure_twiddles(ctx);
    if (st != MCLBM_OK) return st;
    MCLBM_CUDA(launch_spectral(ctx, E, nullptr));
    return MCLBM_OK;
}

int mclbm_sf_trace(mclbm_ctx* ctx, double* S2)
{
    if (!ctx || !S2) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    int st = ensure_twiddles(ctx);
    if (st != MCLBM_OK) return st;
    MCLBM_CUDA(launch_spectral(ctx, nullptr, S2));
    return MCLBM_OK;
}

int mclbm_sf_axes(mclbm_ctx* ctx, int32_t pmax, double* S)
{
    if (!ctx || !S || pmax < 2 || pmax > 8) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument (2 <= pmax <= 8)");
    MCLBM_ON_DEVICE(ctx->device);
    if (ctx->N > 512) return set_error(MCLBM_ERR_SHAPE, "axis structure functions support N <= 512");
    MCLBM_CUDA(launch_sf_axes(ctx, pmax, S));
    return MCLBM_OK;
}

int mclbm_restrict(const mclbm_ctx* ctx, int32_t Qd, double* d_out)
{
    if (!ctx || !d_out || Qd < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    if (ctx->N % Qd != 0) return set_error(MCLBM_ERR_SHAPE, "N must be a multiple of Q");
    MCLBM_CUDA(launch_restrict(ctx, Qd, d_out));
    return MCLBM_OK;
}

size_t mclbm_w1_work_bytes(int32_t MA, int32_t MB, int32_t G) { return w1_work_bytes(MA, MB, G); }

int mclbm_w1_restricted(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G, void* d_work,
                        size_t work_bytes, void* cuda_stream, double* W, double* per_point)
{
    if (!d_a || !d_b || !d_work || !W || G < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    if (MA < 1 || MB < 1 || MA > kMaxW1Samples || MB > kMaxW1Samples)
        return set_error(MCLBM_ERR_SHAPE, "W1 supports 1..2048 samples per ensemble");
    if (work_bytes < w1_work_bytes(MA, MB, G)) return set_error(MCLBM_ERR_OOM, "W1 work buffer too small");
    MCLBM_CUDA(launch_w1(d_a, MA, d_b, MB, G, (char*)d_work, work_bytes, (cudaStream_t)cuda_stream, W, per_point));
    return MCLBM_OK;
}

int mclbm_w1_1pt(mclbm_ctx* A, const mclbm_ctx* B, int32_t Qd, double* W, double* per_point)
{
    if (!A || !B || !W || Qd < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    if (A->device != B->device) return set_error(MCLBM_ERR_INVALID_ARG, "both ensembles must be on one device");
    MCLBM_ON_DEVICE(A->device);
    if (A->N % Qd || B->N % Qd) return set_error(MCLBM_ERR_SHAPE, "N of both ensembles must be multiples of Q");
    if (Qd > 8) return set_error(MCLBM_ERR_SHAPE, "context W1 supports Q <= 8");
    if (B->M > kMaxW1Samples || A->M > kMaxW1Samples)
        return set_error(MCLBM_ERR_SHAPE, "W1 supports 1..2048 samples per ensemble");
    const int G = Qd * Qd * Qd;
    char* region = A->work + A->wl.total;
    double* ra = (double*)region;
    double* rb = ra + (size_t)A->M * G * 3;
    char* scratch = region + (((size_t)(A->M + kMaxW1Samples) * 512 * 3 * sizeof(double) + 255) / 256 * 256);
    // B's pending work is on B's stream: finish it, then read B from A's stream
    MCLBM_CUDA(cudaStreamSynchronize(B->stream));
    mclbm_ctx Bv = *B;
    Bv.stream = A->stream;
    MCLBM_CUDA(launch_restrict(A, Qd, ra));
    MCLBM_CUDA(launch_restrict(&Bv, Qd, rb));
    MCLBM_CUDA(launch_w1(ra, A->M, rb, B->M, G, scratch, w1_work_bytes(A->M, B->M, G), A->stream, W, per_point));
    return MCLBM_OK;
}

int mclbm_device_status(mclbm_ctx* ctx)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    MCLBM_ON_DEVICE(ctx->device);
    int flags[2] = {0, 0};
    MCLBM_CUDA(cudaMemcpyAsync(flags, ctx->work + ctx->wl.flag, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream));
    MCLBM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (flags[1] == MCLBM_ERR_TIMEOUT)
        return set_error(MCLBM_ERR_TIMEOUT, "a bounded device wait of the staged stepper gave up");
    return MCLBM_OK;
}

int mclbm_selftest_timeout(mclbm_ctx* ctx)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    MCLBM_ON_DEVICE(ctx->device);
    MCLBM_CUDA(launch_wait_selftest(ctx));
    return MCLBM_OK;
}

// ---- checkpoint file: magic, format version, velocity count Q, config, units, steps, cur, params,
// lattice bytes, and nothing after them
namespace {
constexpr uint64_t kMagic = 0x4d434c424d434b32ull;  // "MCLBMCK2"
constexpr int32_t kFormatVersion = 2;

// The fields that fix the dynamics of a resumed state: a checkpoint restores only into a context
// whose lattice, shape, storage, streaming pattern, units and options are the same.
bool same_dynamics(const mclbm_config& a, const mclbm_units& ua, const mclbm_config& b, const mclbm_units& ub,
                   std::string* why)
{
    if (a.N != b.N || a.M != b.M) { *why = "N or M"; return false; }
    if (a.precision != b.precision) { *why = "storage precision"; return false; }
    if (a.pattern != b.pattern) { *why = "streaming pattern"; return false; }
    if (a.options != b.options) { *why = "options (exact gamma / Leray)"; return false; }
    if (a.nu != b.nu || a.U_c != b.U_c) { *why = "viscosity or U_c"; return false; }
    if (ua.dt != ub.dt || ua.U_lat != ub.U_lat || ua.omega != ub.omega) { *why = "time step, Ma or omega"; return false; }
    return true;
}
}  // namespace

int mclbm_save(const mclbm_ctx* ctx, const char* path)
{
    if (!ctx || !path) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    const size_t bytes = ctx->elem_bytes * Q * (size_t)ctx->n * ctx->M;
    std::vector<char> host(bytes);
    MCLBM_CUDA(cudaMemcpyAsync(host.data(), lattice_ptr(ctx, ctx->cur), bytes, cudaMemcpyDeviceToHost, ctx->stream));
    MCLBM_CUDA(cudaStreamSynchronize(ctx->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return set_error(MCLBM_ERR_IO, std::string("cannot open ") + path + " for writing");
    const uint64_t magic = kMagic, steps = (uint64_t)ctx->steps;
    const int32_t version = kFormatVersion, q = Q, cur = ctx->cur;
    bool ok = std::fwrite(&magic, sizeof magic, 1, fp) == 1 && std::fwrite(&version, sizeof version, 1, fp) == 1 &&
              std::fwrite(&q, sizeof q, 1, fp) == 1 && std::fwrite(&ctx->cfg, sizeof ctx->cfg, 1, fp) == 1 &&
              std::fwrite(&ctx->units, sizeof ctx->units, 1, fp) == 1 &&
              std::fwrite(&steps, sizeof steps, 1, fp) == 1 && std::fwrite(&cur, sizeof cur, 1, fp) == 1 &&
              std::fwrite(ctx->params.data(), sizeof(double), ctx->params.size(), fp) == ctx->params.size() &&
              std::fwrite(host.data(), 1, bytes, fp) == bytes;
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return set_error(MCLBM_ERR_IO, std::string("writing ") + path + " failed");
    return MCLBM_OK;
}

int mclbm_load(mclbm_ctx* ctx, const char* path)
{
    if (!ctx || !path) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return set_error(MCLBM_ERR_IO, std::string("cannot open ") + path);
    uint64_t magic = 0, steps = 0;
    int32_t version = 0, q = 0, cur = 0;
    mclbm_config cfg;
    mclbm_units units;
    bool ok = std::fread(&magic, sizeof magic, 1, fp) == 1 && magic == kMagic &&
              std::fread(&version, sizeof version, 1, fp) == 1 && std::fread(&q, sizeof q, 1, fp) == 1 &&
              std::fread(&cfg, sizeof cfg, 1, fp) == 1 && std::fread(&units, sizeof units, 1, fp) == 1;
    if (!ok) {
        std::fclose(fp);
        return set_error(MCLBM_ERR_IO, std::string("reading ") + path + " failed (truncated or not a checkpoint)");
    }
    if (version != kFormatVersion) {
        std::fclose(fp);
        return set_error(MCLBM_ERR_IO, "checkpoint format version " + std::to_string(version) + " is not " +
                                           std::to_string(kFormatVersion));
    }
    std::string why;
    if (q != Q) {
        std::fclose(fp);
        return set_error(MCLBM_ERR_SHAPE, "checkpoint holds a D3Q" + std::to_string(q) + " lattice, the library is D3Q" +
                                              std::to_string(Q));
    }
    if (!same_dynamics(cfg, units, ctx->cfg, ctx->units, &why)) {
        std::fclose(fp);
        return set_error(MCLBM_ERR_SHAPE, "checkpoint differs from the context in " + why);
    }
    std::vector<double> params(ctx->params.size());
    const size_t bytes = ctx->elem_bytes * Q * (size_t)ctx->n * ctx->M;
    std::vector<char> host(bytes);
    ok = std::fread(&steps, sizeof steps, 1, fp) == 1 && std::fread(&cur, sizeof cur, 1, fp) == 1 &&
         std::fread(params.data(), sizeof(double), params.size(), fp) == params.size() &&
         std::fread(host.data(), 1, bytes, fp) == bytes;
    const bool at_end = ok && std::fgetc(fp) == EOF;
    std::fclose(fp);
    if (!ok) return set_error(MCLBM_ERR_IO, std::string("reading ") + path + " failed (truncated)");
    if (!at_end) return set_error(MCLBM_ERR_IO, std::string(path) + " has bytes after the lattice (not this layout)");
    if (cur != 0 && cur != 1) return set_error(MCLBM_ERR_IO, "corrupt checkpoint");
    ctx->cur = cur;
    ctx->steps = (int64_t)steps;
    ctx->params = params;
    MCLBM_CUDA(cudaMemcpyAsync(lattice_ptr(ctx, ctx->cur), host.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
    MCLBM_CUDA(cudaMemsetAsync(ctx->work + ctx->wl.flag, 0, 16 * sizeof(int), ctx->stream));
    MCLBM_CUDA(cudaStreamSynchronize(ctx->stream));
    return MCLBM_OK;
}

int mclbm_check_finite(mclbm_ctx* ctx)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    MCLBM_ON_DEVICE(ctx->device);
    int bad = 0;
    MCLBM_CUDA(launch_check_finite(ctx, &bad));
    if (bad) return set_error(MCLBM_ERR_NONFINITE, "non-finite population found");
    return MCLBM_OK;
}

}  // extern "C"

namespace mclbm {
int reinit_ctx(mclbm_ctx* c) { return do_init(c); }
}  // namespace mclbm
