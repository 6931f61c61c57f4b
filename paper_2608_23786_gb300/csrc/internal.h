// Library-internal declarations shared by the translation units of libmclbm.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mclbm.h"
#include "launch.h"

namespace mclbm {

// Sub-allocation of the caller's work buffer (byte offsets, 256-aligned).
struct WorkLayout {
    size_t params;    // [M][24] double
    size_t partial;   // reduction partials, kPartialBytes
    size_t flag;      // int status words (16 ints)
    size_t field;     // velocity fields [4][n] double: one sample's [3][n], or during the paired
                      // spectra the second sample's [3][n] below the first one's u_z
    size_t cplx;      // complex FFT buffer [n] double2
    size_t real;      // power spectrum / autocorrelation [n] double
    size_t real2;     // power spectrum of the second sample of a pair [n] double
    size_t twiddle;   // [N] double2: exp(-2 pi i j / N), j < N
    size_t trig;      // [N][4] double: sin, cos of x_n and 2 x_n; then the same [N][4] as float
    size_t bins;      // shell sums [2][N/2+1] double x M
    size_t total;
};

constexpr size_t kPartialBytes = size_t(8) << 20;  // 8 MiB of reduction partials
constexpr int kMaxW1Samples = 2048;                 // per ensemble in the W1 kernels

}  // namespace mclbm

struct mclbm_ctx {
    mclbm_config cfg;
    mclbm_units units;
    int N, logN, M;
    int64_t n;
    void* pop;
    size_t pop_bytes;
    char* work;
    size_t work_bytes;
    mclbm::WorkLayout wl;
    cudaStream_t stream;
    int device;
    int cur;         // pull: lattice (0/1) holding the current state
    int64_t steps;   // steps since the last initialisation
    std::vector<double> params;       // host copy [M][24]
    std::vector<double> init_coeffs;  // coefficients the initialisation evaluates (L params with the Leray option)
    size_t elem_bytes;
    bool twiddles_ready;  // FFT twiddle table computed in the work buffer
    mclbm::LaunchConfig launch;      // stepper variant of pull steps and AA even steps (autotuned or default)
    mclbm::LaunchConfig launch_odd;  // AA odd steps (pull: equal to launch)
    int num_sms;
    double grad_ms[4];  // last mclbm_grad: forward, recompute, reverse (adjoint kernels), parameter reduction
};

namespace mclbm {

// error reporting (thread-local message)
int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
#define MCLBM_CUDA(call)                                           \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::mclbm::cuda_check(e_, #call); \
    } while (0)

// Makes a context's device (the device current at its creation) current for the duration of a
// call on it, and restores the caller's device afterwards.  A call whose switch fails returns
// MCLBM_ERR_CUDA before it enqueues anything (MCLBM_ON_DEVICE).
class DeviceScope {
public:
    explicit DeviceScope(int device)
    {
        if (cudaGetDevice(&prev_) != cudaSuccess) return;
        if (prev_ == device) {
            ok_ = true;
        } else if (cudaSetDevice(device) == cudaSuccess) {
            ok_ = switched_ = true;
        }
    }
    ~DeviceScope()
    {
        if (switched_) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;

private:
    int prev_ = -1;
    bool ok_ = false, switched_ = false;
};
#define MCLBM_ON_DEVICE(device)                                                                         \
    ::mclbm::DeviceScope mclbm_device_scope_(device);                                                   \
    if (!mclbm_device_scope_.ok())                                                                      \
        return ::mclbm::set_error(MCLBM_ERR_CUDA, "the context's device could not be made current")

WorkLayout work_layout(int N, int M);

// pointers of the population lattices
void* lattice_ptr(const mclbm_ctx* c, int which);

// kernels (launchers return cudaError_t of the launch)
cudaError_t launch_init(const mclbm_ctx* c, const double* d_params);
cudaError_t launch_step(mclbm_ctx* c);  // one step of one context; updates cur and steps
cudaError_t launch_step_with(mclbm_ctx* c, const LaunchConfig& cfg, const LaunchConfig& cfg_odd);
cudaError_t launch_wait_selftest(mclbm_ctx* c);
// one step of several levels in one launch; updates each level's cur and steps
// (AA levels at an odd step take cfg_odd, unless cfg is the staged kind, which serves both)
cudaError_t launch_levels(mclbm_ctx* const* levels, int nlev, const LaunchConfig& cfg, const LaunchConfig& cfg_odd,
                          cudaStream_t s, int* occ);
bool vec_supported(int precision, int vec);
bool launch_supported(int precision, const LaunchConfig& c);
LaunchConfig default_launch(int precision, int pattern, int options);
LaunchConfig default_launch_odd(int precision, int pattern, int options, int Nmax);  // AA odd steps
int exact_vec(int precision);  // the one VEC of the exact-gamma kernel (kind 6)
void leray_map(const double* X, int M, bool transpose, double* Y);  // api.cu
cudaError_t launch_get_populations(const mclbm_ctx* c, int sample, double* d_out);
cudaError_t launch_set_populations(mclbm_ctx* c, int sample, const double* d_in);
cudaError_t launch_moments(const mclbm_ctx* c, int sample, double* d_rho, double* d_u);
cudaError_t launch_field(const mclbm_ctx* c, int sample, double* d_u);  // physical u [3][n]
cudaError_t launch_energy(mclbm_ctx* c, bool with_enstrophy, double* h_E, double* h_Z);
cudaError_t launch_mean_var(const mclbm_ctx* c, double* d_mean, double* d_var);
// mean/var fields and E_m in one pass over the populations (M <= 1024)
cudaError_t launch_energy_mean_var(const mclbm_ctx* c, double* h_E, double* d_mean, double* d_var);
cudaError_t launch_restrict(const mclbm_ctx* c, int Q, double* d_out);
cudaError_t launch_check_finite(mclbm_ctx* c, int* h_bad);
cudaError_t launch_spectral(mclbm_ctx* c, double* h_E, double* h_S2);
cudaError_t launch_sf_axes(mclbm_ctx* c, int pmax, double* h_S);
cudaError_t launch_w1(const double* d_a, int MA, const double* d_b, int MB, int G, char* work, size_t work_bytes,
                      cudaStream_t s, double* h_W, double* h_per_point);
size_t w1_work_bytes(int MA, int MB, int G);

}  // namespace mclbm
