// Batched multi-level stepping, CUDA-graph capture of the schedule, and the
// autotuner of the stepper's launch shape.
//
// A batch holds the levels of a viscosity sequence (each an ensemble context).
// Under diffusive scaling (dt ~ dx^2, Remark "Diffusive scaling"), halving dx with
// the Mach number halved quarters dt, so level l takes substeps[l] lattice steps per
// macro step (e.g. 1, 4, 16).  Sub-step s of a macro step advances every level with
// s % (S / substeps[l]) == 0 (S = max substeps), all of them in one persistent launch
// of the stepper kernel.  The S launches of a macro step (two macro steps when some
// level takes an odd number of steps, so that every level's lattice parity returns
// to its start) are captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "internal.h"

struct mclbm_batch {
    std::vector<mclbm_ctx*> lev;
    std::vector<int> sub;
    int S;
    int period;  // macro steps per captured graph
    cudaStream_t stream;
    mclbm::LaunchConfig launch;      // pull steps and AA even steps
    mclbm::LaunchConfig launch_odd;  // AA odd steps
    bool use_graph;
    bool warmed;
    std::map<std::vector<int64_t>, cudaGraphExec_t> graphs;
    int64_t macro_steps;
};

namespace mclbm {
int reinit_ctx(mclbm_ctx* c);  // api.cu: re-run the initialisation from the stored parameters
}

using namespace mclbm;

namespace {

std::vector<int64_t> signature(const mclbm_batch* b)
{
    std::vector<int64_t> s;
    for (auto* c : b->lev) {
        s.push_back(c->cur);
        s.push_back(c->steps & 1);
    }
    return s;
}

void clear_graphs(mclbm_batch* b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

cudaError_t macro_direct(mclbm_batch* b, const LaunchConfig& cfg, const LaunchConfig& cfg_odd)
{
    std::vector<mclbm_ctx*> part;
    for (int s = 0; s < b->S; ++s) {
        part.clear();
        for (size_t l = 0; l < b->lev.size(); ++l)
            if (s % (b->S / b->sub[l]) == 0) part.push_back(b->lev[l]);
        if (part.empty()) continue;
        cudaError_t e = launch_levels(part.data(), (int)part.size(), cfg, cfg_odd, b->stream, nullptr);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

struct Saved {
    std::vector<int> cur;
    std::vector<int64_t> steps;
};
Saved save(const mclbm_batch* b)
{
    Saved s;
    for (auto* c : b->lev) {
        s.cur.push_back(c->cur);
        s.steps.push_back(c->steps);
    }
    return s;
}
void restore(mclbm_batch* b, const Saved& s)
{
    for (size_t l = 0; l < b->lev.size(); ++l) {
        b->lev[l]->cur = s.cur[l];
        b->lev[l]->steps = s.steps[l];
    }
}

int capture(mclbm_batch* b, cudaGraphExec_t* out)
{
    const Saved before = save(b);
    MCLBM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < b->period && e == cudaSuccess; ++p) e = macro_direct(b, b->launch, b->launch_odd);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    restore(b, before);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_check(e, "kernel launch during graph capture");
    }
    if (e2 != cudaSuccess) return cuda_check(e2, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_check(e, "cudaGraphInstantiate");
    *out = exec;
    return MCLBM_OK;
}

template <class F>
int time_ms(cudaStream_t s, F&& body, double* ms)
{
    cudaEvent_t a, z;
    MCLBM_CUDA(cudaEventCreate(&a));
    MCLBM_CUDA(cudaEventCreate(&z));
    MCLBM_CUDA(cudaEventRecord(a, s));
    cudaError_t e = body();
    cudaError_t e1 = cudaEventRecord(z, s);
    cudaError_t e2 = cudaEventSynchronize(z);
    float t = 0;
    cudaEventElapsedTime(&t, a, z);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (e != cudaSuccess) return cuda_check(e, "autotune trial");
    if (e1 != cudaSuccess) return cuda_check(e1, "cudaEventRecord");
    if (e2 != cudaSuccess) return cuda_check(e2, "cudaEventSynchronize");
    *ms = t;
    return MCLBM_OK;
}

std::vector<LaunchConfig> candidates(int precision, int N, bool exact)
{
    std::vector<LaunchConfig> v;
    if (exact) {  // the exact entropic gamma runs in its one kernel
        v.push_back(LaunchConfig{exact_vec(precision), 128, 6});
        return v;
    }
    const int* vecs;
    int nv;
    if (precision == MCLBM_FP64) {
        vecs = kVecF64;
        nv = sizeof(kVecF64) / sizeof(int);
    } else if (precision == MCLBM_FP32) {
        vecs = kVecF32;
        nv = sizeof(kVecF32) / sizeof(int);
    } else {
        vecs = kVecF16;
        nv = sizeof(kVecF16) / sizeof(int);
    }
    for (int kind : {0, 2, 3, 4, 5})
        for (int i = 0; i < nv; ++i)
            for (int blk : kBlocks)
                if (N % vecs[i] == 0 && launch_supported(precision, LaunchConfig{vecs[i], blk, kind}))
                    v.push_back(LaunchConfig{vecs[i], blk, kind});
    for (int vs : kVecStaged)
        if (N % vs == 0) v.push_back(LaunchConfig{vs, 0, 1});
    return v;
}

int check_shape(const mclbm_ctx* ctx, const LaunchConfig& c)
{
    if (!launch_supported(ctx->cfg.precision, c) || c.vec < 1 || ctx->N % c.vec)
        return set_error(MCLBM_ERR_INVALID_ARG, "unsupported launch shape (kind " + std::to_string(c.kind) + ", vec " +
                                                    std::to_string(c.vec) + ", block " + std::to_string(c.block) + ")");
    if ((c.kind == 6) != ((ctx->cfg.options & MCLBM_OPT_EXACT_GAMMA) != 0))
        return set_error(MCLBM_ERR_INVALID_ARG, "kind 6 is the launch of contexts with MCLBM_OPT_EXACT_GAMMA, and only it");
    return MCLBM_OK;
}

// Shape of one parity given as (kind, vec, block): parity 1 (AA odd steps) needs an AA context,
// and the staged kind serves both parities, so it is set (or replaced) for both.
int set_parity_shape(const std::vector<mclbm_ctx*>& lev, LaunchConfig& even, LaunchConfig& odd, int parity,
                     const LaunchConfig& c)
{
    if (parity != 0 && parity != 1) return set_error(MCLBM_ERR_INVALID_ARG, "parity must be 0 or 1");
    if (parity == 1 && lev[0]->cfg.pattern != MCLBM_AA)
        return set_error(MCLBM_ERR_INVALID_ARG, "parity 1 (odd steps) has its own shape only under AA streaming");
    for (auto* l : lev) {
        int st = check_shape(l, c);
        if (st != MCLBM_OK) return st;
    }
    if (c.kind == 1 || (parity == 0 ? odd.kind : even.kind) == 1) {
        even = odd = c;
    } else {
        (parity == 0 ? even : odd) = c;
    }
    return MCLBM_OK;
}

}  // namespace

extern "C" {

int mclbm_set_launch(mclbm_ctx* ctx, int32_t kind, int32_t vec, int32_t block)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    const LaunchConfig c{vec, kind == 1 ? 0 : block, kind};
    int st = check_shape(ctx, c);
    if (st != MCLBM_OK) return st;
    ctx->launch = ctx->launch_odd = c;
    return MCLBM_OK;
}

int mclbm_get_launch(const mclbm_ctx* ctx, int32_t* kind, int32_t* vec, int32_t* block)
{
    return mclbm_get_launch_parity(ctx, 0, kind, vec, block);
}

int mclbm_set_launch_parity(mclbm_ctx* ctx, int32_t parity, int32_t kind, int32_t vec, int32_t block)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    const std::vector<mclbm_ctx*> one{ctx};
    return set_parity_shape(one, ctx->launch, ctx->launch_odd, parity, LaunchConfig{vec, kind == 1 ? 0 : block, kind});
}

int mclbm_get_launch_parity(const mclbm_ctx* ctx, int32_t parity, int32_t* kind, int32_t* vec, int32_t* block)
{
    if (!ctx) return set_error(MCLBM_ERR_INVALID_ARG, "ctx is NULL");
    if (parity != 0 && parity != 1) return set_error(MCLBM_ERR_INVALID_ARG, "parity must be 0 or 1");
    const LaunchConfig& c = parity == 0 ? ctx->launch : ctx->launch_odd;
    if (kind) *kind = c.kind;
    if (vec) *vec = c.vec;
    if (block) *block = c.block;
    return MCLBM_OK;
}

int mclbm_autotune(mclbm_ctx* ctx, int32_t trial_steps, int32_t* kind, int32_t* vec, int32_t* block, double* best_ms)
{
    if (!ctx || trial_steps < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    if (ctx->steps != 0) return set_error(MCLBM_ERR_INVALID_ARG, "autotune must directly follow an initialisation");
    // per candidate the time of its even and of its odd steps (one event pair per step; pull
    // steps all count as even).  AA: the fastest shape of each parity, unless the staged
    // kind (which serves both parities) is faster over a pair of steps.
    const bool aa = ctx->cfg.pattern == MCLBM_AA;
    double best[2] = {1e300, 1e300}, best_staged = 1e300;
    LaunchConfig bestc[2] = {ctx->launch, ctx->launch_odd}, staged{};
    for (const LaunchConfig& c : candidates(ctx->cfg.precision, ctx->N, (ctx->cfg.options & MCLBM_OPT_EXACT_GAMMA) != 0)) {
        MCLBM_CUDA(launch_step_with(ctx, c, c));  // warm-up (first use also sizes the grid)
        double t[2] = {0, 0};
        int n[2] = {0, 0};
        for (int s = 0; s < (aa ? 2 : 1) * trial_steps; ++s) {
            const int par = aa ? (int)(ctx->steps & 1) : 0;
            double ms = 0;
            int st = time_ms(ctx->stream, [&]() { return launch_step_with(ctx, c, c); }, &ms);
            if (st != MCLBM_OK) return st;
            t[par] += ms;
            n[par] += 1;
        }
        for (int p = 0; p < (aa ? 2 : 1); ++p) {
            const double per = t[p] / n[p];
            if (c.kind != 1 && per < best[p]) {
                best[p] = per;
                bestc[p] = c;
            }
        }
        const double pair = aa ? t[0] / n[0] + t[1] / n[1] : t[0] / n[0];
        if (c.kind == 1 && pair < best_staged) {
            best_staged = pair;
            staged = c;
        }
    }
    double per_step;
    if (!aa) {
        if (best_staged < best[0]) bestc[0] = staged, best[0] = best_staged;
        ctx->launch = ctx->launch_odd = bestc[0];
        per_step = best[0];
    } else if (best_staged < best[0] + best[1]) {
        ctx->launch = ctx->launch_odd = staged;
        per_step = best_staged / 2;
    } else {
        ctx->launch = bestc[0];
        ctx->launch_odd = bestc[1];
        per_step = (best[0] + best[1]) / 2;
    }
    int st = reinit_ctx(ctx);
    if (st != MCLBM_OK) return st;
    if (kind) *kind = ctx->launch.kind;
    if (vec) *vec = ctx->launch.vec;
    if (block) *block = ctx->launch.block;
    if (best_ms) *best_ms = per_step;
    return MCLBM_OK;
}

int mclbm_batch_create(mclbm_ctx* const* levels, int32_t nlev, const int32_t* substeps, mclbm_batch** out)
{
    if (!levels || !substeps || !out || nlev < 1 || nlev > kMaxLevels)
        return set_error(MCLBM_ERR_INVALID_ARG, "need 1.." + std::to_string(kMaxLevels) + " levels");
    *out = nullptr;
    int S = 1;
    for (int l = 0; l < nlev; ++l) {
        if (!levels[l] || substeps[l] < 1 || substeps[l] > 4096) return set_error(MCLBM_ERR_INVALID_ARG, "bad level");
        if (substeps[l] > S) S = substeps[l];
        if (levels[l]->cfg.precision != levels[0]->cfg.precision || levels[l]->cfg.pattern != levels[0]->cfg.pattern)
            return set_error(MCLBM_ERR_INVALID_ARG, "levels of a batch share precision and streaming pattern");
        if ((levels[l]->cfg.options & MCLBM_OPT_EXACT_GAMMA) != (levels[0]->cfg.options & MCLBM_OPT_EXACT_GAMMA))
            return set_error(MCLBM_ERR_INVALID_ARG, "levels of a batch share the gamma option");
        if (levels[l]->stream != levels[0]->stream || levels[l]->device != levels[0]->device)
            return set_error(MCLBM_ERR_INVALID_ARG, "levels of a batch share device and stream");
        for (int k = 0; k < l; ++k)
            if (levels[k] == levels[l]) return set_error(MCLBM_ERR_INVALID_ARG, "a level appears twice");
    }
    int odd = 0;
    for (int l = 0; l < nlev; ++l) {
        if (S % substeps[l]) return set_error(MCLBM_ERR_INVALID_ARG, "every substeps[l] must divide the largest");
        odd |= substeps[l] & 1;
    }
    mclbm_batch* b = new mclbm_batch();
    b->lev.assign(levels, levels + nlev);
    b->sub.assign(substeps, substeps + nlev);
    b->S = S;
    b->period = odd ? 2 : 1;
    b->stream = levels[0]->stream;
    b->launch = levels[0]->launch;
    b->launch_odd = levels[0]->launch_odd;
    {
        // levels[0] on its default odd-step shape: the batch takes the default for its largest level
        const mclbm_config& c0 = levels[0]->cfg;
        int Nmax = 0;
        for (int l = 0; l < nlev; ++l) Nmax = levels[l]->N > Nmax ? levels[l]->N : Nmax;
        const LaunchConfig d0 = default_launch_odd(c0.precision, c0.pattern, c0.options, levels[0]->N);
        const LaunchConfig& cur = levels[0]->launch_odd;
        if (cur.kind == d0.kind && cur.vec == d0.vec && cur.block == d0.block) {
            const LaunchConfig dm = default_launch_odd(c0.precision, c0.pattern, c0.options, Nmax);
            bool ok = true;
            for (int l = 0; l < nlev; ++l) ok = ok && launch_supported(c0.precision, dm) && levels[l]->N % dm.vec == 0;
            if (ok) b->launch_odd = dm;
        }
    }
    b->use_graph = b->stream != nullptr;
    b->warmed = false;
    b->macro_steps = 0;
    *out = b;
    return MCLBM_OK;
}

void mclbm_batch_destroy(mclbm_batch* b)
{
    if (!b) return;
    {
        const DeviceScope scope(b->lev[0]->device);
        clear_graphs(b);
    }
    delete b;
}

int mclbm_batch_set_graph(mclbm_batch* b, int32_t enable)
{
    if (!b) return set_error(MCLBM_ERR_INVALID_ARG, "batch is NULL");
    if (enable && b->stream == nullptr)
        return set_error(MCLBM_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    b->use_graph = enable != 0;
    return MCLBM_OK;
}

int mclbm_batch_set_launch(mclbm_batch* b, int32_t kind, int32_t vec, int32_t block)
{
    if (!b) return set_error(MCLBM_ERR_INVALID_ARG, "batch is NULL");
    MCLBM_ON_DEVICE(b->lev[0]->device);
    const LaunchConfig lc{vec, kind == 1 ? 0 : block, kind};
    for (auto* c : b->lev) {
        int st = check_shape(c, lc);
        if (st != MCLBM_OK) return st;
    }
    b->launch = b->launch_odd = lc;
    clear_graphs(b);
    b->warmed = false;
    return MCLBM_OK;
}

int mclbm_batch_set_launch_parity(mclbm_batch* b, int32_t parity, int32_t kind, int32_t vec, int32_t block)
{
    if (!b) return set_error(MCLBM_ERR_INVALID_ARG, "batch is NULL");
    MCLBM_ON_DEVICE(b->lev[0]->device);
    int st = set_parity_shape(b->lev, b->launch, b->launch_odd, parity, LaunchConfig{vec, kind == 1 ? 0 : block, kind});
    if (st != MCLBM_OK) return st;
    clear_graphs(b);
    b->warmed = false;
    return MCLBM_OK;
}

int mclbm_batch_get_launch_parity(const mclbm_batch* b, int32_t parity, int32_t* kind, int32_t* vec, int32_t* block)
{
    if (!b) return set_error(MCLBM_ERR_INVALID_ARG, "batch is NULL");
    if (parity != 0 && parity != 1) return set_error(MCLBM_ERR_INVALID_ARG, "parity must be 0 or 1");
    const LaunchConfig& c = parity == 0 ? b->launch : b->launch_odd;
    if (kind) *kind = c.kind;
    if (vec) *vec = c.vec;
    if (block) *block = c.block;
    return MCLBM_OK;
}

int mclbm_batch_step(mclbm_batch* b, int64_t macro_steps)
{
    if (!b || macro_steps < 0) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(b->lev[0]->device);
    while (macro_steps > 0) {
        if (b->use_graph && b->warmed && macro_steps >= b->period) {
            const auto sig = signature(b);
            auto it = b->graphs.find(sig);
            if (it == b->graphs.end()) {
                cudaGraphExec_t g = nullptr;
                int st = capture(b, &g);
                if (st != MCLBM_OK) return st;
                it = b->graphs.emplace(sig, g).first;
            }
            MCLBM_CUDA(cudaGraphLaunch(it->second, b->stream));
            for (size_t l = 0; l < b->lev.size(); ++l) b->lev[l]->steps += (int64_t)b->period * b->sub[l];
            b->macro_steps += b->period;
            macro_steps -= b->period;
        } else {
            MCLBM_CUDA(macro_direct(b, b->launch, b->launch_odd));
            b->warmed = true;
            b->macro_steps += 1;
            macro_steps -= 1;
        }
    }
    return MCLBM_OK;
}

int mclbm_batch_autotune(mclbm_batch* b, int32_t trials, int32_t* kind, int32_t* vec, int32_t* block, double* best_ms)
{
    if (!b || trials < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(b->lev[0]->device);
    for (auto* c : b->lev)
        if (c->steps != 0) return set_error(MCLBM_ERR_INVALID_ARG, "autotune must directly follow an initialisation");
    int prec = b->lev[0]->cfg.precision, Nmin = 1 << 30;
    for (auto* c : b->lev) Nmin = c->N < Nmin ? c->N : Nmin;
    const std::vector<LaunchConfig> cands =
        candidates(prec, Nmin, (b->lev[0]->cfg.options & MCLBM_OPT_EXACT_GAMMA) != 0);
    auto fits = [&](const LaunchConfig& c) {
        for (auto* l : b->lev)
            if (l->N % c.vec) return false;
        return true;
    };
    auto trial = [&](const LaunchConfig& even, const LaunchConfig& odd, double* ms) {
        cudaError_t e = macro_direct(b, even, odd);
        if (e != cudaSuccess) return cuda_check(e, "autotune trial");
        return time_ms(
            b->stream,
            [&]() {
                for (int t = 0; t < trials; ++t) {
                    cudaError_t e2 = macro_direct(b, even, odd);
                    if (e2 != cudaSuccess) return e2;
                }
                return cudaSuccess;
            },
            ms);
    };
    // pass 1: one shape for both parities; pass 2 (AA, unless the staged kind won): the odd
    // steps' shape with the even steps' shape of pass 1
    double best = 1e300;
    LaunchConfig bestc = b->launch, besto = b->launch_odd;
    for (const LaunchConfig& c : cands) {
        if (!fits(c)) continue;
        double ms = 0;
        int st = trial(c, c, &ms);
        if (st != MCLBM_OK) return st;
        if (ms < best) {
            best = ms;
            bestc = besto = c;
        }
    }
    if (b->lev[0]->cfg.pattern == MCLBM_AA && bestc.kind != 1)
        for (const LaunchConfig& c : cands) {
            if (!fits(c) || c.kind == 1 || (c.vec == bestc.vec && c.block == bestc.block && c.kind == bestc.kind))
                continue;
            double ms = 0;
            int st = trial(bestc, c, &ms);
            if (st != MCLBM_OK) return st;
            if (ms < best) {
                best = ms;
                besto = c;
            }
        }
    b->launch = bestc;
    b->launch_odd = besto;
    clear_graphs(b);
    b->warmed = false;
    for (auto* c : b->lev) {
        int st = reinit_ctx(c);
        if (st != MCLBM_OK) return st;
    }
    b->macro_steps = 0;
    if (kind) *kind = bestc.kind;
    if (vec) *vec = bestc.vec;
    if (block) *block = bestc.block;
    if (best_ms) *best_ms = best / trials;
    return MCLBM_OK;
}

int64_t mclbm_batch_macro_steps(const mclbm_batch* b) { return b ? b->macro_steps : -1; }

}  // extern "C"
