// Warp-specialised stream + KBC collide kernel with shared-memory staging of the
// source rows by bulk asynchronous copies (cp.async.bulk, completion on mbarriers).
//
// Tiles.  A tile is TY consecutive rows (all N x) of one z-plane of one sample of one
// level.  For population i the tile needs rows y - c_iy of plane z - c_iz (slot i for
// pull and even AA steps without the shift, slot opp(i) for odd AA steps): TY
// contiguous rows, or two pieces where the shift wraps around y.  So a tile is 19..21
// row-block copies of whole rows (N * b bytes per row: 16-byte aligned and sized for
// every N >= 8), and the x-shift is applied when the consumers read shared memory,
// with the periodic wrap inside the row.
//
// Warp roles.  The last warp's first lane is the producer: it walks the block's
// tiles, waits until the consumers have released a stage (`empty` barrier), arms the
// stage's `full` barrier with the tile's byte count and issues the copies.  The other
// warps are consumers: they wait on `full`, collide every node of the tile and store
// the post-collision populations straight to global memory (vector stores where the
// destination is aligned), then release the stage.  With STAGES stages in flight per
// block the memory system sees tens of kilobytes of outstanding reads per block
// independent of the consumers' register use.
//
// Every wait is bounded in time: it polls mbarrier.try_wait (each poll may suspend the
// thread for at most kSuspendHintNs) until the barrier completes or kWaitLimitNs of
// %globaltimer time have passed.  A wait that gives up writes MCLBM_ERR_TIMEOUT into the
// error word and the block stops taking tiles.  Consumer waits also re-read the error word
// every kErrPollEvery polls and leave as soon as it is set (by another block's timeout, or
// left over from an earlier launch, in which case the producer issues nothing), so after a
// timeout every later launch returns within about one poll interval instead of running out
// the limit.  Before returning, the producer waits (again bounded) until every copy it
// issued has landed, so no copy targets the shared memory of a finished block.
#pragma once
#include <cuda_fp16.h>

#include "stepper_impl.cuh"

namespace mclbm {

constexpr int kConsumerWarps = 8;
constexpr int kStagedThreads = (kConsumerWarps + 1) * 32;
constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;  // 200 ms of %globaltimer time per wait
constexpr uint32_t kSuspendHintNs = 2000;                 // longest suspension of one try_wait poll
constexpr int kErrPollEvery = 256;                        // consumer polls between reads of the error word
constexpr int kTimeoutCode = -6;                          // MCLBM_ERR_TIMEOUT

template <class E>
struct StagedArgs {
    int nlev;
    int stages;
    int stage_elems;                      // Q * max tile nodes
    int64_t tile_prefix[kMaxLevels + 1];  // tile offsets of the levels
    int ty[kMaxLevels];                   // rows per tile of each level
    LevelArgs<E> lev[kMaxLevels];
    int* err;                             // error word (0 = ok)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of barrier `bar` for at most limit_ns nanoseconds of %globaltimer
// time.  With err != NULL the wait also gives up as soon as *err is nonzero (read every
// kErrPollEvery polls).  Returns true when the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs,
                                                  const int* err = nullptr)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & (kErrPollEvery - 1)) == 0) {
            if (err && *(volatile const int*)err != 0) return false;
            if (global_ns() - t0 > limit_ns) return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

struct TileCoord {
    int l, m, z, y0, ty;
};

template <class E>
__device__ __forceinline__ TileCoord tile_coord(const StagedArgs<E>& a, int64_t t)
{
    int l = 0;
#pragma unroll 1
    while (l + 1 < a.nlev && t >= a.tile_prefix[l + 1]) ++l;
    const int64_t r = t - a.tile_prefix[l];
    const int N = a.lev[l].g.N, ty = a.ty[l];
    const int per_plane = N / ty;
    TileCoord c;
    c.l = l;
    c.ty = ty;
    c.y0 = (int)(r % per_plane) * ty;
    c.z = (int)((r / per_plane) % N);
    c.m = (int)(r / ((int64_t)per_plane * N));
    return c;
}

// Producer warp: copy the source rows of tile `tc` into stage buffer `buf`.  Lane 0 arms
// the stage's barrier with the tile's byte count; then lane i < 19 issues the one or two
// row-block copies of population i.
template <class E, int PATTERN>
__device__ __forceinline__ void issue_tile(const StagedArgs<E>& a, const TileCoord& tc, E* buf, uint32_t full_bar, int lane)
{
    const LevelArgs<E>& L = a.lev[tc.l];
    const Geom g = L.g;
    const int N = g.N, ty = tc.ty;
    const int64_t row_bytes = (int64_t)N * sizeof(E);
    if (lane == 0) mbar_arrive_expect_tx(full_bar, (uint32_t)(Q * ty * row_bytes));
    __syncwarp();
    if (lane >= Q) return;
    const int i = lane;
    const E* sample = L.src + (int64_t)tc.m * Q * g.n;
    const bool aa_odd = PATTERN == 1 && L.parity == 1;
    const bool shift = PATTERN == 0 || aa_odd;
    const int sl = aa_odd ? opp(i) : i;
    const int dy = shift ? cy(i) : 0, dz = shift ? cz(i) : 0;
    const E* plane = sample + (int64_t)sl * g.n + (int64_t)g.wrap(tc.z - dz) * N * N;
    const uint32_t dst = smem_u32(buf + (int64_t)i * ty * N);
    const int first = tc.y0 - dy;  // first source row (may be -1 or run past N - 1)
    if (first >= 0 && first + ty <= N) {
        bulk_g2s(dst, plane + (int64_t)first * N, (uint32_t)(ty * row_bytes), full_bar);
    } else if (first < 0) {  // rows N-1, 0, 1, ..., ty-2
        bulk_g2s(dst, plane + (int64_t)(N - 1) * N, (uint32_t)row_bytes, full_bar);
        if (ty > 1) bulk_g2s(dst + (uint32_t)row_bytes, plane, (uint32_t)((ty - 1) * row_bytes), full_bar);
    } else {  // rows first .. N-1, then 0
        const int head = N - first;
        if (head > 0) bulk_g2s(dst, plane + (int64_t)first * N, (uint32_t)(head * row_bytes), full_bar);
        bulk_g2s(dst + (uint32_t)(head * row_bytes), plane, (uint32_t)((ty - head) * row_bytes), full_bar);
    }
}

// Consumers: collide the nodes of a staged tile and store the results.
template <class E, int PATTERN, int VEC>
__device__ __forceinline__ void consume_tile(const StagedArgs<E>& a, const TileCoord& tc, const E* buf, int ctid)
{
    using C = typename Storage<E>::compute;
    const LevelArgs<E>& L = a.lev[tc.l];
    const Geom g = L.g;
    const int N = g.N, ty = tc.ty;
    const int nodes = ty * N;
    const bool aa = PATTERN == 1;
    const bool aa_odd = aa && L.parity == 1;
    const bool shift_x = PATTERN == 0 || aa_odd;
    E* sample = L.dst + (int64_t)tc.m * Q * g.n;
#pragma unroll 1
    for (int j0 = ctid * VEC; j0 < nodes; j0 += kConsumerWarps * 32 * VEC) {
        const int r = j0 / N, x0 = j0 % N;
        const int y = tc.y0 + r;
        C v[Q][VEC];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const E* rowp = buf + (int64_t)i * nodes + r * N;
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const int xs = shift_x ? ((x0 + k - cx(i)) & (N - 1)) : (x0 + k);
                v[i][k] = to_c<E>(rowp[xs]);
            }
        }
        collide_run<E, VEC>(v, L);
        if (!aa_odd) {
            const int64_t node = g.node(x0, y, tc.z);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                E w[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) w[k] = from_c<E>(v[i][k]);
                vstore<E, VEC>(sample + (int64_t)(aa ? opp(i) : i) * g.n + node, w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                E* row = sample + (int64_t)i * g.n + g.node(0, g.wrap(y + cy(i)), g.wrap(tc.z + cz(i)));
#pragma unroll
                for (int k = 0; k < VEC; ++k) row[(x0 + k + cx(i)) & (N - 1)] = from_c<E>(v[i][k]);
            }
        }
    }
}

template <class E, int PATTERN, int VEC>
__global__ void __launch_bounds__(kStagedThreads) k_step_staged(const StagedArgs<E> a)
{
    extern __shared__ __align__(128) unsigned char staged_smem[];  // the dynamic shared memory
    uint64_t* bars = reinterpret_cast<uint64_t*>(staged_smem);  // [stages] full, [stages] empty
    E* stage0 = reinterpret_cast<E*>(staged_smem + 256);
    const int S = a.stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);                  // full: the producer's arrive + bytes
            mbar_init(smem_u32(&bars[S + s]), kConsumerWarps);  // empty: one arrive per consumer warp
        }
        mbar_fence_init();
    }
    __syncthreads();
    const int64_t total = a.tile_prefix[a.nlev];
    if (warp == kConsumerWarps) {
        int64_t k = 0;
        for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++k) {
            const int s = (int)(k % S);
            const uint32_t ph = (uint32_t)((k / S) & 1);
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait_bounded(smem_u32(&bars[S + s]), ph ^ 1u, kWaitLimitNs, a.err) ? 1 : 0;
                if (!ok && *(volatile int*)a.err == 0) atomicExch(a.err, kTimeoutCode);
                if (*(volatile int*)a.err != 0) ok = 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            issue_tile<E, PATTERN>(a, tile_coord(a, t), stage0 + (int64_t)s * a.stage_elems, smem_u32(&bars[s]), lane);
            __syncwarp();
        }
        // drain: the last phase armed on every stage must have completed
        if (lane == 0) {
            const int64_t armed = k;
            for (int s = 0; s < S && s < armed; ++s) {
                const int64_t last = armed - 1 - ((armed - 1 - s) % S);  // last iteration that used stage s
                if (!mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((last / S) & 1))) atomicExch(a.err, kTimeoutCode);
            }
        }
        return;
    }
    const int ctid = threadIdx.x;  // 0 .. consumers*32 - 1
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int s = (int)(k % S);
        const uint32_t ph = (uint32_t)((k / S) & 1);
        if (!mbar_wait_bounded(smem_u32(&bars[s]), ph, kWaitLimitNs, a.err)) {
            if (*(volatile int*)a.err == 0) atomicExch(a.err, kTimeoutCode);
            break;
        }
        consume_tile<E, PATTERN, VEC>(a, tile_coord(a, t), stage0 + (int64_t)s * a.stage_elems, ctid);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars[S + s]));
    }
}

}  // namespace mclbm
