// Stepper variant with the prefetch held in shared memory.  Same thread mapping, x-shift
// shuffles and store paths as k_step_prefetch (stepper_impl.cuh), but the loads of the
// runs ahead are asynchronous copies (cp.async) into a per-thread ring of STAGES slots in
// shared memory instead of registers: the registers then hold only the run being
// collided, and STAGES - 1 runs per thread stay in flight during its arithmetic.
//
// Shared memory per block: STAGES x Q x BLOCK vectors of VEC elements, plus one 4-byte
// edge word per stage, x-moving population and thread (the element before or after the
// run that no lane holds; for FP16 the aligned pair of halves that contains it).  Each thread
// reads back only the slots it filled, after its own cp.async.wait_group, so no block
// barrier is involved and no wait can stall on another thread.
#pragma once
#include "stepper_impl.cuh"

namespace mclbm {

template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src)
{
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// populations with c_x != 0, numbered 0 .. kEdges - 1 in velocity order
constexpr int edge_index(int i)
{
    int k = 0;
    for (int j = 0; j < i; ++j) k += cx(j) != 0;
    return k;
}
constexpr int kEdges = edge_index(Q);

template <class E, int VEC, int BLOCK, int STAGES>
struct AsyncRing {
    static constexpr int kVB = VEC * (int)sizeof(E);  // bytes of one vector slot
    static constexpr int kVecBytes = STAGES * Q * BLOCK * kVB;
    static constexpr int kBytes = kVecBytes + STAGES * kEdges * BLOCK * 4;
    uint32_t base;  // shared-window address of the ring
    int tid;
    __device__ __forceinline__ uint32_t vec_slot(int stage, int i) const
    {
        return base + (uint32_t)(((stage * Q + i) * BLOCK + tid) * kVB);
    }
    __device__ __forceinline__ uint32_t edge_slot(int stage, int i) const
    {
        return base + (uint32_t)(kVecBytes + ((stage * kEdges + edge_index(i)) * BLOCK + tid) * 4);
    }
};

// the 4-byte aligned word that holds element e of a row
template <class E>
__device__ __forceinline__ const void* edge_word(const E* row, int e)
{
    if constexpr (sizeof(E) == 2)
        return row + (e & ~1);
    else
        return row + e;
}

// WRAP: every row lies within one warp and its lanes rotate (row_lane), so no edge word is copied.
template <class E, int VEC, int BLOCK, int STAGES, int FIX, bool WRAP = false, int I = 0>
__device__ __forceinline__ void async_issue_all(const E* base, const Geom& g, const RunLoc& p, int lane,
                                                const AsyncRing<E, VEC, BLOCK, STAGES>& ring, int stage)
{
    if constexpr (I < Q) {
        const int mode = FIX >= 0 ? FIX : p.mode;
        const bool shift = mode != 1;
        const int slot = mode == 2 ? Dir<I>::o : I;
        const int ry = shift ? g.wrap(p.y - Dir<I>::y) : p.y;
        const int rz = shift ? g.wrap(p.z - Dir<I>::z) : p.z;
        const E* row = base + (int64_t)slot * g.n + g.node(0, ry, rz);
        cp_async<AsyncRing<E, VEC, BLOCK, STAGES>::kVB>(ring.vec_slot(stage, I), row + p.x0);
        if constexpr (WRAP) {
        } else if constexpr (Dir<I>::x > 0) {
            if (shift && (lane == 0 || p.x0 == 0))
                cp_async<4>(ring.edge_slot(stage, I), edge_word(row, (p.x0 - 1) & (g.N - 1)));
        } else if constexpr (Dir<I>::x < 0) {
            if (shift && (lane == 31 || p.x0 + VEC == g.N))
                cp_async<4>(ring.edge_slot(stage, I), edge_word(row, (p.x0 + VEC) & (g.N - 1)));
        }
        async_issue_all<E, VEC, BLOCK, STAGES, FIX, WRAP, I + 1>(base, g, p, lane, ring, stage);
    }
}

// Read one population's run back from the ring.  CXI > 0: the edge is element x0 - 1,
// odd for FP16 (high half of its pair); CXI < 0: element x0 + VEC, even (low half).
template <class E, int VEC, int BLOCK, int STAGES, int CXI>
__device__ __forceinline__ RawRun<E, VEC> ring_read(const unsigned char* smem, int stage, int i, int tid)
{
    using Ring = AsyncRing<E, VEC, BLOCK, STAGES>;
    using R = typename RawOf<Ring::kVB>::type;
    RawRun<E, VEC> r;
    const R w = *reinterpret_cast<const R*>(smem + ((stage * Q + i) * BLOCK + tid) * Ring::kVB);
    memcpy(r.w, &w, sizeof(R));
    if constexpr (CXI != 0) {
        const unsigned int e = *reinterpret_cast<const unsigned int*>(
            smem + Ring::kVecBytes + ((stage * kEdges + edge_index(i)) * BLOCK + tid) * 4);
        if constexpr (sizeof(E) == 2) {
            const unsigned short h = CXI > 0 ? (unsigned short)(e >> 16) : (unsigned short)(e & 0xffffu);
            memcpy(&r.edge, &h, 2);
        } else {
            memcpy(&r.edge, &e, 4);
        }
    }
    return r;
}

template <class E, int VEC, int BLOCK, int STAGES, int FIX, bool WRAP = false, int I = 0>
__device__ __forceinline__ void async_finish_all(const unsigned char* smem, int stage, int tid, const Geom& g,
                                                 const RunLoc& p, int lane, typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (I < Q) {
        const int mode = FIX >= 0 ? FIX : p.mode;
        if (mode != 1) {
            const RawRun<E, VEC> r = ring_read<E, VEC, BLOCK, STAGES, WRAP ? 0 : Dir<I>::x>(smem, stage, I, tid);
            finish_row<E, VEC, Dir<I>::x, WRAP, FIX == 0>(r, p.x0, g.N, lane, v[I]);
        } else {
            const RawRun<E, VEC> r = ring_read<E, VEC, BLOCK, STAGES, 0>(smem, stage, I, tid);
            finish_row<E, VEC, 0>(r, p.x0, g.N, lane, v[I]);
        }
        async_finish_all<E, VEC, BLOCK, STAGES, FIX, WRAP, I + 1>(smem, stage, tid, g, p, lane, v);
    }
}

// FIX as in k_step_prefetch.  STAGES - 1 runs ahead are in flight; a thread's k-th run is
// read from stage k mod STAGES.  Every thread commits one copy group per run slot (empty
// past its last run), so wait_group STAGES - 1 always means "the current run has landed".
// ONE: a single-level launch (the level's arguments at a compile-time index; see locate).
template <class E, int VEC, int PATTERN, int BLOCK, int FIX, int STAGES, bool WRAP = false, bool ONE = false>
__global__ void __launch_bounds__(BLOCK) k_step_async(const BatchArgs<E> args)
{
    static_assert(Storage<E>::shifted, "the shared-memory prefetch variant serves the FP32 and FP16 storage");
    static_assert(sizeof(E) == 4 || VEC % 2 == 0, "FP16 runs must be whole 4-byte words");
    using C = typename Storage<E>::compute;
    using Ring = AsyncRing<E, VEC, BLOCK, STAGES>;
    // the D3Q19 FP16 AA even step of a multi-level launch collides with the intrinsic arithmetic
    // (the same bits; its schedule measured 86.7% -> 89.9% of the copy bandwidth at 128^3 x 32),
    // every other kernel with the assembly form, which measured faster for them (FP16 AA odd 81.2%
    // against 78.1%, FP32 pull 99.5% against 99.1%, the single-level FP16 even step 90.0% against
    // 87.5%)
    using Arith = std::conditional_t<Q == 19 && std::is_same<E, __half>::value && FIX == 1 && !ONE, lanes::Native,
                                     lanes::Asm>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int64_t total = args.prefix[args.nlev];
    const int64_t stride = (int64_t)gridDim.x * BLOCK;
    int64_t t = blockIdx.x * (int64_t)BLOCK + threadIdx.x;
    if (t >= total) return;  // whole warps: totals and strides are multiples of 32
    Ring ring;
    ring.base = (uint32_t)__cvta_generic_to_shared(smem);
    ring.tid = threadIdx.x;
    // runs t, t + stride, ... ; loc[s] is the run issued s slots after the current one
    RunLoc loc[STAGES - 1];
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        const int64_t ts = t + s * stride;
        if (ts < total) {
            loc[s] = locate<E, VEC, ONE>(args, ts, PATTERN);
            const LevelArgs<E>& L = args.lev[ONE ? 0 : loc[s].l];
            async_issue_all<E, VEC, BLOCK, STAGES, FIX, WRAP>(L.src + (int64_t)loc[s].m * Q * L.g.n, L.g, loc[s], lane,
                                                             ring, s);
        }
        cp_async_commit();
    }
    int stage = 0;
    for (;;) {
        const RunLoc cur = loc[0];
        const int64_t ta = t + (int64_t)(STAGES - 1) * stride;  // run to issue now
        RunLoc ahead = cur;
        if (ta < total) {
            ahead = locate<E, VEC, ONE>(args, ta, PATTERN);
            const LevelArgs<E>& La = args.lev[ONE ? 0 : ahead.l];
            int sa = stage + STAGES - 1;
            if (sa >= STAGES) sa -= STAGES;
            async_issue_all<E, VEC, BLOCK, STAGES, FIX, WRAP>(La.src + (int64_t)ahead.m * Q * La.g.n, La.g, ahead, lane,
                                                             ring, sa);
        }
        cp_async_commit();
        cp_async_wait<STAGES - 1>();
        const LevelArgs<E>& L = args.lev[ONE ? 0 : cur.l];
        const Geom g = L.g;
        C v[Q][VEC];
        async_finish_all<E, VEC, BLOCK, STAGES, FIX, WRAP>(smem, stage, threadIdx.x, g, cur, lane, v);
        collide_run<E, VEC, (VEC % 2 == 0), false, Arith>(v, L);
        E* base = L.dst + (int64_t)cur.m * Q * g.n;
        const int mode = FIX >= 0 ? FIX : cur.mode;
        if (mode == 0)
            scatter_all<E, VEC, 0>(base, g, cur.x0, cur.y, cur.z, lane, v);
        else if (mode == 1)
            store_own_opp<E, VEC>(base, g, cur.node, v);
        else
            scatter_all<E, VEC, 1, WRAP>(base, g, cur.x0, cur.y, cur.z, lane, v);
        t += stride;
        if (t >= total) break;
#pragma unroll
        for (int s = 0; s + 1 < STAGES - 1; ++s) loc[s] = loc[s + 1];
        loc[STAGES - 2] = ahead;
        stage = stage + 1 == STAGES ? 0 : stage + 1;
    }
    cp_async_wait<0>();  // nothing may stay in flight into a buffer that is released at exit
}

}  // namespace mclbm
