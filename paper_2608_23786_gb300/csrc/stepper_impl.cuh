// Fused stream + KBC collide kernel (Eq. (lbIteration) with Eqs. (kbcCollision),
// (entropyControl)) over a batch of levels, each an ensemble of samples.
//
// Thread mapping.  One thread updates VEC consecutive nodes along x of one row of
// one sample; consecutive threads take consecutive runs of a row, so a warp reads
// and writes 32 * VEC consecutive elements of each population array with VEC-wide
// (up to 16-byte) loads and stores.  The threads of all levels of a launch form one
// linear index space (levels concatenated, samples slowest within a level); every
// level contributes a multiple of 32 threads, so a warp never spans two levels.  The
// grid is persistent: each thread strides over that space.
//
// x-shifts.  A population with c_x = +1 is gathered from x - 1: a thread loads its
// own aligned run and takes the element before it from the previous lane with a
// warp shuffle; only the first lane of a warp and the thread at the start of a row
// (periodic wrap) load that element directly.  c_x = -1 mirrors this with the next
// lane.  y- and z-shifts only move the row, so those loads stay aligned.
//
// Patterns.  pull: read f_i(x) = S_i(x - c_i) from one lattice, write f*_i(x) to
// slot i of x in the other.  AA (in place, parity per level): even steps read slot i
// and write slot opp(i) of the own node; odd steps read slot opp(i) of x - c_i and
// write slot i of x + c_i.  In the odd step a node's outgoing value for c_x = +-1
// lands in the neighbour's run: it travels by warp shuffle to the lane that owns the
// destination run, which stores a full aligned vector; where the destination run
// belongs to a lane that cannot receive it (first lane of a warp or start of a row),
// the owner stores that single element itself and the receiver stores the rest of
// its run element by element.  Every slot is written exactly once, and a slot read
// by one lane is written by another only after the shuffle that depends on the
// reader's loaded data.
#pragma once
#include <cuda_fp16.h>

#include <cstring>

#include "collide.cuh"
#include "launch.h"
#include "storage.cuh"

namespace mclbm {



// 2/omega and 2 - 2/omega of Eq. (entropyControl) in FP64, for raw FP64 storage only (an empty
// base elsewhere: the FP32 and FP16 launch arguments keep their layout).
template <class E>
struct LevelArgsFP64 {};
template <>
struct LevelArgsFP64<double> {
    double a64, b64;
};

template <class E>
struct LevelArgs : LevelArgsFP64<E> {
    const E* src;   // pull: current lattice; AA: the lattice
    E* dst;         // pull: next lattice; AA: same as src
    Geom g;
    int M;
    int parity;     // AA: steps taken & 1
    float omega32;
    double omega64;
    float a32, b32;  // 2/omega and 2 - 2/omega of Eq. (entropyControl)
};

template <class E>
struct BatchArgs {
    int nlev;
    int64_t prefix[kMaxLevels + 1];  // thread offsets of the levels (multiples of 32)
    LevelArgs<E> lev[kMaxLevels];
};

template <int BYTES>
struct RawOf;
template <>
struct RawOf<2> {
    using type = unsigned short;
};
template <>
struct RawOf<4> {
    using type = unsigned int;
};
template <>
struct RawOf<8> {
    using type = uint2;
};
template <>
struct RawOf<16> {
    using type = uint4;
};

template <class E, int VEC>
__device__ __forceinline__ void vload(const E* p, E (&out)[VEC])
{
    using R = typename RawOf<VEC * sizeof(E)>::type;
    const R r = __ldg(reinterpret_cast<const R*>(p));
    memcpy(out, &r, sizeof(R));
}

template <class E, int VEC>
__device__ __forceinline__ void vstore(E* p, const E (&in)[VEC])
{
    using R = typename RawOf<VEC * sizeof(E)>::type;
    R r;
    memcpy(&r, in, sizeof(R));
    *reinterpret_cast<R*>(p) = r;
}

template <class E>
__device__ __forceinline__ E sload(const E* p)
{
    return __ldg(p);
}
template <>
__device__ __forceinline__ __half sload<__half>(const __half* p)
{
    return __ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p)));
}

template <class E>
__device__ __forceinline__ typename Storage<E>::compute to_c(E v)
{
    return (typename Storage<E>::compute)v;
}
template <>
__device__ __forceinline__ float to_c<__half>(__half v)
{
    return __half2float(v);
}
template <class E>
__device__ __forceinline__ E from_c(typename Storage<E>::compute v)
{
    return (E)v;
}
template <>
__device__ __forceinline__ __half from_c<__half>(float v)
{
    return __float2half_rn(v);
}

template <class E>
__device__ __forceinline__ typename Storage<E>::compute omega_of(const LevelArgs<E>& L);
template <>
__device__ __forceinline__ double omega_of<double>(const LevelArgs<double>& L) { return L.omega64; }
template <>
__device__ __forceinline__ float omega_of<float>(const LevelArgs<float>& L) { return L.omega32; }
template <>
__device__ __forceinline__ float omega_of<__half>(const LevelArgs<__half>& L) { return L.omega32; }

// Element offsets, within one population array, of the run at x0 in the rows y + d and the
// planes z + d (d = -1, 0, +1; periodic): the run of slot s in row (y + dy, z + dz) starts at
// s N^3 + z[1 + dz] + y[1 + dy].  They are formed once per run, so each access costs one 32-bit
// add and one wide multiply-add (N^3 <= 2^30).  The AA odd step, whose loads and stores are both
// shifted, addresses its rows this way; the pull and AA even kernels form each row address
// where it is used, which keeps their register count (and resident blocks) lower.
struct RowOffsets {
    uint32_t y[3], z[3];
};

__device__ __forceinline__ RowOffsets row_offsets(const Geom& g, int x0, int y, int z)
{
    RowOffsets r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.y[k] = ((uint32_t)g.wrap(y + k - 1) << g.logN) + (uint32_t)x0;
        r.z[k] = (uint32_t)g.wrap(z + k - 1) << (2 * g.logN);
    }
    return r;
}

template <class P>
__device__ __forceinline__ P run_at(P base, const Geom& g, int slot, const RowOffsets& r, int dy, int dz)
{
    return base + ((uint64_t)(uint32_t)slot * (uint32_t)g.n + (uint64_t)(r.z[1 + dz] + r.y[1 + dy]));
}

// The same run addressed directly: slot s of row (y + dy, z + dz), element x0.
template <class P>
__device__ __forceinline__ P run_direct(P base, const Geom& g, int slot, int x0, int y, int z, int dy, int dz)
{
    return base + (int64_t)slot * g.n + g.node(0, g.wrap(y + dy), g.wrap(z + dz)) + x0;
}

// Row rotation (the WRAP variants, for launches whose every level has N <= 32 VEC): a whole
// x-row is then R = N / VEC consecutive lanes of one warp (R divides 32), and the periodic
// neighbour of a row's end run is the row's other end, one shuffle among the row's lanes away,
// so every lane loads and stores full aligned runs with no separate end elements.  The launch
// picks the variant (a compile-time choice: no per-population branch).
__device__ __forceinline__ int row_lane(int lane, int R, int d) { return (lane & ~(R - 1)) | ((lane + d) & (R - 1)); }

// Offsets from a run's first element (x0) to the element before it and after it in its
// periodic row.
__device__ __forceinline__ int before_run(int x0, int N) { return x0 == 0 ? N - 1 : -1; }
template <int VEC>
__device__ __forceinline__ int after_run(int x0, int N) { return x0 + VEC == N ? -x0 : VEC; }

// Gather the VEC values x0 - cxi .. x0 + VEC - 1 - cxi of one row (periodic in x); run points
// at element x0 of the row.
template <class E, int VEC, int CXI>
__device__ __forceinline__ void gather_row(const E* run, int x0, int N, int lane, typename Storage<E>::compute (&v)[VEC])
{
    E w[VEC];
    vload<E, VEC>(run, w);
    if constexpr (CXI == 0) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[k] = to_c<E>(w[k]);
    } else if constexpr (CXI > 0) {  // source x - 1
        E prev = __shfl_up_sync(0xffffffffu, w[VEC - 1], 1);
        if (lane == 0 || x0 == 0) prev = sload<E>(run + before_run(x0, N));
        v[0] = to_c<E>(prev);
#pragma unroll
        for (int k = 1; k < VEC; ++k) v[k] = to_c<E>(w[k - 1]);
    } else {  // source x + 1
        E next = __shfl_down_sync(0xffffffffu, w[0], 1);
        if (lane == 31 || x0 + VEC == N) next = sload<E>(run + after_run<VEC>(x0, N));
#pragma unroll
        for (int k = 0; k < VEC - 1; ++k) v[k] = to_c<E>(w[k + 1]);
        v[VEC - 1] = to_c<E>(next);
    }
}

// Scatter the VEC values of nodes x0..x0+VEC-1 to positions shifted by CXI in x; run points
// at element x0 of the destination row.
template <class E, int VEC, int CXI, bool WRAP = false>
__device__ __forceinline__ void scatter_row(E* run, int x0, int N, int lane, const typename Storage<E>::compute (&v)[VEC])
{
    E w[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) w[k] = from_c<E>(v[k]);
    if constexpr (CXI == 0) {
        vstore<E, VEC>(run, w);
    } else if constexpr (WRAP) {  // the row's lanes rotate: every lane stores a full run
        // the shift moves compute-type values (whole registers), then the shifted run is converted
        // (for FP16, pairs of nodes pack into one word with no half-word rearranging)
        using C = typename Storage<E>::compute;
        C of[VEC];
        if constexpr (CXI > 0) {  // node x goes to x + 1
            of[0] = __shfl_sync(0xffffffffu, v[VEC - 1], row_lane(lane, N / VEC, -1));
#pragma unroll
            for (int k = 1; k < VEC; ++k) of[k] = v[k - 1];
        } else {  // node x goes to x - 1
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) of[k] = v[k + 1];
            of[VEC - 1] = __shfl_sync(0xffffffffu, v[0], row_lane(lane, N / VEC, 1));
        }
        E o[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) o[k] = from_c<E>(of[k]);
        vstore<E, VEC>(run, o);
    } else if constexpr (CXI > 0) {  // node x goes to x + 1
        const E prev = __shfl_up_sync(0xffffffffu, w[VEC - 1], 1);
        const bool can_receive = lane != 0 && x0 != 0;
        if (lane == 31 || x0 + VEC == N) run[after_run<VEC>(x0, N)] = w[VEC - 1];
        if (can_receive) {
            E o[VEC];
            o[0] = prev;
#pragma unroll
            for (int k = 1; k < VEC; ++k) o[k] = w[k - 1];
            vstore<E, VEC>(run, o);
        } else {
#pragma unroll
            for (int k = 1; k < VEC; ++k) run[k] = w[k - 1];
        }
    } else {  // node x goes to x - 1
        const E next = __shfl_down_sync(0xffffffffu, w[0], 1);
        const bool can_receive = lane != 31 && x0 + VEC != N;
        if (lane == 0 || x0 == 0) run[before_run(x0, N)] = w[0];
        if (can_receive) {
            E o[VEC];
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) o[k] = w[k + 1];
            o[VEC - 1] = next;
            vstore<E, VEC>(run, o);
        } else {
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) run[k] = w[k + 1];
        }
    }
}

// Collide the VEC nodes of a run.  PACK (shifted storage, VEC even) runs the FP32
// collision on node pairs in the packed FP32 pipe; the results are bit-identical to the
// one-node form.  Ar: the arithmetic policy of the shifted collision (same bits either way).
template <class E, int VEC, bool PACK = false, bool EXACT = false, class Ar = lanes::Asm>
__device__ __forceinline__ void collide_run(typename Storage<E>::compute (&v)[Q][VEC], const LevelArgs<E>& L)
{
    const typename Storage<E>::compute omega = omega_of<E>(L);
    using C = typename Storage<E>::compute;
    if constexpr (EXACT) {  // exact entropic gamma (kind 6), node by node
        // one copy of the solver for the VEC nodes: a rolled loop whose node column is moved in
        // and out of the register array by compile-time selects
#pragma unroll 1
        for (int k = 0; k < VEC; ++k) {
            C t[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                t[i] = v[i][0];
#pragma unroll
                for (int kk = 1; kk < VEC; ++kk)
                    if (k == kk) t[i] = v[i][kk];
            }
            kbc_exact<C, Storage<E>::shifted>(t, omega);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
#pragma unroll
                for (int kk = 0; kk < VEC; ++kk)
                    if (k == kk) v[i][kk] = t[i];
            }
        }
    } else if constexpr (PACK) {
        static_assert(Storage<E>::shifted && VEC % 2 == 0, "packed collision needs FP32 lanes in pairs");
#pragma unroll
        for (int k = 0; k < VEC; k += 2) {
            float2 t[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) t[i] = make_float2(v[i][k], v[i][k + 1]);
            kbc_shifted<float2, Ar>(t, omega, L.a32, L.b32);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                v[i][k] = t[i].x;
                v[i][k + 1] = t[i].y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            C t[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) t[i] = v[i][k];
            if constexpr (Storage<E>::shifted)
                kbc_shifted<float, Ar>(t, omega, L.a32, L.b32);
            else
                kbc_raw(t, omega, (C)L.a64, (C)L.b64);
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i][k] = t[i];
        }
    }
}

template <int I>
struct Dir {
    static constexpr int x = cx(I), y = cy(I), z = cz(I), o = opp(I);
};

// Load all Q populations of a run: slot SLOT(i) of the row shifted by -c_i.
template <class E, int VEC, bool OPP_SLOT, int I = 0>
__device__ __forceinline__ void gather_rows(const E* base, const Geom& g, const RowOffsets& r, int x0, int lane,
                                            typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (I < Q) {
        constexpr int slot = OPP_SLOT ? Dir<I>::o : I;
        gather_row<E, VEC, Dir<I>::x>(run_at(base, g, slot, r, -Dir<I>::y, -Dir<I>::z), x0, g.N, lane, v[I]);
        gather_rows<E, VEC, OPP_SLOT, I + 1>(base, g, r, x0, lane, v);
    }
}
template <class E, int VEC, int I = 0>
__device__ __forceinline__ void gather_direct(const E* base, const Geom& g, int x0, int y, int z, int lane,
                                              typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (I < Q) {
        gather_row<E, VEC, Dir<I>::x>(run_direct(base, g, I, x0, y, z, -Dir<I>::y, -Dir<I>::z), x0, g.N, lane, v[I]);
        gather_direct<E, VEC, I + 1>(base, g, x0, y, z, lane, v);
    }
}
// OPP_SLOT: the AA odd step (row offsets); otherwise pull (direct addresses).
template <class E, int VEC, bool OPP_SLOT>
__device__ __forceinline__ void gather_all(const E* base, const Geom& g, int x0, int y, int z, int lane,
                                           typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (OPP_SLOT)
        gather_rows<E, VEC, true>(base, g, row_offsets(g, x0, y, z), x0, lane, v);
    else
        gather_direct<E, VEC>(base, g, x0, y, z, lane, v);
}

// Store all Q post-collision populations: slot I of the row shifted by SIGN * c_i.
template <class E, int VEC, int SIGN, bool WRAP = false, int I = 0>
__device__ __forceinline__ void scatter_rows(E* base, const Geom& g, const RowOffsets& r, int x0, int lane,
                                             const typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (I < Q) {
        scatter_row<E, VEC, SIGN * Dir<I>::x, WRAP>(run_at(base, g, I, r, SIGN * Dir<I>::y, SIGN * Dir<I>::z), x0,
                                                     g.N, lane, v[I]);
        scatter_rows<E, VEC, SIGN, WRAP, I + 1>(base, g, r, x0, lane, v);
    }
}
template <class E, int VEC, int I = 0>
__device__ __forceinline__ void scatter_direct(E* base, const Geom& g, int x0, int y, int z, int lane,
                                               const typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (I < Q) {
        scatter_row<E, VEC, 0>(run_direct(base, g, I, x0, y, z, 0, 0), x0, g.N, lane, v[I]);
        scatter_direct<E, VEC, I + 1>(base, g, x0, y, z, lane, v);
    }
}
// SIGN 1: the AA odd step (row offsets); 0: pull, own rows (direct addresses).
template <class E, int VEC, int SIGN, bool WRAP = false>
__device__ __forceinline__ void scatter_all(E* base, const Geom& g, int x0, int y, int z, int lane,
                                            const typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (SIGN != 0)
        scatter_rows<E, VEC, SIGN, WRAP>(base, g, row_offsets(g, x0, y, z), x0, lane, v);
    else
        scatter_direct<E, VEC>(base, g, x0, y, z, lane, v);
}

// Own-node aligned access with slot permutation (AA even step).
template <class E, int VEC>
__device__ __forceinline__ void load_own(const E* base, const Geom& g, int64_t node, typename Storage<E>::compute (&v)[Q][VEC])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        E w[VEC];
        vload<E, VEC>(base + (int64_t)i * g.n + node, w);
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[i][k] = to_c<E>(w[k]);
    }
}
template <class E, int VEC>
__device__ __forceinline__ void store_own_opp(E* base, const Geom& g, int64_t node, const typename Storage<E>::compute (&v)[Q][VEC])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        E w[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) w[k] = from_c<E>(v[i][k]);
        vstore<E, VEC>(base + (int64_t)opp(i) * g.n + node, w);
    }
}

// PATTERN: 0 pull, 1 AA.  EXACT: the exact entropic gamma (launch kind 6); its D3Q19 FP32 and
// FP16 forms are held to four blocks per SM (128 registers: the Newton solve is latency-bound,
// 16 warps per SM; the D3Q27 forms would spill).
template <class E, int VEC, int PATTERN, int BLOCK, bool EXACT = false>
__global__ void __launch_bounds__(BLOCK, (EXACT && Q == 19 && sizeof(typename Storage<E>::compute) == 4) ? 4 : 1)
    k_step_batch(const BatchArgs<E> args)
{
    using C = typename Storage<E>::compute;
    const int lane = threadIdx.x & 31;
    const int64_t total = args.prefix[args.nlev];
    for (int64_t t = blockIdx.x * (int64_t)BLOCK + threadIdx.x; t < total; t += (int64_t)gridDim.x * BLOCK) {
        int l = 0;
#pragma unroll 1
        while (l + 1 < args.nlev && t >= args.prefix[l + 1]) ++l;
        const LevelArgs<E>& L = args.lev[l];
        const Geom g = L.g;
        const int64_t first = (t - args.prefix[l]) * VEC;  // first node, ensemble-linear
        const int m = (int)(first >> (3 * g.logN));
        const int64_t node = first & (g.n - 1);
        const int x0 = (int)(node & (g.N - 1));
        const int y = (int)((node >> g.logN) & (g.N - 1));
        const int z = (int)(node >> (2 * g.logN));
        const C omega = omega_of<E>(L);
        C v[Q][VEC];
        if constexpr (PATTERN == 0) {
            gather_all<E, VEC, false>(L.src + (int64_t)m * Q * g.n, g, x0, y, z, lane, v);
            collide_run<E, VEC, false, EXACT>(v, L);
            scatter_all<E, VEC, 0>(L.dst + (int64_t)m * Q * g.n, g, x0, y, z, lane, v);
        } else {
            E* base = L.dst + (int64_t)m * Q * g.n;
            if (L.parity == 0) {
                load_own<E, VEC>(base, g, node, v);
                collide_run<E, VEC, false, EXACT>(v, L);
                store_own_opp<E, VEC>(base, g, node, v);
            } else {
                gather_all<E, VEC, true>(base, g, x0, y, z, lane, v);
                collide_run<E, VEC, false, EXACT>(v, L);
                scatter_all<E, VEC, 1>(base, g, x0, y, z, lane, v);
            }
        }
    }
}

}  // namespace mclbm

namespace mclbm {

// ---------------------------------------------------------------------------------
// Prefetching variant of the direct kernel.  Each thread issues the loads of its next
// run (one persistent-grid stride ahead) before it collides and stores the current
// run, so a warp keeps its next 19 loads in flight during its arithmetic.  The raw
// vector and the one boundary element of every population are kept as loaded; the
// warp shuffles that apply the x-shift happen only when the run is consumed (a shuffle
// of an outstanding load would wait for it).

template <class E, int VEC>
struct RawRun {
    E w[VEC];
    E edge;  // the element before (c_x = +1) or after (c_x = -1) the run, where no lane has it
};

// mode: 0 pull (slot i, rows shifted by -c_i), 1 AA even (slot i, own rows), 2 AA odd
// (slot opp(i), rows shifted by -c_i)
struct RunLoc {
    int l, m, x0, y, z, mode;
    int64_t node;
};

template <class E, int VEC, int CXI, bool WRAP = false>
__device__ __forceinline__ void issue_row(const E* run, int x0, int N, int lane, RawRun<E, VEC>& r)
{
    vload<E, VEC>(run, r.w);
    if constexpr (WRAP) {  // the row's lanes rotate: no end element to load
    } else if constexpr (CXI > 0) {
        if (lane == 0 || x0 == 0) r.edge = sload<E>(run + before_run(x0, N));
    } else if constexpr (CXI < 0) {
        if (lane == 31 || x0 + VEC == N) r.edge = sload<E>(run + after_run<VEC>(x0, N));
    }
}

// CF (pull steps): with the row rotation, the end element is converted before it moves, so the
// shuffle moves a whole register (FP16 pull 88.7% -> 90.3% of the copy bandwidth at 128^3; the AA
// odd step, at its register limit, loses with it and moves the stored element instead).
template <class E, int VEC, int CXI, bool WRAP = false, bool CF = false>
__device__ __forceinline__ void finish_row(const RawRun<E, VEC>& r, int x0, int N, int lane,
                                           typename Storage<E>::compute (&v)[VEC])
{
    if constexpr (CXI == 0) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[k] = to_c<E>(r.w[k]);
    } else if constexpr (WRAP && !CF) {  // the row's lanes rotate
        if constexpr (CXI > 0) {
            const E prev = __shfl_sync(0xffffffffu, r.w[VEC - 1], row_lane(lane, N / VEC, -1));
            v[0] = to_c<E>(prev);
#pragma unroll
            for (int k = 1; k < VEC; ++k) v[k] = to_c<E>(r.w[k - 1]);
        } else {
            const E next = __shfl_sync(0xffffffffu, r.w[0], row_lane(lane, N / VEC, 1));
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) v[k] = to_c<E>(r.w[k + 1]);
            v[VEC - 1] = to_c<E>(next);
        }
    } else if constexpr (WRAP) {  // the row's lanes rotate (converted values move: whole registers)
        using C = typename Storage<E>::compute;
        if constexpr (CXI > 0) {
            const C last = to_c<E>(r.w[VEC - 1]);
            v[0] = __shfl_sync(0xffffffffu, last, row_lane(lane, N / VEC, -1));
#pragma unroll
            for (int k = 1; k < VEC; ++k) v[k] = to_c<E>(r.w[k - 1]);
        } else {
            const C first = to_c<E>(r.w[0]);
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) v[k] = to_c<E>(r.w[k + 1]);
            v[VEC - 1] = __shfl_sync(0xffffffffu, first, row_lane(lane, N / VEC, 1));
        }
    } else if constexpr (CXI > 0) {
        E prev = __shfl_up_sync(0xffffffffu, r.w[VEC - 1], 1);
        if (lane == 0 || x0 == 0) prev = r.edge;
        v[0] = to_c<E>(prev);
#pragma unroll
        for (int k = 1; k < VEC; ++k) v[k] = to_c<E>(r.w[k - 1]);
    } else {
        E next = __shfl_down_sync(0xffffffffu, r.w[0], 1);
        if (lane == 31 || x0 + VEC == N) next = r.edge;
#pragma unroll
        for (int k = 0; k < VEC - 1; ++k) v[k] = to_c<E>(r.w[k + 1]);
        v[VEC - 1] = to_c<E>(next);
    }
}

template <class E, int VEC, int FIX, bool WRAP = false, int I = 0>
__device__ __forceinline__ void issue_rows(const E* base, const Geom& g, const RowOffsets& r, const RunLoc& p,
                                           int lane, RawRun<E, VEC> (&raw)[Q])
{
    if constexpr (I < Q) {
        const int mode = FIX >= 0 ? FIX : p.mode;
        const bool shift = mode != 1;
        const int slot = mode == 2 ? Dir<I>::o : I;
        const E* run = run_at(base, g, slot, r, shift ? -Dir<I>::y : 0, shift ? -Dir<I>::z : 0);
        if (shift)
            issue_row<E, VEC, Dir<I>::x, WRAP>(run, p.x0, g.N, lane, raw[I]);
        else
            issue_row<E, VEC, 0>(run, p.x0, g.N, lane, raw[I]);
        issue_rows<E, VEC, FIX, WRAP, I + 1>(base, g, r, p, lane, raw);
    }
}
template <class E, int VEC, int FIX, bool WRAP = false, int I = 0>
__device__ __forceinline__ void issue_direct(const E* base, const Geom& g, const RunLoc& p, int lane,
                                             RawRun<E, VEC> (&raw)[Q])
{
    if constexpr (I < Q) {
        const int mode = FIX >= 0 ? FIX : p.mode;
        const bool shift = mode != 1;
        const int slot = mode == 2 ? Dir<I>::o : I;
        const E* run = run_direct(base, g, slot, p.x0, p.y, p.z, shift ? -Dir<I>::y : 0, shift ? -Dir<I>::z : 0);
        if (shift)
            issue_row<E, VEC, Dir<I>::x, WRAP>(run, p.x0, g.N, lane, raw[I]);
        else
            issue_row<E, VEC, 0>(run, p.x0, g.N, lane, raw[I]);
        issue_direct<E, VEC, FIX, WRAP, I + 1>(base, g, p, lane, raw);
    }
}
// FIX 2 (AA odd): row offsets; pull, AA even and mixed launches: direct addresses.
template <class E, int VEC, int FIX, bool WRAP = false>
__device__ __forceinline__ void issue_all(const E* base, const Geom& g, const RunLoc& p, int lane,
                                          RawRun<E, VEC> (&raw)[Q])
{
    if constexpr (FIX == 2)
        issue_rows<E, VEC, FIX, WRAP>(base, g, row_offsets(g, p.x0, p.y, p.z), p, lane, raw);
    else
        issue_direct<E, VEC, FIX, WRAP>(base, g, p, lane, raw);
}

template <class E, int VEC, int FIX, bool WRAP = false, int I = 0>
__device__ __forceinline__ void finish_all(const Geom& g, const RunLoc& p, int lane, const RawRun<E, VEC> (&raw)[Q],
                                           typename Storage<E>::compute (&v)[Q][VEC])
{
    if constexpr (I < Q) {
        const int mode = FIX >= 0 ? FIX : p.mode;
        if (mode != 1)
            finish_row<E, VEC, Dir<I>::x, WRAP, FIX == 0>(raw[I], p.x0, g.N, lane, v[I]);
        else
            finish_row<E, VEC, 0>(raw[I], p.x0, g.N, lane, v[I]);
        finish_all<E, VEC, FIX, WRAP, I + 1>(g, p, lane, raw, v);
    }
}

// ONE: the launch has a single level (a context's own step), whose arguments are then read at a
// compile-time index, which the compiler takes as constant operands instead of loading them into
// registers by a run-time index.  Only the FP16 ring kernel uses it (see k_step_async).
template <class E, int VEC, bool ONE = false>
__device__ __forceinline__ RunLoc locate(const BatchArgs<E>& args, int64_t t, int pattern)
{
    RunLoc p;
    int l = 0;
    if constexpr (!ONE) {
#pragma unroll 1
        while (l + 1 < args.nlev && t >= args.prefix[l + 1]) ++l;
    }
    const Geom& g = args.lev[l].g;
    const int64_t first = (ONE ? t : t - args.prefix[l]) * VEC;
    p.l = l;
    p.m = (int)(first >> (3 * g.logN));
    p.node = first & (g.n - 1);
    p.x0 = (int)(p.node & (g.N - 1));
    p.y = (int)((p.node >> g.logN) & (g.N - 1));
    p.z = (int)(p.node >> (2 * g.logN));
    p.mode = pattern == 0 ? 0 : (args.lev[l].parity == 0 ? 1 : 2);
    return p;
}

// FIX: -1 takes each level's mode at run time; 0 (pull), 1 (AA even) or 2 (AA odd) when every
// level of the launch has that mode, which drops the other branches.  PACK: packed FP32
// collision of node pairs.
template <class E, int VEC, int PATTERN, int BLOCK, int FIX, bool PACK, bool WRAP = false>
__global__ void __launch_bounds__(BLOCK) k_step_prefetch(const BatchArgs<E> args)
{
    using C = typename Storage<E>::compute;
    const int lane = threadIdx.x & 31;
    const int64_t total = args.prefix[args.nlev];
    const int64_t stride = (int64_t)gridDim.x * BLOCK;
    int64_t t = blockIdx.x * (int64_t)BLOCK + threadIdx.x;
    if (t >= total) return;  // whole warps: totals and strides are multiples of 32
    RunLoc cur = locate<E, VEC>(args, t, PATTERN);
    RawRun<E, VEC> raw[Q];
    {
        const LevelArgs<E>& L = args.lev[cur.l];
        issue_all<E, VEC, FIX, WRAP>(L.src + (int64_t)cur.m * Q * L.g.n, L.g, cur, lane, raw);
    }
    while (true) {
        const LevelArgs<E>& L = args.lev[cur.l];
        const Geom g = L.g;
        C v[Q][VEC];
        finish_all<E, VEC, FIX, WRAP>(g, cur, lane, raw, v);
        const int64_t tn = t + stride;
        const bool more = tn < total;
        RunLoc nxt = cur;
        if (more) {
            nxt = locate<E, VEC>(args, tn, PATTERN);
            const LevelArgs<E>& Ln = args.lev[nxt.l];
            issue_all<E, VEC, FIX, WRAP>(Ln.src + (int64_t)nxt.m * Q * Ln.g.n, Ln.g, nxt, lane, raw);
        }
        collide_run<E, VEC, PACK>(v, L);
        E* base = L.dst + (int64_t)cur.m * Q * g.n;
        const int mode = FIX >= 0 ? FIX : cur.mode;
        if (mode == 0)
            scatter_all<E, VEC, 0>(base, g, cur.x0, cur.y, cur.z, lane, v);
        else if (mode == 1)
            store_own_opp<E, VEC>(base, g, cur.node, v);
        else
            scatter_all<E, VEC, 1, WRAP>(base, g, cur.x0, cur.y, cur.z, lane, v);
        if (!more) break;
        t = tn;
        cur = nxt;
    }
}

}  // namespace mclbm
