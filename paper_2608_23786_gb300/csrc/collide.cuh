// KBC collision of one node (Sec. "Entropic multi-relaxation lattice Boltzmann
// scheme", Eqs. (equilibrium), (kbcCollision), (entropyControl)), in two forms:
//
//  kbc_raw      - raw populations f_i, the plain method (used in FP64);
//  kbc_shifted  - normalised deviations h_i = f_i / w_i - 1 (Assumption "Uniform
//                 low Mach regime" (i): f = w (1 + eps g)), used for the FP32 and
//                 FP16 storage with FP32 arithmetic.  Working on h removes the
//                 cancellation of f - f^eq around f ~ w.
//
// The shear part Ds carries exactly the deviatoric raw second moments
// D_ab = P_ab - delta_ab tr(P)/3 of f^neq (tensors N and Pi of Table
// "frequencySummary"): Ds = D_aa / 2 on the faces +-e_a, s l P_ab / 4 on the
// edge s e_a + l e_b, 0 at rest.  Dh = f^neq - Ds holds the remaining (T, Q, A)
// moments.  gamma = 2/omega - (2 - 2/omega) <Ds|Dh>/<Dh|Dh> with
// <X|Y> = sum X_i Y_i / f^eq_i; gamma = 2 (BGK) where <Dh|Dh> vanishes.
#pragma once
#include <type_traits>

#include "lattice.cuh"

namespace mclbm {

// Signed sum over the populations: sum_i s(i) v_i with s(i) a compile-time
// sign in {-1, 0, 1}; the zero terms are dropped at compile time.
#define MCLBM_SIGNED_ADD(acc, sgn, v) \
    do {                              \
        if ((sgn) > 0) acc += (v);    \
        else if ((sgn) < 0) acc -= (v); \
    } while (0)

// Velocities i = 2p + 1 and 2p + 2 are opposite (the library order).
constexpr bool opposite_pairs_adjacent()
{
    for (int i = 1; i < Q; i += 2)
        if (opp(i) != i + 1) return false;
    return true;
}
static_assert(opposite_pairs_adjacent(), "kbc_raw pairs velocity 2p + 1 with its opposite 2p + 2");

// Plain KBC on raw populations (in place).  Returns gamma.  a = 2/omega and b = 2 - 2/omega
// are passed in (formed once on the host).  Divisions are the costly FP64 operations here: 1/rho
// is formed once, the 1/f^eq of an opposite pair come from one reciprocal of their product
// (1/f^eq_i = f^eq_j / (f^eq_i f^eq_j)), and tr(P)/3 is a product with 1/3: 1 + 1 + (Q - 1)/2
// + 1 divisions per node (12 for D3Q19) instead of 45.
template <class T>
__host__ __device__ __forceinline__ T kbc_raw(T (&f)[Q], T omega, T a, T b)
{
    T rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        MCLBM_SIGNED_ADD(jx, cx(i), f[i]);
        MCLBM_SIGNED_ADD(jy, cy(i), f[i]);
        MCLBM_SIGNED_ADD(jz, cz(i), f[i]);
    }
    const T rinv = T(1) / rho;
    const T ux = jx * rinv, uy = jy * rinv, uz = jz * rinv;
    const T uu = ux * ux + uy * uy + uz * uz;
    T feq[Q], fneq[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T cu = 0;
        MCLBM_SIGNED_ADD(cu, cx(i), ux);
        MCLBM_SIGNED_ADD(cu, cy(i), uy);
        MCLBM_SIGNED_ADD(cu, cz(i), uz);
        feq[i] = rho * weight<T>(i) * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        fneq[i] = f[i] - feq[i];
    }
    // raw second moments of f^neq
    T pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (cx(i) != 0) pxx += fneq[i];
        if (cy(i) != 0) pyy += fneq[i];
        if (cz(i) != 0) pzz += fneq[i];
        MCLBM_SIGNED_ADD(pxy, cx(i) * cy(i), fneq[i]);
        MCLBM_SIGNED_ADD(pxz, cx(i) * cz(i), fneq[i]);
        MCLBM_SIGNED_ADD(pyz, cy(i) * cz(i), fneq[i]);
    }
    const T tr3 = (pxx + pyy + pzz) * (T(1) / T(3));
    T ds[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int n2 = norm2(i);
        if (n2 == 0 || n2 == 3) ds[i] = 0;  // rest and (D3Q27) corners carry no shear
        else if (n2 == 1) ds[i] = T(0.5) * ((cx(i) ? pxx : (cy(i) ? pyy : pzz)) - tr3);
        else {
            const T p = (cz(i) == 0) ? pxy : ((cy(i) == 0) ? pxz : pyz);
            const int s = (cz(i) == 0) ? cx(i) * cy(i) : ((cy(i) == 0) ? cx(i) * cz(i) : cy(i) * cz(i));
            ds[i] = s > 0 ? T(0.25) * p : -T(0.25) * p;
        }
    }
    T sh = 0, hh = 0;
    {
        const T dh = fneq[0] - ds[0];
        const T dhw = dh * (T(1) / feq[0]);
        sh += ds[0] * dhw;
        hh += dh * dhw;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {  // opposite pair (i, i + 1): one division
        const T r = T(1) / (feq[i] * feq[i + 1]);
        const T dh0 = fneq[i] - ds[i], dh1 = fneq[i + 1] - ds[i + 1];
        const T dhw0 = dh0 * (feq[i + 1] * r), dhw1 = dh1 * (feq[i] * r);
        sh += ds[i] * dhw0;
        hh += dh0 * dhw0;
        sh += ds[i + 1] * dhw1;
        hh += dh1 * dhw1;
    }
    const T gamma = (hh == T(0)) ? T(2) : a - b * sh / hh;
    const T bo = T(0.5) * omega * gamma;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T dh = fneq[i] - ds[i];
        f[i] = f[i] - omega * ds[i] - bo * dh;
    }
    return gamma;
}

// Guard of <Dh|Dh> in the FP32 shifted form (values are f/w-normalised; below
// this the higher-order non-equilibrium is at rounding level).
constexpr float kHHGuard = 1e-30f;

// Lane arithmetic of the FP32 shifted collision.  A lane type V is float (one node) or
// float2 (two nodes in the packed FP32 pipe of sm_100+: one add, multiply or fma
// instruction serves both).  Every operation rounds once to nearest, with no contraction
// left to the compiler, so a node gets bit-identical results in either lane type.
namespace lanes {
template <class V>
__device__ __forceinline__ V bc(float s);
template <>
__device__ __forceinline__ float bc<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 bc<float2>(float s) { return make_float2(s, s); }
// Both lane types are written in PTX with the rounding mode spelled out: an add or multiply
// with an explicit rounding modifier is never fused with a neighbour into an fma, and no
// compiler pass above the assembler rewrites them, which keeps the two lane types
// bit-identical.
__device__ __forceinline__ float add(float a, float b)
{
    float d;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float mul(float a, float b)
{
    float d;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float fma(float a, float b, float c)
{
    float d;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// a - b = a + (-1) b, rounded once (the same form as the packed subtraction)
__device__ __forceinline__ float sub(float a, float b) { return fma(b, -1.f, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%6, %7};\n\tfma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
// a - b = a + (-1) b, rounded once: the same value as the scalar subtraction
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return fma(b, make_float2(-1.f, -1.f), a); }
// Hardware reciprocal approximation (rcp.approx, within one ulp; subnormals flushed).  The
// arguments here are 1 + O(Ma) densities and equilibria, and <Dh|Dh> above its guard.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// lane-wise scalar function
template <class F>
__device__ __forceinline__ float map(float a, F f) { return f(a); }
template <class F>
__device__ __forceinline__ float2 map(float2 a, F f) { return make_float2(f(a.x), f(a.y)); }
template <class F>
__device__ __forceinline__ float map(float a, float b, F f) { return f(a, b); }
template <class F>
__device__ __forceinline__ float2 map(float2 a, float2 b, F f) { return make_float2(f(a.x, b.x), f(a.y, b.y)); }

// The arithmetic of a collision as a policy: Asm, the PTX forms above; Native, the
// round-to-nearest intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn and the packed __fadd2_rn,
// __fmul2_rn, __ffma2_rn of sm_100+), which round the same way and are never contracted either,
// so both give the same bits.  They differ only in what the compiler sees (opaque assembly or the
// operations themselves), hence in its register allocation and instruction schedule; the stepper
// takes the one measured faster for each kernel.
struct Asm {
    template <class V>
    static __device__ __forceinline__ V add(V x, V y) { return lanes::add(x, y); }
    template <class V>
    static __device__ __forceinline__ V mul(V x, V y) { return lanes::mul(x, y); }
    template <class V>
    static __device__ __forceinline__ V fma(V x, V y, V z) { return lanes::fma(x, y, z); }
    template <class V>
    static __device__ __forceinline__ V sub(V x, V y) { return lanes::sub(x, y); }
};
struct Native {
    static __device__ __forceinline__ float add(float x, float y) { return __fadd_rn(x, y); }
    static __device__ __forceinline__ float mul(float x, float y) { return __fmul_rn(x, y); }
    static __device__ __forceinline__ float fma(float x, float y, float z) { return __fmaf_rn(x, y, z); }
    static __device__ __forceinline__ float sub(float x, float y) { return __fmaf_rn(y, -1.f, x); }
    static __device__ __forceinline__ float2 add(float2 x, float2 y) { return __fadd2_rn(x, y); }
    static __device__ __forceinline__ float2 mul(float2 x, float2 y) { return __fmul2_rn(x, y); }
    static __device__ __forceinline__ float2 fma(float2 x, float2 y, float2 z) { return __ffma2_rn(x, y, z); }
    static __device__ __forceinline__ float2 sub(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }
};
}  // namespace lanes

// The shifted collision hard-codes the library velocity order: odd i and i + 1 are
// opposite, the first non-zero component of an odd velocity is +1, and the pairs run
// +-x, +-y, +-z, xy(++), xy(+-), xz(++), xz(+-), yz(++), yz(+-).
constexpr bool shifted_order_holds()
{
    for (int i = 1; i < Q; i += 2) {
        if (opp(i) != i + 1) return false;
        const int first = cx(i) != 0 ? cx(i) : (cy(i) != 0 ? cy(i) : cz(i));
        if (first != 1) return false;
    }
    return cx(1) == 1 && cy(3) == 1 && cz(5) == 1 && cx(7) == 1 && cy(7) == 1 && cx(9) == 1 && cy(9) == -1 &&
           cx(11) == 1 && cz(11) == 1 && cx(13) == 1 && cz(13) == -1 && cy(15) == 1 && cz(15) == 1 &&
           cy(17) == 1 && cz(17) == -1;
}
static_assert(shifted_order_holds(), "kbc_shifted assumes the library velocity order");

// c_i . j for odd i (compile-time constant after unrolling)
template <class V, class Ar = lanes::Asm>
__device__ __forceinline__ V c_dot(int i, V jx, V jy, V jz)
{
    const auto add = [](V x, V y) { return Ar::add(x, y); };
    const auto sub = [](V x, V y) { return Ar::sub(x, y); };
    if (cx(i) != 0 && cy(i) != 0 && cz(i) != 0) {  // corner (D3Q27)
        const V t = cy(i) > 0 ? add(jx, jy) : sub(jx, jy);
        return cz(i) > 0 ? add(t, jz) : sub(t, jz);
    }
    if (cx(i) == 0 && cy(i) == 0) return jz;
    if (cx(i) == 0) return cz(i) == 0 ? jy : (cz(i) > 0 ? add(jy, jz) : sub(jy, jz));
    if (cy(i) != 0) return cy(i) > 0 ? add(jx, jy) : sub(jx, jy);
    if (cz(i) != 0) return cz(i) > 0 ? add(jx, jz) : sub(jx, jz);
    return jx;
}

#ifndef MCLBM_D3Q27
// KBC on normalised deviations h_i = f_i / w_i - 1 (in place), FP32, one node (V = float)
// or two (V = float2).  a = 2/omega and b = 2 - 2/omega are passed in (computed once on the
// host); the reciprocals 1/rho, 1/(1 + heq_i) and 1/hh are the hardware approximation (one
// ulp, below the FP32 rounding already present in the sums).  Ar: the arithmetic policy
// (lanes::Asm or lanes::Native, the same bits).
template <class V, class Ar = lanes::Asm>
__device__ __forceinline__ V kbc_shifted(V (&h)[Q], float omega, float a, float b)
{
    using lanes::bc;
    using lanes::map;
    using lanes::rcp_approx;
    const auto add = [](auto x, auto y) { return Ar::add(x, y); };
    const auto mul = [](auto x, auto y) { return Ar::mul(x, y); };
    const auto fma = [](auto x, auto y, auto z) { return Ar::fma(x, y, z); };
    const auto sub = [](auto x, auto y) { return Ar::sub(x, y); };
    const V one = bc<V>(1.f), W0 = bc<V>(1.0f / 3.0f), W1 = bc<V>(1.0f / 18.0f), W2 = bc<V>(1.0f / 36.0f);
    const auto frcp = [](float x) { return rcp_approx(x); };
    // density deviation and momentum: sum w h, sum w c h (d_p: difference of pair p)
    const V s1 = add(add(add(h[1], h[2]), add(h[3], h[4])), add(h[5], h[6]));
    const V s2 = add(add(add(add(h[7], h[8]), add(h[9], h[10])), add(add(h[11], h[12]), add(h[13], h[14]))),
                     add(add(h[15], h[16]), add(h[17], h[18])));
    const V drho = fma(W0, h[0], fma(W1, s1, mul(W2, s2)));
    const V rho = add(one, drho);
    V d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) d[p] = sub(h[2 * p + 1], h[2 * p + 2]);
    const V jx = fma(W1, d[0], mul(W2, add(add(d[3], d[4]), add(d[5], d[6]))));
    const V jy = fma(W1, d[1], mul(W2, add(sub(d[3], d[4]), add(d[7], d[8]))));
    const V jz = fma(W1, d[2], mul(W2, add(sub(d[5], d[6]), sub(d[7], d[8]))));
    const V rinv = map(rho, frcp);
    const V jj15 = mul(bc<V>(-1.5f), fma(jx, jx, fma(jy, jy, mul(jz, jz))));
    // f^eq / w - 1 = (rho - 1) + 3 c.j + (4.5 (c.j)^2 - 1.5 |j|^2) / rho: the linear term in c.j
    // carries exactly the node's momentum whatever the rounding of 1/rho.  Opposite velocities
    // share the even part q and differ in the sign of 3 c.j.
    V heq[Q], n[Q];
    heq[0] = fma(jj15, rinv, drho);
    n[0] = sub(h[0], heq[0]);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const V cj = c_dot<V, Ar>(i, jx, jy, jz);
        const V q = fma(rinv, fma(bc<V>(4.5f), mul(cj, cj), jj15), drho);
        heq[i] = fma(bc<V>(3.f), cj, q);
        heq[i + 1] = fma(bc<V>(-3.f), cj, q);
        n[i] = sub(h[i], heq[i]);
        n[i + 1] = sub(h[i + 1], heq[i + 1]);
    }
    // second moments of f^neq (normalised): P_ab = sum w c_a c_b n
    const V a78 = add(n[7], n[8]), a910 = add(n[9], n[10]), a1112 = add(n[11], n[12]);
    const V a1314 = add(n[13], n[14]), a1516 = add(n[15], n[16]), a1718 = add(n[17], n[18]);
    const V exy = add(a78, a910), exz = add(a1112, a1314), eyz = add(a1516, a1718);
    const V pxx = fma(W1, add(n[1], n[2]), mul(W2, add(exy, exz)));
    const V pyy = fma(W1, add(n[3], n[4]), mul(W2, add(exy, eyz)));
    const V pzz = fma(W1, add(n[5], n[6]), mul(W2, add(exz, eyz)));
    const V tr3 = mul(add(add(pxx, pyy), pzz), bc<V>(1.0f / 3.0f));
    // Shear part normalised by w (equal on opposite velocities): s = 9 D_c on the faces (D_c =
    // P_cc - tr/3) and s l P_ab / (4 w2) = +-D_c / 4 on the edges (D_c = the edge-sum difference,
    // sign + for pairs p = 3, 5, 7 and - for p = 4, 6, 8).  The factors enter only as constants
    // of single fma or multiply operations, never as a separately rounded product.
    V D[6];
    D[0] = sub(pxx, tr3);
    D[1] = sub(pyy, tr3);
    D[2] = sub(pzz, tr3);
    D[3] = sub(a78, a910);
    D[4] = sub(a1112, a1314);
    D[5] = sub(a1516, a1718);
    // k = Dh / w = n - s;  <Ds|Dh> = sum w s k / (1 + heq),  <Dh|Dh> = sum w k^2 / (1 + heq)
    V k[Q], A[9];
    k[0] = n[0];
    const V kr0 = mul(k[0], map(add(one, heq[0]), frcp));
    V hf = bc<V>(0.f), he = bc<V>(0.f);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const V Dp = D[p < 3 ? p : 3 + (p - 3) / 2];
        const float ms = p < 3 ? -9.f : ((p - 3) % 2 == 1 ? 0.25f : -0.25f);  // -s / D
        k[i] = fma(Dp, bc<V>(ms), n[i]);
        k[i + 1] = fma(Dp, bc<V>(ms), n[i + 1]);
        const V ka = mul(k[i], map(add(one, heq[i]), frcp));
        const V kb = mul(k[i + 1], map(add(one, heq[i + 1]), frcp));
        A[p] = add(ka, kb);
        if (p == 0)
            hf = fma(kb, k[i + 1], mul(ka, k[i]));
        else if (p < 3)
            hf = fma(kb, k[i + 1], fma(ka, k[i], hf));
        else if (p == 3)
            he = fma(kb, k[i + 1], mul(ka, k[i]));
        else
            he = fma(kb, k[i + 1], fma(ka, k[i], he));
    }
    // sh = w1 sum_faces 9 D (ka + kb) + w2 sum_edges (+-D / 4)(ka + kb), w1 9 = 1/2, w2 / 4 = 1/144
    const V sf = fma(D[0], A[0], fma(D[1], A[1], mul(D[2], A[2])));
    const V se = fma(D[3], sub(A[3], A[4]), fma(D[4], sub(A[5], A[6]), mul(D[5], sub(A[7], A[8]))));
    const V sh = fma(bc<V>(0.5f), sf, mul(bc<V>(1.0f / 144.0f), se));
    const V hh = fma(W0, mul(kr0, k[0]), fma(W1, hf, mul(W2, he)));
    const V gamma = map(hh, sh, [a, b, fma, mul](float hs, float ss) {
        return hs <= kHHGuard ? 2.0f : fma(-b, mul(ss, rcp_approx(hs)), a);
    });
    // f* = f - omega Ds - (omega gamma / 2) Dh, written as f^eq + (1 - omega) Ds + (1 - beta) Dh so
    // that h is not needed past n (fewer live registers)
    const V omb = fma(bc<V>(-0.5f * omega), gamma, one);  // 1 - beta
    h[0] = fma(omb, k[0], heq[0]);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const float sd = p < 3 ? 9.f : ((p - 3) % 2 == 1 ? -0.25f : 0.25f);  // s / D
        const V cs = bc<V>(sd * (1.0f - omega));
        const V Dp = D[p < 3 ? p : 3 + (p - 3) / 2];
        h[i] = fma(omb, k[i], fma(Dp, cs, heq[i]));
        h[i + 1] = fma(omb, k[i + 1], fma(Dp, cs, heq[i + 1]));
    }
    return gamma;
}

#else  // MCLBM_D3Q27

// D3Q27 form of kbc_shifted: the same operations written out over the 13 opposite pairs
// (p = 0..2 faces, 3..8 edges as in D3Q19, 9..12 corners (+++), (++-), (+-+), (+--)).  The
// shear part is D_aa / 2 on faces, s l P_ab / 4 on edges and 0 on corners; normalised by the
// weights, s = D_aa / (2 w1) = 6.75 D_aa and s l P_ab / (4 w2) = +-13.5 P_ab.  P_ab includes
// the corners.  As in the D3Q19 form, constant factors enter as operands of single operations.
constexpr bool d3q27_order_holds()
{
    return cx(19) == 1 && cy(19) == 1 && cz(19) == 1 && cx(21) == 1 && cy(21) == 1 && cz(21) == -1 &&
           cx(23) == 1 && cy(23) == -1 && cz(23) == 1 && cx(25) == 1 && cy(25) == -1 && cz(25) == -1;
}
static_assert(d3q27_order_holds(), "kbc_shifted assumes the library's D3Q27 corner order");

// (Ar: accepted for a uniform call; this form is written in the Asm arithmetic.)
template <class V, class Ar = lanes::Asm>
__device__ __forceinline__ V kbc_shifted(V (&h)[Q], float omega, float a, float b)
{
    static_assert(std::is_same<Ar, lanes::Asm>::value, "the D3Q27 collision takes the Asm arithmetic");
    using namespace lanes;
    const V one = bc<V>(1.f);
    const V W0 = bc<V>(8.0f / 27.0f), W1 = bc<V>(2.0f / 27.0f), W2 = bc<V>(1.0f / 54.0f), W3 = bc<V>(1.0f / 216.0f);
    const auto frcp = [](float x) { return rcp_approx(x); };
    // density deviation and momentum
    const V s1 = add(add(add(h[1], h[2]), add(h[3], h[4])), add(h[5], h[6]));
    const V s2 = add(add(add(add(h[7], h[8]), add(h[9], h[10])), add(add(h[11], h[12]), add(h[13], h[14]))),
                     add(add(h[15], h[16]), add(h[17], h[18])));
    const V s3 = add(add(add(h[19], h[20]), add(h[21], h[22])), add(add(h[23], h[24]), add(h[25], h[26])));
    const V drho = fma(W0, h[0], fma(W1, s1, fma(W2, s2, mul(W3, s3))));
    const V rho = add(one, drho);
    V d[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) d[p] = sub(h[2 * p + 1], h[2 * p + 2]);
    const V jx = fma(W1, d[0], fma(W2, add(add(d[3], d[4]), add(d[5], d[6])),
                                   mul(W3, add(add(d[9], d[10]), add(d[11], d[12])))));
    const V jy = fma(W1, d[1], fma(W2, add(sub(d[3], d[4]), add(d[7], d[8])),
                                   mul(W3, sub(add(d[9], d[10]), add(d[11], d[12])))));
    const V jz = fma(W1, d[2], fma(W2, add(sub(d[5], d[6]), sub(d[7], d[8])),
                                   mul(W3, add(sub(d[9], d[10]), sub(d[11], d[12])))));
    const V rinv = map(rho, frcp);
    const V jj15 = mul(bc<V>(-1.5f), fma(jx, jx, fma(jy, jy, mul(jz, jz))));
    V heq[Q], n[Q];
    heq[0] = fma(jj15, rinv, drho);
    n[0] = sub(h[0], heq[0]);
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        const V cj = c_dot(i, jx, jy, jz);
        const V q = fma(rinv, fma(bc<V>(4.5f), mul(cj, cj), jj15), drho);
        heq[i] = fma(bc<V>(3.f), cj, q);
        heq[i + 1] = fma(bc<V>(-3.f), cj, q);
        n[i] = sub(h[i], heq[i]);
        n[i + 1] = sub(h[i + 1], heq[i + 1]);
    }
    // second moments of f^neq (normalised): pair sums A_p = n_i + n_{i+1}
    V A[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) A[p] = add(n[2 * p + 1], n[2 * p + 2]);
    const V exy = add(A[3], A[4]), exz = add(A[5], A[6]), eyz = add(A[7], A[8]);
    const V cs = add(add(A[9], A[10]), add(A[11], A[12]));  // every corner has c_a^2 = 1
    const V cxy = sub(add(A[9], A[10]), add(A[11], A[12]));
    const V cxz = add(sub(A[9], A[10]), sub(A[11], A[12]));
    const V cyz = sub(sub(A[9], A[10]), sub(A[11], A[12]));
    const V pxx = fma(W1, A[0], fma(W2, add(exy, exz), mul(W3, cs)));
    const V pyy = fma(W1, A[1], fma(W2, add(exy, eyz), mul(W3, cs)));
    const V pzz = fma(W1, A[2], fma(W2, add(exz, eyz), mul(W3, cs)));
    const V tr3 = mul(add(add(pxx, pyy), pzz), bc<V>(1.0f / 3.0f));
    V D[6];
    D[0] = sub(pxx, tr3);
    D[1] = sub(pyy, tr3);
    D[2] = sub(pzz, tr3);
    D[3] = fma(W2, sub(A[3], A[4]), mul(W3, cxy));  // P_xy
    D[4] = fma(W2, sub(A[5], A[6]), mul(W3, cxz));  // P_xz
    D[5] = fma(W2, sub(A[7], A[8]), mul(W3, cyz));  // P_yz
    // k = n - s;  <Ds|Dh> = sum w s k / (1 + heq),  <Dh|Dh> = sum w k^2 / (1 + heq)
    V k[Q], B[9];
    k[0] = n[0];
    const V kr0 = mul(k[0], map(add(one, heq[0]), frcp));
    V hf = bc<V>(0.f), he = bc<V>(0.f), hc = bc<V>(0.f);
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        if (p < 9) {
            const V Dp = D[p < 3 ? p : 3 + (p - 3) / 2];
            const float ms = p < 3 ? -6.75f : ((p - 3) % 2 == 1 ? 13.5f : -13.5f);  // -s / D
            k[i] = fma(Dp, bc<V>(ms), n[i]);
            k[i + 1] = fma(Dp, bc<V>(ms), n[i + 1]);
        } else {
            k[i] = n[i];
            k[i + 1] = n[i + 1];
        }
        const V ka = mul(k[i], map(add(one, heq[i]), frcp));
        const V kb = mul(k[i + 1], map(add(one, heq[i + 1]), frcp));
        if (p < 9) B[p] = add(ka, kb);
        if (p == 0)
            hf = fma(kb, k[i + 1], mul(ka, k[i]));
        else if (p < 3)
            hf = fma(kb, k[i + 1], fma(ka, k[i], hf));
        else if (p == 3)
            he = fma(kb, k[i + 1], mul(ka, k[i]));
        else if (p < 9)
            he = fma(kb, k[i + 1], fma(ka, k[i], he));
        else if (p == 9)
            hc = fma(kb, k[i + 1], mul(ka, k[i]));
        else
            hc = fma(kb, k[i + 1], fma(ka, k[i], hc));
    }
    // sh = w1 sum_faces 6.75 D (ka + kb) + w2 sum_edges (+-13.5 P)(ka + kb): w1 6.75 = 1/2,
    // w2 13.5 = 1/4
    const V sf = fma(D[0], B[0], fma(D[1], B[1], mul(D[2], B[2])));
    const V se = fma(D[3], sub(B[3], B[4]), fma(D[4], sub(B[5], B[6]), mul(D[5], sub(B[7], B[8]))));
    const V sh = fma(bc<V>(0.5f), sf, mul(bc<V>(0.25f), se));
    const V hh = fma(W0, mul(kr0, k[0]), fma(W1, hf, fma(W2, he, mul(W3, hc))));
    const V gamma = map(hh, sh, [a, b](float hs, float ss) {
        return hs <= kHHGuard ? 2.0f : fma(-b, mul(ss, rcp_approx(hs)), a);
    });
    // f* = f^eq + (1 - omega) Ds + (1 - beta) Dh
    const V omb = fma(bc<V>(-0.5f * omega), gamma, one);
    h[0] = fma(omb, k[0], heq[0]);
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        if (p < 9) {
            const float sd = p < 3 ? 6.75f : ((p - 3) % 2 == 1 ? -13.5f : 13.5f);  // s / D
            const V cs1 = bc<V>(sd * (1.0f - omega));
            const V Dp = D[p < 3 ? p : 3 + (p - 3) / 2];
            h[i] = fma(omb, k[i], fma(Dp, cs1, heq[i]));
            h[i + 1] = fma(omb, k[i + 1], fma(Dp, cs1, heq[i + 1]));
        } else {
            h[i] = fma(omb, k[i], heq[i]);
            h[i + 1] = fma(omb, k[i + 1], heq[i + 1]);
        }
    }
    return gamma;
}

#endif  // MCLBM_D3Q27

// ---- Exact entropic gamma (option MCLBM_OPT_EXACT_GAMMA) -----------------------------------
// gamma minimises H(f*(g)) = sum f*_i ln(f*_i / w_i), Eq. (kbc_entropy), over the line
// f*(g) = f - omega Ds - (omega g / 2) Dh with 0 <= g <= 4 / omega (the relaxation factor
// omega g / 2 of Dh in the stable [0, 2]; with the polynomial equilibrium the unconstrained
// minimiser grows like 1 / |Dh| near equilibrium).  Since sum Dh = 0 the stationary point is
// the root of G(g) = sum Dh_i ln(f*_i / w_i); G decreases (G' = -(omega / 2) sum Dh_i^2 / f*_i)
// where every f*_i > 0, so the constrained minimiser is the root or the nearer end point.
// Written with r_i = f*_i / w_i = 1 + am1_i - g b_i (b_i = (omega / 2) Dh_i / w_i):
// safeguarded Newton (FP32) or Halley (FP64) iteration from the closed form, keeping a bracket
// of the root and bisecting where a step leaves it.  T = double (FP64) or float (FP32).
template <class T>
__device__ __forceinline__ T log1p_of(T x)
{
    if constexpr (sizeof(T) == 8)
        return log1p(x);
    else
        return log1pf(x);
}

template <class T>
__device__ __forceinline__ T exact_gamma_refine(const T (&am1)[Q], const T (&b)[Q], T omega, T g0, int max_iter,
                                                T rel_tol)
{
    // constrained interval: 0 <= g <= 4 / omega and every r_i = 1 + am1_i - g b_i > 0 (a
    // division only where the positivity bound binds)
    T lo = T(0), hi = T(4) / omega;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T a = T(1) + am1[i];
        if (b[i] > T(0) && hi * b[i] > a) hi = a / b[i];
        else if (b[i] < T(0) && lo * b[i] > a) lo = a / b[i];
    }
    if (!(lo < hi)) return g0;
    // H is convex along the line.  G = sum w_i b_i ln r_i equals -dH/dg up to a positive factor
    // (sum w_i b_i = 0: Dh carries no mass), so G decreases with g: G(hi) >= 0 means that H still
    // decreases at hi (the minimum is at hi), G(lo) <= 0 that it increases from lo.  The sign of G
    // at a bracket end is known once an iterate has replaced that end; an end of the interval is
    // evaluated (probe) only when a step would leave the bracket through it, since the closed-form
    // start lies close to an interior root for most nodes.  One evaluation site serves the
    // iterates and the probes (the sum is unrolled over the velocities with a logarithm each).
    // FP64 takes Halley steps (G'' = -sum w_i b_i^3 / r_i^2), FP32 Newton steps; G' and G'' only
    // steer the step, so FP32 forms b_i / r_i with the approximate division.
    const T eps = sizeof(T) == 8 ? T(2.220446049250313e-16) : T(1.1920929e-7);
    T g = (g0 > lo && g0 < hi) ? g0 : T(0.5) * (lo + hi);
    bool lo_known = false, hi_known = false;
    int probe = 0;  // 0: G at the iterate g; 1: at hi; 2: at lo
    for (int it = 0; it < max_iter; ++it) {
        const T ge = probe == 0 ? g : (probe == 1 ? hi : lo);
        T G = 0, Gp = 0, Gpp = 0, S = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // r_i - 1 formed first, so that r close to 1 keeps its digits in the logarithm
            const T x = am1[i] - ge * b[i];
            const T wb = weight<T>(i) * b[i];
            const T t = wb * log1p_of<T>(x);
            G += t;
            S += fabs(t);
            T q;  // b_i / r_i
            if constexpr (sizeof(T) == 8)
                q = b[i] / (T(1) + x);
            else
                q = __fdividef(b[i], T(1) + x);
            Gp -= wb * q;
            if constexpr (sizeof(T) == 8) Gpp -= wb * q * q;
        }
        T gn;
        if (probe != 0) {
            if (probe == 1) {
                if (!(G < T(0))) return hi;  // H decreases up to hi
                hi_known = true;
            } else {
                if (!(G > T(0))) return lo;  // H increases from lo
                lo_known = true;
            }
            probe = 0;
            gn = T(0.5) * (lo + hi);
        } else {
            if (fabs(G) <= T(4 * Q) * eps * S) return g;  // G at the rounding level of its own terms
            if (G > T(0)) {
                lo = g;
                lo_known = true;
            } else {
                hi = g;
                hi_known = true;
            }
            gn = g - G / Gp;
            if constexpr (sizeof(T) == 8) {
                const T den = T(2) * Gp * Gp - G * Gpp;
                if (den > T(0)) gn = g - T(2) * G * Gp / den;
            }
            if (!(gn > lo && gn < hi)) {
                if (!(gn < hi) && !hi_known) {
                    probe = 1;
                    continue;
                }
                if (!(gn > lo) && !lo_known) {
                    probe = 2;
                    continue;
                }
                gn = T(0.5) * (lo + hi);
            }
        }
        if (fabs(gn - g) <= rel_tol * fabs(g)) return gn;
        g = gn;
    }
    return g;
}

// KBC with the exact gamma, one node, any velocity set, in the normalised deviations
// h = f / w - 1 (raw FP64 populations are converted on entry and exit; FP32 storage holds h).
// The equilibrium, shear part and closed-form gamma are those of kbc_shifted written over all
// velocities; the closed form starts the Newton iteration.  Returns gamma.
template <class T, bool SHIFTED>
__device__ __forceinline__ T kbc_exact(T (&f)[Q], T omega)
{
    T h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = SHIFTED ? f[i] : f[i] * inv_weight<T>(i) - T(1);
    T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T wh = weight<T>(i) * h[i];
        drho += wh;
        MCLBM_SIGNED_ADD(jx, cx(i), wh);
        MCLBM_SIGNED_ADD(jy, cy(i), wh);
        MCLBM_SIGNED_ADD(jz, cz(i), wh);
    }
    const T rinv = T(1) / (T(1) + drho);
    const T jj = jx * jx + jy * jy + jz * jz;
    T heq[Q], n[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T cj = 0;
        MCLBM_SIGNED_ADD(cj, cx(i), jx);
        MCLBM_SIGNED_ADD(cj, cy(i), jy);
        MCLBM_SIGNED_ADD(cj, cz(i), jz);
        heq[i] = drho + T(3) * cj + rinv * (T(4.5) * cj * cj - T(1.5) * jj);
        n[i] = h[i] - heq[i];
    }
    T pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T wn = weight<T>(i) * n[i];
        if (cx(i) != 0) pxx += wn;
        if (cy(i) != 0) pyy += wn;
        if (cz(i) != 0) pzz += wn;
        MCLBM_SIGNED_ADD(pxy, cx(i) * cy(i), wn);
        MCLBM_SIGNED_ADD(pxz, cx(i) * cz(i), wn);
        MCLBM_SIGNED_ADD(pyz, cy(i) * cz(i), wn);
    }
    const T tr3 = (pxx + pyy + pzz) / T(3);
    T s[Q], k[Q];
    T sh = 0, hh = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int n2 = norm2(i);
        if (n2 == 0 || n2 == 3) s[i] = 0;
        else if (n2 == 1) s[i] = T(0.5) * inv_weight<T>(i) * ((cx(i) ? pxx : (cy(i) ? pyy : pzz)) - tr3);
        else {
            const T p = (cz(i) == 0) ? pxy : ((cy(i) == 0) ? pxz : pyz);
            const int sg = (cz(i) == 0) ? cx(i) * cy(i) : ((cy(i) == 0) ? cx(i) * cz(i) : cy(i) * cz(i));
            s[i] = (sg > 0 ? T(0.25) : -T(0.25)) * inv_weight<T>(i) * p;
        }
        k[i] = n[i] - s[i];
        // the closed form only starts the iteration: FP32 divides approximately
        T wk;
        if constexpr (sizeof(T) == 8)
            wk = weight<T>(i) * k[i] / (T(1) + heq[i]);
        else
            wk = __fdividef(weight<T>(i) * k[i], T(1) + heq[i]);
        sh += wk * s[i];
        hh += wk * k[i];
    }
    const T guard = sizeof(T) == 8 ? T(0) : T(kHHGuard);
    T gamma = (hh <= guard) ? T(2) : T(2) / omega - (T(2) - T(2) / omega) * sh / hh;
    if (hh > guard) {
        // f*_i / w_i = 1 + (h_i - omega s_i) - g (omega / 2) k_i
        T am1[Q], b[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            am1[i] = h[i] - omega * s[i];
            b[i] = T(0.5) * omega * k[i];
        }
        gamma = exact_gamma_refine<T>(am1, b, omega, gamma, sizeof(T) == 8 ? 60 : 30, sizeof(T) == 8 ? T(1e-15) : T(1e-7));
    }
    const T bo = T(0.5) * omega * gamma;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T hs = h[i] - omega * s[i] - bo * k[i];
        f[i] = SHIFTED ? hs : weight<T>(i) * (T(1) + hs);
    }
    return gamma;
}

}  // namespace mclbm
