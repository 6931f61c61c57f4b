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
#include "lattice.cuh"

namespace mclbm {

// Signed sum over the populations: sum_i s(i) v_i with s(i) a compile-time
// sign in {-1, 0, 1}; the zero terms are dropped at compile time.
#define MCLBM_SIGNED_ADD(acc, sgn, v) \
    do {                              \
        if ((sgn) > 0) acc += (v);    \
        else if ((sgn) < 0) acc -= (v); \
    } while (0)

// Plain KBC on raw populations (in place).  Returns gamma.
template <class T>
__host__ __device__ __forceinline__ T kbc_raw(T (&f)[Q], T omega)
{
    T rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        MCLBM_SIGNED_ADD(jx, cx(i), f[i]);
        MCLBM_SIGNED_ADD(jy, cy(i), f[i]);
        MCLBM_SIGNED_ADD(jz, cz(i), f[i]);
    }
    const T ux = jx / rho, uy = jy / rho, uz = jz / rho;
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
    const T tr3 = (pxx + pyy + pzz) / T(3);
    T ds[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int n2 = norm2(i);
        if (n2 == 0) ds[i] = 0;
        else if (n2 == 1) ds[i] = T(0.5) * ((cx(i) ? pxx : (cy(i) ? pyy : pzz)) - tr3);
        else {
            const T p = (cz(i) == 0) ? pxy : ((cy(i) == 0) ? pxz : pyz);
            const int s = (cz(i) == 0) ? cx(i) * cy(i) : ((cy(i) == 0) ? cx(i) * cz(i) : cy(i) * cz(i));
            ds[i] = s > 0 ? T(0.25) * p : -T(0.25) * p;
        }
    }
    T sh = 0, hh = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T dh = fneq[i] - ds[i];
        sh += ds[i] * dh / feq[i];
        hh += dh * dh / feq[i];
    }
    const T gamma = (hh == T(0)) ? T(2) : T(2) / omega - (T(2) - T(2) / omega) * sh / hh;
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

// KBC on normalised deviations h_i = f_i / w_i - 1 (in place), FP32.  a = 2/omega and
// b = 2 - 2/omega are passed in (computed once on the host); the reciprocals 1/rho and
// w_i / (1 + heq_i) and the quotient sh/hh use the fast approximate division (a few ulp,
// below the FP32 rounding already present in the sums).
__device__ __forceinline__ float kbc_shifted(float (&h)[Q], float omega, float a, float b)
{
    constexpr float w0 = 1.0f / 3.0f, w1 = 1.0f / 18.0f, w2 = 1.0f / 36.0f;
    // density deviation and momentum: sum w h, sum w c h
    float s0 = h[0], s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int i = 1; i < 7; ++i) s1 += h[i];
#pragma unroll
    for (int i = 7; i < Q; ++i) s2 += h[i];
    const float drho = w0 * s0 + w1 * s1 + w2 * s2;
    const float rho = 1.0f + drho;
    const float jx = w1 * (h[1] - h[2]) + w2 * ((h[7] - h[8]) + (h[9] - h[10]) + (h[11] - h[12]) + (h[13] - h[14]));
    const float jy = w1 * (h[3] - h[4]) + w2 * ((h[7] - h[8]) - (h[9] - h[10]) + (h[15] - h[16]) + (h[17] - h[18]));
    const float jz = w1 * (h[5] - h[6]) + w2 * ((h[11] - h[12]) - (h[13] - h[14]) + (h[15] - h[16]) - (h[17] - h[18]));
    const float rinv = __fdividef(1.0f, rho);
    const float jj = jx * jx + jy * jy + jz * jz;
    // f^eq / w - 1 = (rho - 1) + 3 c.j + (4.5 (c.j)^2 - 1.5 |j|^2) / rho: the linear term in c.j
    // carries exactly the node's momentum whatever the rounding of 1/rho.  Opposite velocities
    // share the even part q and differ in the sign of 3 c.j.
    float heq[Q], n[Q];
    heq[0] = drho - 1.5f * jj * rinv;
    n[0] = h[0] - heq[0];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        float cj = 0.f;
        MCLBM_SIGNED_ADD(cj, cx(i), jx);
        MCLBM_SIGNED_ADD(cj, cy(i), jy);
        MCLBM_SIGNED_ADD(cj, cz(i), jz);
        const float q = drho + rinv * (4.5f * cj * cj - 1.5f * jj);
        heq[i] = q + 3.0f * cj;
        heq[i + 1] = q - 3.0f * cj;
        n[i] = h[i] - heq[i];
        n[i + 1] = h[i + 1] - heq[i + 1];
    }
    // second moments of f^neq (normalised): P_ab = sum w c_a c_b n
    const float ex = n[7] + n[8] + n[9] + n[10];      // xy edges
    const float exz = n[11] + n[12] + n[13] + n[14];  // xz edges
    const float eyz = n[15] + n[16] + n[17] + n[18];  // yz edges
    const float pxx = w1 * (n[1] + n[2]) + w2 * (ex + exz);
    const float pyy = w1 * (n[3] + n[4]) + w2 * (ex + eyz);
    const float pzz = w1 * (n[5] + n[6]) + w2 * (exz + eyz);
    const float pxy = w2 * ((n[7] + n[8]) - (n[9] + n[10]));
    const float pxz = w2 * ((n[11] + n[12]) - (n[13] + n[14]));
    const float pyz = w2 * ((n[15] + n[16]) - (n[17] + n[18]));
    const float tr3 = (pxx + pyy + pzz) * (1.0f / 3.0f);
    // shear part normalised by w (equal on opposite velocities): faces 9 D_aa, edges 9 s l P_ab
    float sp[9];
    sp[0] = 9.0f * (pxx - tr3);
    sp[1] = 9.0f * (pyy - tr3);
    sp[2] = 9.0f * (pzz - tr3);
    sp[3] = 9.0f * pxy;
    sp[4] = -9.0f * pxy;
    sp[5] = 9.0f * pxz;
    sp[6] = -9.0f * pxz;
    sp[7] = 9.0f * pyz;
    sp[8] = -9.0f * pyz;
    // <Ds|Dh> and <Dh|Dh> with 1/f^eq = 1/(w (1 + heq)): sum w s k / (1 + heq)
    float k[Q];
    k[0] = n[0];
    float hh = __fdividef(w0, 1.0f + heq[0]) * k[0] * k[0];
    float sh = 0.f;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        k[i] = n[i] - sp[p];
        k[i + 1] = n[i + 1] - sp[p];
        const float wa = __fdividef(weight<float>(i), 1.0f + heq[i]);
        const float wb = __fdividef(weight<float>(i), 1.0f + heq[i + 1]);
        const float ka = wa * k[i], kb = wb * k[i + 1];
        sh += sp[p] * (ka + kb);
        hh += ka * k[i] + kb * k[i + 1];
    }
    const float gamma = (hh <= kHHGuard) ? 2.0f : a - b * __fdividef(sh, hh);
    const float bo = 0.5f * omega * gamma;
    h[0] = h[0] - bo * k[0];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        h[i] = h[i] - omega * sp[p] - bo * k[i];
        h[i + 1] = h[i + 1] - omega * sp[p] - bo * k[i + 1];
    }
    return gamma;
}

}  // namespace mclbm
