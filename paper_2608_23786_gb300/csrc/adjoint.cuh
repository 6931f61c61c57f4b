// Hand-written vector-Jacobian product of the KBC collision (Eqs. (equilibrium),
// (kbcCollision), (entropyControl)), including the derivative of the stabiliser gamma.
//
// Forward, in the normalised deviations h = f / w - 1 of one node:
//   rho = 1 + sum w h, u = (sum w c h) / rho, e_i = f^eq_i / w_i = rho P_i(u),
//   n = h - (e - 1) (f^neq / w), s = Ds / w (shear part), k = Dh / w = n - s,
//   sh = sum w s k / e, hh = sum w k^2 / e, gamma = a - b sh / hh (a = 2/omega,
//   b = 2 - 2/omega; gamma = 2 where hh <= guard), f* = f - omega Ds - beta Dh,
//   beta = omega gamma / 2.
// Given mu = dJ/df* (raw units), the product returns lambda = dJ/df:
//   dJ = mu.df - omega mu.dDs - beta mu.dDh + Gam dgamma,  Gam = -(omega/2) mu.Dh,
//   dgamma = A1 dsh + A2 dhh,  A1 = -b/hh,  A2 = b sh/hh^2,
//   dsh = sum (dDs Dh + Ds dDh)/feq - Ds Dh dfeq/feq^2,
//   dhh = sum 2 Dh dDh/feq - Dh^2 dfeq/feq^2,
// so dJ = mu.df + g_s.dDs + g_h.dDh + g_eq.dfeq with
//   g_s = -omega mu + Gam A1 k/e,   g_h = -beta mu + Gam (A1 s + 2 A2 k)/e,
//   g_eq = -Gam (A1 s k + A2 k^2)/e^2.
// With R1 = (mu.Dh)/hh and R2 = sh/hh (c = omega b / 2): Gam A1 = c R1, Gam A2 = -c R1 R2,
// so every term is a product of the two ratios with components of k and s; no 1/hh^2
// is formed (it underflows in FP32 where Dh is small).
// Ds = A f^neq with the fixed shear projection A and Dh = (I - A) f^neq, f^neq = f - f^eq:
//   r = A^T (g_s - g_h) + g_h,  q = g_eq - r,  dJ = (mu + r).df + q.dfeq,
// and f^eq(rho, u) with drho = sum df, du = (dj - u drho)/rho, dj = sum c df gives
//   lambda_j = mu_j + r_j + (Q_rho - Q_u.u/rho) + Q_u.c_j/rho,
//   Q_rho = sum q_i w_i e_i / rho,  Q_u = sum q_i rho w_i (3 c_i + 9 (c_i.u) c_i - 3 u).
// A^T v is formed through the adjoint second moments
//   Pi_dd = (v_{+d} + v_{-d})/2 - (sum over faces v)/6,  Pi_ab = (sum over ab edges s l v)/4,
//   (A^T v)_j = sum_d Pi_dd c_jd^2 + sum_{a<b} Pi_ab c_ja c_jb.
#pragma once
#include "collide.cuh"

namespace mclbm {

// 1/x: IEEE in FP64, the hardware reciprocal approximation in FP32 (one ulp; the arguments are
// 1 + O(Ma) densities and equilibria, and <Dh|Dh> above its guard)
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return lanes::rcp_approx(x); }

template <class T>
__device__ __forceinline__ void kbc_vjp(const T (&h)[Q], const T (&mu)[Q], T omega, T hh_guard, T (&lam)[Q])
{
    // ---- forward quantities
    T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T wh = weight<T>(i) * h[i];
        drho += wh;
        MCLBM_SIGNED_ADD(jx, cx(i), wh);
        MCLBM_SIGNED_ADD(jy, cy(i), wh);
        MCLBM_SIGNED_ADD(jz, cz(i), wh);
    }
    const T rho = T(1) + drho;
    const T irho = recip(rho);
    const T ux = jx * irho, uy = jy * irho, uz = jz * irho;
    const T uu = ux * ux + uy * uy + uz * uz;
    T e[Q], ie[Q], n[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T cu = 0;
        MCLBM_SIGNED_ADD(cu, cx(i), ux);
        MCLBM_SIGNED_ADD(cu, cy(i), uy);
        MCLBM_SIGNED_ADD(cu, cz(i), uz);
        const T heq = drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        e[i] = T(1) + heq;
        ie[i] = recip(e[i]);
        n[i] = h[i] - heq;
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
    const T tr3 = (pxx + pyy + pzz) * (T(1) / T(3));
    T s[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int n2 = norm2(i);
        if (n2 == 0) s[i] = 0;
        else if (n2 == 1) s[i] = T(9) * ((cx(i) ? pxx : (cy(i) ? pyy : pzz)) - tr3);
        else {
            const T p = (cz(i) == 0) ? pxy : ((cy(i) == 0) ? pxz : pyz);
            const int sg = (cz(i) == 0) ? cx(i) * cy(i) : ((cy(i) == 0) ? cx(i) * cz(i) : cy(i) * cz(i));
            s[i] = sg > 0 ? T(9) * p : -T(9) * p;
        }
    }
    T sh = 0, hh = 0, mk = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T k = n[i] - s[i];
        const T wk = weight<T>(i) * k * ie[i];
        sh += wk * s[i];
        hh += wk * k;
        mk += mu[i] * weight<T>(i) * k;  // mu . Dh
    }
    const T a = T(2) / omega, b = T(2) - T(2) / omega;
    const bool active = hh > hh_guard;
    const T ihh = active ? recip(hh) : T(0);
    const T R2 = sh * ihh;
    const T R1 = mk * ihh;
    const T gamma = active ? a - b * R2 : T(2);
    const T beta = T(0.5) * omega * gamma;
    const T c1 = T(0.5) * omega * b * R1;  // Gam A1
    const T c2 = -c1 * R2;                 // Gam A2
    // ---- coefficient vectors (raw units)
    T gs[Q], gh[Q], geq[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T k = n[i] - s[i];
        gs[i] = -omega * mu[i] + c1 * k * ie[i];
        gh[i] = -beta * mu[i] + (c1 * s[i] + T(2) * c2 * k) * ie[i];
        geq[i] = -(c1 * s[i] * k + c2 * k * k) * (ie[i] * ie[i]);
    }
    // ---- r = A^T (gs - gh) + gh via adjoint second moments
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = gs[i] - gh[i];
    T faces = 0;
#pragma unroll
    for (int i = 1; i < 7; ++i) faces += d[i];
    const T f6 = faces * (T(1) / T(6));
    const T Pxx = T(0.5) * (d[1] + d[2]) - f6;
    const T Pyy = T(0.5) * (d[3] + d[4]) - f6;
    const T Pzz = T(0.5) * (d[5] + d[6]) - f6;
    const T Pxy = T(0.25) * ((d[7] + d[8]) - (d[9] + d[10]));
    const T Pxz = T(0.25) * ((d[11] + d[12]) - (d[13] + d[14]));
    const T Pyz = T(0.25) * ((d[15] + d[16]) - (d[17] + d[18]));
    T r[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        T at = 0;
        if (cx(j) != 0) at += Pxx;
        if (cy(j) != 0) at += Pyy;
        if (cz(j) != 0) at += Pzz;
        MCLBM_SIGNED_ADD(at, cx(j) * cy(j), Pxy);
        MCLBM_SIGNED_ADD(at, cx(j) * cz(j), Pxz);
        MCLBM_SIGNED_ADD(at, cy(j) * cz(j), Pyz);
        r[j] = at + gh[j];
    }
    // ---- equilibrium chain
    T Qr = 0, Qx = 0, Qy = 0, Qz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T q = geq[i] - r[i];
        const T wq = weight<T>(i) * q;
        Qr += wq * e[i];
        T cu = 0;
        MCLBM_SIGNED_ADD(cu, cx(i), ux);
        MCLBM_SIGNED_ADD(cu, cy(i), uy);
        MCLBM_SIGNED_ADD(cu, cz(i), uz);
        const T t9 = T(3) + T(9) * cu;
        T gx = -T(3) * ux, gy = -T(3) * uy, gz = -T(3) * uz;
        MCLBM_SIGNED_ADD(gx, cx(i), t9);
        MCLBM_SIGNED_ADD(gy, cy(i), t9);
        MCLBM_SIGNED_ADD(gz, cz(i), t9);
        Qx += wq * rho * gx;
        Qy += wq * rho * gy;
        Qz += wq * rho * gz;
    }
    Qr *= irho;
    const T qx = Qx * irho, qy = Qy * irho, qz = Qz * irho;
    const T base = Qr - (qx * ux + qy * uy + qz * uz);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        T v = mu[j] + r[j] + base;
        MCLBM_SIGNED_ADD(v, cx(j), qx);
        MCLBM_SIGNED_ADD(v, cy(j), qy);
        MCLBM_SIGNED_ADD(v, cz(j), qz);
        lam[j] = v;
    }
}

}  // namespace mclbm
