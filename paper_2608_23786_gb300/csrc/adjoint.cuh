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
#include <type_traits>

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
        // normalised shear part s = Ds / w: D_aa / (2 w) on faces, s l P_ab / (4 w) on edges,
        // 0 at rest and on (D3Q27) corners
        if (n2 == 0 || n2 == 3) s[i] = 0;
        else if (n2 == 1) s[i] = T(0.5) * inv_weight<T>(i) * ((cx(i) ? pxx : (cy(i) ? pyy : pzz)) - tr3);
        else {
            const T p = (cz(i) == 0) ? pxy : ((cy(i) == 0) ? pxz : pyz);
            const int sg = (cz(i) == 0) ? cx(i) * cy(i) : ((cy(i) == 0) ? cx(i) * cz(i) : cy(i) * cz(i));
            s[i] = (sg > 0 ? T(0.25) : -T(0.25)) * inv_weight<T>(i) * p;
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

#ifndef MCLBM_D3Q27
// The same product for the FP32 path in the lane form of collide.cuh (V = float for one node,
// float2 for two nodes in the packed FP32x2 instructions), with opposite velocities paired:
// the pair shares s, c_i c_i^T and the even part of the equilibrium, so A^T v, the
// equilibrium chain and the c_j . Q_u term are formed once per pair.  With nq = -q and
// NV = sum_i nq_i w_i (3 c_i + 9 (c_i . u) c_i - 3 u) (so Q_u / rho = -NV) and
// NQr = sum_i nq_i w_i e_i (so Q_rho = -NQr / rho):
//   lambda_j = mu_j + r_j + (NV . u - NQr / rho) - c_j . NV,
// and a pair (c, -c) contributes 3 w [(nq_+ - nq_-) + 3 (c . u)(nq_+ + nq_-)] c - 3 w u (nq_+ + nq_-)
// to NV.  Forward quantities are those of kbc_shifted (same operations up to k); gamma = 2 and
// no dgamma where <Dh|Dh> is at or below kHHGuard.
template <class V, class Ar = lanes::Asm>
__device__ __forceinline__ void kbc_vjp_shifted(const V (&h)[Q], const V (&mu)[Q], float omega, float a, float b,
                                                V (&lam)[Q])
{
    static_assert(std::is_same<Ar, lanes::Asm>::value, "the D3Q19 transposed collision takes the Asm arithmetic");
    using namespace lanes;
    const V one = bc<V>(1.f), W0 = bc<V>(1.0f / 3.0f), W1 = bc<V>(1.0f / 18.0f), W2 = bc<V>(1.0f / 36.0f);
    const auto frcp = [](float x) { return rcp_approx(x); };
    // ---- forward, as kbc_shifted
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
    V heq[Q], n[Q];
    heq[0] = fma(jj15, rinv, drho);
    n[0] = sub(h[0], heq[0]);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const V cj = c_dot(i, jx, jy, jz);
        const V q = fma(rinv, fma(bc<V>(4.5f), mul(cj, cj), jj15), drho);
        heq[i] = fma(bc<V>(3.f), cj, q);
        heq[i + 1] = fma(bc<V>(-3.f), cj, q);
        n[i] = sub(h[i], heq[i]);
        n[i + 1] = sub(h[i + 1], heq[i + 1]);
    }
    const V a78 = add(n[7], n[8]), a910 = add(n[9], n[10]), a1112 = add(n[11], n[12]);
    const V a1314 = add(n[13], n[14]), a1516 = add(n[15], n[16]), a1718 = add(n[17], n[18]);
    const V exy = add(a78, a910), exz = add(a1112, a1314), eyz = add(a1516, a1718);
    const V pxx = fma(W1, add(n[1], n[2]), mul(W2, add(exy, exz)));
    const V pyy = fma(W1, add(n[3], n[4]), mul(W2, add(exy, eyz)));
    const V pzz = fma(W1, add(n[5], n[6]), mul(W2, add(exz, eyz)));
    const V tr3 = mul(add(add(pxx, pyy), pzz), bc<V>(1.0f / 3.0f));
    V D[6];
    D[0] = sub(pxx, tr3);
    D[1] = sub(pyy, tr3);
    D[2] = sub(pzz, tr3);
    D[3] = sub(a78, a910);
    D[4] = sub(a1112, a1314);
    D[5] = sub(a1516, a1718);
    // k = Dh / w, ie = w / f^eq = 1 / (1 + heq), kr = k ie
    V k[Q], ie[Q], kr[Q];
    k[0] = n[0];
    ie[0] = map(add(one, heq[0]), frcp);
    kr[0] = mul(k[0], ie[0]);
    V A[9];
    V hf = bc<V>(0.f), he = bc<V>(0.f), mf = bc<V>(0.f), me = bc<V>(0.f);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const V Dp = D[p < 3 ? p : 3 + (p - 3) / 2];
        const float ms = p < 3 ? -9.f : ((p - 3) % 2 == 1 ? 0.25f : -0.25f);  // -s / D
        k[i] = fma(Dp, bc<V>(ms), n[i]);
        k[i + 1] = fma(Dp, bc<V>(ms), n[i + 1]);
        ie[i] = map(add(one, heq[i]), frcp);
        ie[i + 1] = map(add(one, heq[i + 1]), frcp);
        kr[i] = mul(k[i], ie[i]);
        kr[i + 1] = mul(k[i + 1], ie[i + 1]);
        A[p] = add(kr[i], kr[i + 1]);
        const V hp = fma(kr[i + 1], k[i + 1], mul(kr[i], k[i]));
        const V mp = fma(mu[i + 1], k[i + 1], mul(mu[i], k[i]));
        if (p < 3) {
            hf = p == 0 ? hp : add(hf, hp);
            mf = p == 0 ? mp : add(mf, mp);
        } else {
            he = p == 3 ? hp : add(he, hp);
            me = p == 3 ? mp : add(me, mp);
        }
    }
    const V sf = fma(D[0], A[0], fma(D[1], A[1], mul(D[2], A[2])));
    const V se = fma(D[3], sub(A[3], A[4]), fma(D[4], sub(A[5], A[6]), mul(D[5], sub(A[7], A[8]))));
    const V sh = fma(bc<V>(0.5f), sf, mul(bc<V>(1.0f / 144.0f), se));
    const V hh = fma(W0, mul(kr[0], k[0]), fma(W1, hf, mul(W2, he)));
    const V mk = fma(W0, mul(mu[0], k[0]), fma(W1, mf, mul(W2, me)));  // mu . Dh
    // ---- gamma and the coefficients of dgamma (R1 = mu.Dh / hh, R2 = sh / hh; zero where inactive)
    const V ihh = map(hh, [](float x) { return x > kHHGuard ? rcp_approx(x) : 0.f; });
    const V R2 = mul(sh, ihh);
    const V R1 = mul(mk, ihh);
    const V gamma = map(hh, R2, [a, b](float x, float r2) { return x > kHHGuard ? fma(-b, r2, a) : 2.0f; });
    const V nbeta = mul(bc<V>(-0.5f * omega), gamma);
    const V c1 = mul(bc<V>(0.5f * omega * b), R1);
    const V c2 = mul(c1, mul(bc<V>(-1.f), R2));
    const V tc2 = mul(bc<V>(2.f), c2);
    const V nom = bc<V>(-omega);
    // ---- coefficient vectors: gh, nq = -(geq) + r, dd = gs - gh (s_i = sd D_c per pair)
    V gh[Q], ng[Q], dd[Q];
    gh[0] = fma(nbeta, mu[0], mul(mul(tc2, k[0]), ie[0]));
    ng[0] = mul(mul(kr[0], ie[0]), mul(c2, k[0]));
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const float sd = p < 3 ? 9.f : ((p - 3) % 2 == 1 ? -0.25f : 0.25f);  // s / D
        const V c1s = mul(c1, mul(bc<V>(sd), D[p < 3 ? p : 3 + (p - 3) / 2]));
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const int j = i + o;
            const V gs = fma(c1, kr[j], mul(nom, mu[j]));
            gh[j] = fma(nbeta, mu[j], mul(fma(tc2, k[j], c1s), ie[j]));
            ng[j] = mul(mul(kr[j], ie[j]), fma(c2, k[j], c1s));
            dd[j] = sub(gs, gh[j]);
        }
    }
    // ---- r = A^T dd + gh through the adjoint second moments
    const V F = add(add(add(dd[1], dd[2]), add(dd[3], dd[4])), add(dd[5], dd[6]));
    const V nf6 = mul(bc<V>(-1.0f / 6.0f), F);
    const V Pxx = fma(bc<V>(0.5f), add(dd[1], dd[2]), nf6);
    const V Pyy = fma(bc<V>(0.5f), add(dd[3], dd[4]), nf6);
    const V Pzz = fma(bc<V>(0.5f), add(dd[5], dd[6]), nf6);
    const V Pxy = mul(bc<V>(0.25f), sub(add(dd[7], dd[8]), add(dd[9], dd[10])));
    const V Pxz = mul(bc<V>(0.25f), sub(add(dd[11], dd[12]), add(dd[13], dd[14])));
    const V Pyz = mul(bc<V>(0.25f), sub(add(dd[15], dd[16]), add(dd[17], dd[18])));
    V r[Q];
    r[0] = gh[0];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        V at;
        if (p == 0) at = Pxx;
        else if (p == 1) at = Pyy;
        else if (p == 2) at = Pzz;
        else if (p < 5) at = p == 3 ? add(add(Pxx, Pyy), Pxy) : sub(add(Pxx, Pyy), Pxy);
        else if (p < 7) at = p == 5 ? add(add(Pxx, Pzz), Pxz) : sub(add(Pxx, Pzz), Pxz);
        else at = p == 7 ? add(add(Pyy, Pzz), Pyz) : sub(add(Pyy, Pzz), Pyz);
        r[i] = add(at, gh[i]);
        r[i + 1] = add(at, gh[i + 1]);
    }
    // ---- equilibrium chain: NQr = sum w nq e, NV = sum w nq (3c + 9 (c.u) c - 3u)
    const V nq0 = add(ng[0], r[0]);
    const V rinv3 = mul(bc<V>(3.f), rinv);
    V qf = mul(nq0, add(one, heq[0]));  // rest term of NQr (weight applied below)
    V ef = bc<V>(0.f), ee = bc<V>(0.f), sgf = bc<V>(0.f), sge = bc<V>(0.f);
    V vf[3], vx = bc<V>(0.f), vy = bc<V>(0.f), vz = bc<V>(0.f);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const V nqa = add(ng[i], r[i]), nqb = add(ng[i + 1], r[i + 1]);
        const V ep = fma(nqb, add(one, heq[i + 1]), mul(nqa, add(one, heq[i])));
        const V sg = add(nqa, nqb);
        const V v = fma(sg, mul(c_dot(i, jx, jy, jz), rinv3), sub(nqa, nqb));
        if (p < 3) {
            ef = p == 0 ? ep : add(ef, ep);
            sgf = p == 0 ? sg : add(sgf, sg);
            vf[p] = v;
        } else {
            ee = p == 3 ? ep : add(ee, ep);
            sge = p == 3 ? sg : add(sge, sg);
            if (cx(i) > 0) vx = add(vx, v);
            if (cy(i) > 0) vy = add(vy, v);
            else if (cy(i) < 0) vy = sub(vy, v);
            if (cz(i) > 0) vz = add(vz, v);
            else if (cz(i) < 0) vz = sub(vz, v);
        }
    }
    const V NQr = fma(W0, qf, fma(W1, ef, mul(W2, ee)));
    const V Swnq = fma(W0, nq0, fma(W1, sgf, mul(W2, sge)));
    const V nrinv = mul(bc<V>(-1.f), rinv);
    const V NVx = mul(bc<V>(3.f), fma(mul(jx, nrinv), Swnq, fma(W1, vf[0], mul(W2, vx))));
    const V NVy = mul(bc<V>(3.f), fma(mul(jy, nrinv), Swnq, fma(W1, vf[1], mul(W2, vy))));
    const V NVz = mul(bc<V>(3.f), fma(mul(jz, nrinv), Swnq, fma(W1, vf[2], mul(W2, vz))));
    // base = NV . u - NQr / rho,  u = j / rho
    const V base = fma(rinv, fma(NVx, jx, fma(NVy, jy, mul(NVz, jz))), mul(NQr, nrinv));
    lam[0] = add(add(mu[0], r[0]), base);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const V cN = c_dot(i, NVx, NVy, NVz);
        lam[i] = add(add(mu[i], r[i]), sub(base, cN));
        lam[i + 1] = add(add(mu[i + 1], r[i + 1]), add(base, cN));
    }
}

#else  // MCLBM_D3Q27

// D3Q27 form of the paired product: the operations of the D3Q19 form above with the 13 pairs
// (faces p = 0..2, edges 3..8, corners 9..12 with zero shear part), the D3Q27 weights, the
// corners in P_ab and in the equilibrium chain, and (A^T v)_j = Pxx + Pyy + Pzz + sum_{a<b}
// c_ja c_jb P_ab on the corners.  To keep 27 pairs of values from exhausting the registers the
// coefficients are written through kr_j = k_j / (1 + heq_j) (k dies after the forward sums):
// gh_j = -beta mu_j + 2 c2 kr_j + c1s_j ie_j, ng_j = kr_j (c2 kr_j + c1s_j ie_j), and each
// velocity keeps only u_j = mu_j + gh_j (for lambda) and v_j = ng_j + gh_j (for the chain).
template <class V, class Ar = lanes::Asm>
__device__ __forceinline__ void kbc_vjp_shifted(const V (&h)[Q], const V (&mu)[Q], float omega, float a, float b,
                                                V (&lam)[Q])
{
    using lanes::bc;
    using lanes::map;
    using lanes::rcp_approx;
    const auto add = [](auto x, auto y) { return Ar::add(x, y); };
    const auto mul = [](auto x, auto y) { return Ar::mul(x, y); };
    const auto fma = [](auto x, auto y, auto z) { return Ar::fma(x, y, z); };
    const auto sub = [](auto x, auto y) { return Ar::sub(x, y); };
    const V one = bc<V>(1.f);
    const V W0 = bc<V>(8.0f / 27.0f), W1 = bc<V>(2.0f / 27.0f), W2 = bc<V>(1.0f / 54.0f), W3 = bc<V>(1.0f / 216.0f);
    const auto frcp = [](float x) { return rcp_approx(x); };
    // ---- forward, as the D3Q27 kbc_shifted
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
    V eh[Q], n[Q];  // eh = 1 + heq
    {
        const V heq0 = fma(jj15, rinv, drho);
        eh[0] = add(one, heq0);
        n[0] = sub(h[0], heq0);
    }
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        const V cj = c_dot<V, Ar>(i, jx, jy, jz);
        const V q = fma(rinv, fma(bc<V>(4.5f), mul(cj, cj), jj15), drho);
        const V ha = fma(bc<V>(3.f), cj, q), hb = fma(bc<V>(-3.f), cj, q);
        eh[i] = add(one, ha);
        eh[i + 1] = add(one, hb);
        n[i] = sub(h[i], ha);
        n[i + 1] = sub(h[i + 1], hb);
    }
    V Ap[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) Ap[p] = add(n[2 * p + 1], n[2 * p + 2]);
    const V exy = add(Ap[3], Ap[4]), exz = add(Ap[5], Ap[6]), eyz = add(Ap[7], Ap[8]);
    const V csum = add(add(Ap[9], Ap[10]), add(Ap[11], Ap[12]));
    const V cxy = sub(add(Ap[9], Ap[10]), add(Ap[11], Ap[12]));
    const V cxz = add(sub(Ap[9], Ap[10]), sub(Ap[11], Ap[12]));
    const V cyz = sub(sub(Ap[9], Ap[10]), sub(Ap[11], Ap[12]));
    const V pxx = fma(W1, Ap[0], fma(W2, add(exy, exz), mul(W3, csum)));
    const V pyy = fma(W1, Ap[1], fma(W2, add(exy, eyz), mul(W3, csum)));
    const V pzz = fma(W1, Ap[2], fma(W2, add(exz, eyz), mul(W3, csum)));
    const V tr3 = mul(add(add(pxx, pyy), pzz), bc<V>(1.0f / 3.0f));
    V D[6];
    D[0] = sub(pxx, tr3);
    D[1] = sub(pyy, tr3);
    D[2] = sub(pzz, tr3);
    D[3] = fma(W2, sub(Ap[3], Ap[4]), mul(W3, cxy));
    D[4] = fma(W2, sub(Ap[5], Ap[6]), mul(W3, cxz));
    D[5] = fma(W2, sub(Ap[7], Ap[8]), mul(W3, cyz));
    // k = Dh / w (in n), ie = 1 / (1 + heq), kr = k ie
    V ie[Q], kr[Q];
    ie[0] = map(eh[0], frcp);
    kr[0] = mul(n[0], ie[0]);
    V A[9];
    V hf = bc<V>(0.f), he = bc<V>(0.f), hc = bc<V>(0.f), mf = bc<V>(0.f), me = bc<V>(0.f), mc = bc<V>(0.f);
    const V hh0 = mul(kr[0], n[0]), mk0 = mul(mu[0], n[0]);
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        if (p < 9) {
            const V Dp = D[p < 3 ? p : 3 + (p - 3) / 2];
            const float ms = p < 3 ? -6.75f : ((p - 3) % 2 == 1 ? 13.5f : -13.5f);  // -s / D
            n[i] = fma(Dp, bc<V>(ms), n[i]);
            n[i + 1] = fma(Dp, bc<V>(ms), n[i + 1]);
        }
        ie[i] = map(eh[i], frcp);
        ie[i + 1] = map(eh[i + 1], frcp);
        kr[i] = mul(n[i], ie[i]);
        kr[i + 1] = mul(n[i + 1], ie[i + 1]);
        if (p < 9) A[p] = add(kr[i], kr[i + 1]);
        const V hp = fma(kr[i + 1], n[i + 1], mul(kr[i], n[i]));
        const V mp = fma(mu[i + 1], n[i + 1], mul(mu[i], n[i]));
        if (p < 3) {
            hf = p == 0 ? hp : add(hf, hp);
            mf = p == 0 ? mp : add(mf, mp);
        } else if (p < 9) {
            he = p == 3 ? hp : add(he, hp);
            me = p == 3 ? mp : add(me, mp);
        } else {
            hc = p == 9 ? hp : add(hc, hp);
            mc = p == 9 ? mp : add(mc, mp);
        }
    }
    // sh: w1 6.75 = 1/2, w2 13.5 = 1/4
    const V sf = fma(D[0], A[0], fma(D[1], A[1], mul(D[2], A[2])));
    const V se = fma(D[3], sub(A[3], A[4]), fma(D[4], sub(A[5], A[6]), mul(D[5], sub(A[7], A[8]))));
    const V sh = fma(bc<V>(0.5f), sf, mul(bc<V>(0.25f), se));
    const V hh = fma(W0, hh0, fma(W1, hf, fma(W2, he, mul(W3, hc))));
    const V mk = fma(W0, mk0, fma(W1, mf, fma(W2, me, mul(W3, mc))));  // mu . Dh
    const V ihh = map(hh, [](float x) { return x > kHHGuard ? rcp_approx(x) : 0.f; });
    const V R2 = mul(sh, ihh);
    const V R1 = mul(mk, ihh);
    const V gamma = map(hh, R2, [a, b, fma](float x, float r2) { return x > kHHGuard ? fma(-b, r2, a) : 2.0f; });
    const V nbeta = mul(bc<V>(-0.5f * omega), gamma);
    const V c1 = mul(bc<V>(0.5f * omega * b), R1);
    const V c2 = mul(c1, mul(bc<V>(-1.f), R2));
    const V tc2 = mul(bc<V>(2.f), c2);
    const V gsd = sub(bc<V>(-omega), nbeta);  // gs - gh = (-omega + beta) mu + (c1 - 2 c2) kr - c1s ie
    const V ktd = sub(c1, tc2);
    // ---- per velocity: dd (faces and edges), u = mu + gh, v = ng + gh (corners: s = 0)
    V u[Q], v[Q], dd[19];
    {
        const V g0 = fma(nbeta, mu[0], mul(tc2, kr[0]));
        u[0] = add(mu[0], g0);
        v[0] = fma(kr[0], mul(c2, kr[0]), g0);
    }
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        if (p < 9) {
            const float sd = p < 3 ? 6.75f : ((p - 3) % 2 == 1 ? -13.5f : 13.5f);  // s / D
            const V c1s = mul(c1, mul(bc<V>(sd), D[p < 3 ? p : 3 + (p - 3) / 2]));
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int j = i + o;
                const V si = mul(c1s, ie[j]);
                const V g = fma(nbeta, mu[j], fma(tc2, kr[j], si));
                dd[j] = fma(gsd, mu[j], fma(ktd, kr[j], mul(bc<V>(-1.f), si)));
                u[j] = add(mu[j], g);
                v[j] = fma(kr[j], fma(c2, kr[j], si), g);
            }
        } else {
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int j = i + o;
                const V g = fma(nbeta, mu[j], mul(tc2, kr[j]));
                u[j] = add(mu[j], g);
                v[j] = fma(kr[j], mul(c2, kr[j]), g);
            }
        }
    }
    // ---- adjoint second moments from dd (faces and edges)
    const V F = add(add(add(dd[1], dd[2]), add(dd[3], dd[4])), add(dd[5], dd[6]));
    const V nf6 = mul(bc<V>(-1.0f / 6.0f), F);
    const V Pxx = fma(bc<V>(0.5f), add(dd[1], dd[2]), nf6);
    const V Pyy = fma(bc<V>(0.5f), add(dd[3], dd[4]), nf6);
    const V Pzz = fma(bc<V>(0.5f), add(dd[5], dd[6]), nf6);
    const V Pxy = mul(bc<V>(0.25f), sub(add(dd[7], dd[8]), add(dd[9], dd[10])));
    const V Pxz = mul(bc<V>(0.25f), sub(add(dd[11], dd[12]), add(dd[13], dd[14])));
    const V Pyz = mul(bc<V>(0.25f), sub(add(dd[15], dd[16]), add(dd[17], dd[18])));
    const V Pd3 = add(add(Pxx, Pyy), Pzz);
    const auto at_of = [&](int p) -> V {
        const int i = 2 * p + 1;
        if (p == 0) return Pxx;
        if (p == 1) return Pyy;
        if (p == 2) return Pzz;
        if (p < 5) return p == 3 ? add(add(Pxx, Pyy), Pxy) : sub(add(Pxx, Pyy), Pxy);
        if (p < 7) return p == 5 ? add(add(Pxx, Pzz), Pxz) : sub(add(Pxx, Pzz), Pxz);
        if (p < 9) return p == 7 ? add(add(Pyy, Pzz), Pyz) : sub(add(Pyy, Pzz), Pyz);
        V at = cx(i) * cy(i) > 0 ? add(Pd3, Pxy) : sub(Pd3, Pxy);
        at = cx(i) * cz(i) > 0 ? add(at, Pxz) : sub(at, Pxz);
        return cy(i) * cz(i) > 0 ? add(at, Pyz) : sub(at, Pyz);
    };
    // ---- equilibrium chain on nq = ng + r = v + A^T dd
    const V nq0 = v[0];
    const V rinv3 = mul(bc<V>(3.f), rinv);
    const V qf = mul(nq0, eh[0]);
    V ef = bc<V>(0.f), ee = bc<V>(0.f), ec = bc<V>(0.f), sgf = bc<V>(0.f), sge = bc<V>(0.f), sgc = bc<V>(0.f);
    V vf[3], vx = bc<V>(0.f), vy = bc<V>(0.f), vz = bc<V>(0.f), ux3 = bc<V>(0.f), uy3 = bc<V>(0.f), uz3 = bc<V>(0.f);
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        const V at = at_of(p);
        const V nqa = add(v[i], at), nqb = add(v[i + 1], at);
        const V ep = fma(nqb, eh[i + 1], mul(nqa, eh[i]));
        const V sg = add(nqa, nqb);
        const V w = fma(sg, mul(c_dot<V, Ar>(i, jx, jy, jz), rinv3), sub(nqa, nqb));
        if (p < 3) {
            ef = p == 0 ? ep : add(ef, ep);
            sgf = p == 0 ? sg : add(sgf, sg);
            vf[p] = w;
        } else if (p < 9) {
            ee = p == 3 ? ep : add(ee, ep);
            sge = p == 3 ? sg : add(sge, sg);
            if (cx(i) > 0) vx = add(vx, w);
            if (cy(i) > 0) vy = add(vy, w);
            else if (cy(i) < 0) vy = sub(vy, w);
            if (cz(i) > 0) vz = add(vz, w);
            else if (cz(i) < 0) vz = sub(vz, w);
        } else {
            ec = p == 9 ? ep : add(ec, ep);
            sgc = p == 9 ? sg : add(sgc, sg);
            ux3 = add(ux3, w);  // every corner has c_x = +1 on its odd member
            uy3 = cy(i) > 0 ? add(uy3, w) : sub(uy3, w);
            uz3 = cz(i) > 0 ? add(uz3, w) : sub(uz3, w);
        }
    }
    const V NQr = fma(W0, qf, fma(W1, ef, fma(W2, ee, mul(W3, ec))));
    const V Swnq = fma(W0, nq0, fma(W1, sgf, fma(W2, sge, mul(W3, sgc))));
    const V nrinv = mul(bc<V>(-1.f), rinv);
    const V NVx = mul(bc<V>(3.f), fma(mul(jx, nrinv), Swnq, fma(W1, vf[0], fma(W2, vx, mul(W3, ux3)))));
    const V NVy = mul(bc<V>(3.f), fma(mul(jy, nrinv), Swnq, fma(W1, vf[1], fma(W2, vy, mul(W3, uy3)))));
    const V NVz = mul(bc<V>(3.f), fma(mul(jz, nrinv), Swnq, fma(W1, vf[2], fma(W2, vz, mul(W3, uz3)))));
    const V base = fma(rinv, fma(NVx, jx, fma(NVy, jy, mul(NVz, jz))), mul(NQr, nrinv));
    // lambda = mu + r + base - c . NV with mu + r = u + A^T dd
    lam[0] = add(u[0], base);
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int i = 2 * p + 1;
        const V at = at_of(p);
        const V cN = c_dot<V, Ar>(i, NVx, NVy, NVz);
        lam[i] = add(add(u[i], at), sub(base, cN));
        lam[i + 1] = add(add(u[i + 1], at), add(base, cN));
    }
}

#endif  // MCLBM_D3Q27

}  // namespace mclbm
