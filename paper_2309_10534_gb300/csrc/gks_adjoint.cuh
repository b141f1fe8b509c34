// gks_adjoint.cuh -- reverse-mode (vector-Jacobian) counterparts of the
// per-point arithmetic in gks_device.cuh, written out by hand.
//
// Scope: the collision-free interface flux (tau = 0, the setting of the
// paper's smooth-flow tests, Sec. 5.1 and 5.5) in 2-D: the kinetic merge of
// the two reconstructed sides into the equilibrium state and its slopes
// (Eqs. 2.6, 3.25, 3.26), the Euler flux of that state and its time
// derivative from the compatibility condition (Sec. 2.2).  TENO-D is taken
// with the stencil selection of the forward pass held fixed: once the
// selection (large stencil, or which small stencils with weights 1/3) is
// fixed, every reconstructed value and slope is a linear function of the
// five cell averages, and its transpose is below.
//
// Convention: a function named *_vjp adds, to the g* outputs, the product of
// the transposed Jacobian of the forward function with the given cotangents
// of the forward outputs; it recomputes what it needs of the forward values.
#pragma once

#include "gks_device.cuh"

namespace gks {

// ------------------------------------------------------------------ TENO-D, frozen selection
// transpose of the quadratic coefficients b_k, c_k of teno_select
template <typename T>
GKS_HD void teno_bc_T(const T* gb, const T* gc, T* gq)
{
    // b0 = (q0 - 4 q1 + 3 q2)/2, c0 = (q0 - 2 q1 + q2)/2
    gq[0] += T(0.5) * (gb[0] + gc[0]);
    gq[1] += T(-2) * gb[0] - gc[0];
    gq[2] += T(1.5) * gb[0] + T(0.5) * gc[0];
    // b1 = (q3 - q1)/2, c1 = (q1 - 2 q2 + q3)/2
    gq[1] += T(0.5) * (gc[1] - gb[1]);
    gq[2] -= gc[1];
    gq[3] += T(0.5) * (gb[1] + gc[1]);
    // b2 = (-3 q2 + 4 q3 - q4)/2, c2 = (q2 - 2 q3 + q4)/2
    gq[2] += T(-1.5) * gb[2] + T(0.5) * gc[2];
    gq[3] += T(2) * gb[2] - gc[2];
    gq[4] += T(0.5) * (gc[2] - gb[2]);
}

// transpose of the quartic's Legendre-type coefficients u1..u4 of teno_select
template <typename T>
GKS_HD void teno_u_T(T gu1, T gu2, T gu3, T gu4, T* gq)
{
    const T a = gu1 * T(1.0 / 120.0), b = gu2 * T(1.0 / 56.0), c = gu3 * T(1.0 / 12.0), d = gu4 * T(1.0 / 24.0);
    gq[0] += T(11) * a - T(3) * b - c + d;
    gq[1] += T(-82) * a + T(40) * b + T(2) * c - T(4) * d;
    gq[2] += T(-74) * b + T(6) * d;
    gq[3] += T(82) * a + T(40) * b - T(2) * c - T(4) * d;
    gq[4] += T(-11) * a - T(3) * b + c + d;
}

// transpose of teno_faces: cotangents of (vp, dp, vm, dm), added to gq[0..4]
template <typename T>
GKS_HD void teno_faces_T(const TenoSel<T>& S, T gvp, T gdp, T gvm, T gdm, T* gq)
{
    if (S.large) {  // Eqs. (4.8), (4.9) and their mirror
        gq[0] += (T(2) * gvp - T(3) * gvm) * T(1.0 / 60.0) + gdm * T(1.0 / 12.0);
        gq[1] += (T(-13) * gvp + T(27) * gvm) * T(1.0 / 60.0) + (gdp - T(15) * gdm) * T(1.0 / 12.0);
        gq[2] += T(47) * (gvp + gvm) * T(1.0 / 60.0) + T(15) * (gdm - gdp) * T(1.0 / 12.0);
        gq[3] += (T(27) * gvp - T(13) * gvm) * T(1.0 / 60.0) + (T(15) * gdp - gdm) * T(1.0 / 12.0);
        gq[4] += (T(-3) * gvp + T(2) * gvm) * T(1.0 / 60.0) - gdp * T(1.0 / 12.0);
        return;
    }
    // vp = q2 + sum w (b/2 + c/6), vm = q2 + sum w (c/6 - b/2),
    // dp = sum w (b + c), dm = sum w (b - c)
    const T sb = T(0.5) * (gvp - gvm) + gdp + gdm;
    const T sc = (gvp + gvm) * T(1.0 / 6.0) + gdp - gdm;
    T gb[3], gc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gb[k] = S.w[k] * sb;
        gc[k] = S.w[k] * sc;
    }
    gq[2] += gvp + gvm;
    teno_bc_T(gb, gc, gq);
}

// transpose of teno_gauss at xi = g: cotangents of (v, d), added to gq[0..4]
template <typename T>
GKS_HD void teno_gauss_T(const TenoSel<T>& S, T g, T gv, T gd, T* gq)
{
    gq[2] += gv;
    if (S.large) {
        // v = q2 + u1 g - u3 g/15 - u4/180, d = u1 + 2 u2 g + u3/10 - (2/21) u4 g
        teno_u_T(g * gv + gd, T(2) * g * gd, g * gv * T(-1.0 / 15.0) + T(0.1) * gd,
                 gv * T(-1.0 / 180.0) - T(2.0 / 21.0) * g * gd, gq);
        return;
    }
    // v = q2 + sum w b g, d = sum w (b + 2 c g)
    T gb[3], gc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gb[k] = S.w[k] * (g * gv + gd);
        gc[k] = S.w[k] * T(2) * g * gd;
    }
    teno_bc_T(gb, gc, gq);
}

// ------------------------------------------------------------------ kinetic layer (2-D)
// euler_jvp's dF = (dF/dW)(U, V, h) d: adds (dF/dW)^T y to gd and the
// derivatives with respect to U, V, h to gU, gV, gh
template <typename T>
GKS_HD void euler_jvpF_vjp(const T* d, T U, T V, T h, T gm1, const T* y, T* gd, T& gU, T& gV, T& gh)
{
    const T q = T(0.5) * (U * U + V * V);
    const T dp = gm1 * (d[3] - U * d[1] - V * d[2] + q * d[0]);
    // dF0 = d1, dF1 = 2 U d1 - U^2 d0 + dp, dF2 = cross, dF3 = U (d3 + dp) + h (d1 - U d0)
    const T gdp = y[1] + U * y[3];
    const T gcross = y[2];
    gd[1] += y[0] + T(2) * U * y[1] + h * y[3];
    gd[0] += -U * U * y[1] - h * U * y[3];
    gd[3] += U * y[3];
    gU += T(2) * (d[1] - U * d[0]) * y[1] + (d[3] + dp - h * d[0]) * y[3];
    gh += (d[1] - U * d[0]) * y[3];
    // cross = V d1 + U d2 - U V d0
    gd[1] += V * gcross;
    gd[2] += U * gcross;
    gd[0] += -U * V * gcross;
    gU += (d[2] - V * d[0]) * gcross;
    gV += (d[1] - U * d[0]) * gcross;
    // dp = gm1 (d3 - U d1 - V d2 + q d0)
    const T gg = gm1 * gdp;
    gd[3] += gg;
    gd[1] -= U * gg;
    gd[2] -= V * gg;
    gd[0] += q * gg;
    gU += (U * d[0] - d[1]) * gg;
    gV += (V * d[0] - d[2]) * gg;
}

// the same for euler_jvp's dG (tangential flux)
template <typename T>
GKS_HD void euler_jvpG_vjp(const T* d, T U, T V, T h, T gm1, const T* y, T* gd, T& gU, T& gV, T& gh)
{
    const T q = T(0.5) * (U * U + V * V);
    const T dp = gm1 * (d[3] - U * d[1] - V * d[2] + q * d[0]);
    // dG0 = d2, dG1 = cross, dG2 = 2 V d2 - V^2 d0 + dp, dG3 = V (d3 + dp) + h (d2 - V d0)
    const T gdp = y[2] + V * y[3];
    const T gcross = y[1];
    gd[2] += y[0] + T(2) * V * y[2] + h * y[3];
    gd[0] += -V * V * y[2] - h * V * y[3];
    gd[3] += V * y[3];
    gV += T(2) * (d[2] - V * d[0]) * y[2] + (d[3] + dp - h * d[0]) * y[3];
    gh += (d[2] - V * d[0]) * y[3];
    gd[1] += V * gcross;
    gd[2] += U * gcross;
    gd[0] += -U * V * gcross;
    gU += (d[2] - V * d[0]) * gcross;
    gV += (d[1] - U * d[0]) * gcross;
    const T gg = gm1 * gdp;
    gd[3] += gg;
    gd[1] -= U * gg;
    gd[2] -= V * gg;
    gd[0] += q * gg;
    gU += (U * d[0] - d[1]) * gg;
    gV += (V * d[0] - d[2]) * gg;
}

// micro_slope (closed-form solve of Eq. 2.7): cotangent ga of a -> gb, gU,
// gV, glam, ginv2l
template <typename T>
GKS_HD void micro_slope_vjp(const T* b, T U, T V, T lam, T inv2l, T ntot, T inv_ntot, const T* ga, T* gb, T& gU,
                            T& gV, T& glam, T& ginv2l)
{
    const T E = T(0.5) * (U * U + V * V + ntot * inv2l);
    const T R2 = b[1] - U * b[0];
    const T R3 = b[2] - V * b[0];
    const T R4 = T(2) * (b[3] - E * b[0]);
    const T tl = T(2) * lam;
    const T X = R4 - T(2) * U * R2 - T(2) * V * R3;
    const T a3 = tl * tl * inv_ntot * X;
    const T a2 = tl * R3 - V * a3;
    const T a1 = tl * R2 - U * a3;
    // a0 = b0 - U a1 - V a2 - E a3
    T ga1 = ga[1] - U * ga[0], ga2 = ga[2] - V * ga[0], ga3 = ga[3] - E * ga[0];
    gb[0] += ga[0];
    gU -= a1 * ga[0];
    gV -= a2 * ga[0];
    T gE = -a3 * ga[0];
    // a1 = tl R2 - U a3, a2 = tl R3 - V a3
    T gtl = R2 * ga1 + R3 * ga2;
    T gR2 = tl * ga1, gR3 = tl * ga2;
    gU -= a3 * ga1;
    gV -= a3 * ga2;
    ga3 -= U * ga1 + V * ga2;
    // a3 = tl^2 inv_ntot X
    gtl += T(2) * tl * inv_ntot * X * ga3;
    const T gX = tl * tl * inv_ntot * ga3;
    const T gR4 = gX;
    gU -= T(2) * R2 * gX;
    gR2 -= T(2) * U * gX;
    gV -= T(2) * R3 * gX;
    gR3 -= T(2) * V * gX;
    // R4 = 2 (b3 - E b0), R3 = b2 - V b0, R2 = b1 - U b0
    gb[3] += T(2) * gR4;
    gE -= T(2) * b[0] * gR4;
    gb[0] -= T(2) * E * gR4 + V * gR3 + U * gR2;
    gb[2] += gR3;
    gV -= b[0] * gR3;
    gb[1] += gR2;
    gU -= b[0] * gR2;
    // E, tl
    gU += U * gE;
    gV += V * gE;
    ginv2l += T(0.5) * ntot * gE;
    glam += T(2) * gtl;
}

// o = H a (hmv): cotangent go -> gH (10 unique entries), ga
template <typename T>
GKS_HD void hmv_vjp(const T* H, const T* a, const T* go, T* gH, T* ga)
{
    gH[0] += a[0] * go[0];
    gH[1] += a[1] * go[0] + a[0] * go[1];
    gH[2] += a[2] * go[0] + a[0] * go[2];
    gH[3] += a[3] * go[0] + a[0] * go[3];
    gH[4] += a[1] * go[1];
    gH[5] += a[2] * go[1] + a[1] * go[2];
    gH[6] += a[3] * go[1] + a[1] * go[3];
    gH[7] += a[2] * go[2];
    gH[8] += a[3] * go[2] + a[2] * go[3];
    gH[9] += a[3] * go[3];
    ga[0] += H[0] * go[0] + H[1] * go[1] + H[2] * go[2] + H[3] * go[3];
    ga[1] += H[1] * go[0] + H[4] * go[1] + H[5] * go[2] + H[6] * go[3];
    ga[2] += H[2] * go[0] + H[5] * go[1] + H[7] * go[2] + H[8] * go[3];
    ga[3] += H[3] * go[0] + H[6] * go[1] + H[8] * go[2] + H[9] * go[3];
}

// hmat<0,0> (2-D): cotangent gH -> gu[0..4], gv[1..4], gxi2, gxi4 (v[0] = 1)
template <typename T>
GKS_HD void hmat00_vjp(const T* u, const T* v, T xi2, T xi4, const T* H, const T* gH, T* gu, T* gv, T& gxi2,
                       T& gxi4)
{
    T g0 = gH[0], g1 = gH[1], g2 = gH[2], g4 = gH[4], g7 = gH[7];
    // H9 = (u4 + u0 v4 + H0 xi4 + 2 (u2 v2 + (H4 + H7) xi2)) / 4
    const T q9 = T(0.25) * gH[9];
    gu[4] += q9;
    gu[0] += v[4] * q9;
    gv[4] += u[0] * q9;
    g0 += xi4 * q9;
    gxi4 += H[0] * q9;
    gu[2] += T(2) * v[2] * q9;
    gv[2] += T(2) * u[2] * q9;
    g4 += T(2) * xi2 * q9;
    g7 += T(2) * xi2 * q9;
    gxi2 += T(2) * (H[4] + H[7]) * q9;
    // H8 = (u2 v1 + u0 v3 + H2 xi2) / 2
    const T q8 = T(0.5) * gH[8];
    gu[2] += v[1] * q8;
    gv[1] += u[2] * q8;
    gu[0] += v[3] * q8;
    gv[3] += u[0] * q8;
    g2 += xi2 * q8;
    gxi2 += H[2] * q8;
    // H6 = (u3 + u1 v2 + H1 xi2) / 2
    const T q6 = T(0.5) * gH[6];
    gu[3] += q6;
    gu[1] += v[2] * q6;
    gv[2] += u[1] * q6;
    g1 += xi2 * q6;
    gxi2 += H[1] * q6;
    // H3 = (H4 + H7 + H0 xi2) / 2
    const T q3 = T(0.5) * gH[3];
    g4 += q3;
    g7 += q3;
    g0 += xi2 * q3;
    gxi2 += H[0] * q3;
    // H7 = u0 v2, H5 = u1 v1, H4 = u2, H2 = u0 v1, H1 = u1, H0 = u0
    gu[0] += v[2] * g7 + v[1] * g2 + g0;
    gv[2] += u[0] * g7;
    gu[1] += v[1] * gH[5] + g1;
    gv[1] += u[1] * gH[5] + u[0] * g2;
    gu[2] += g4;
}

// Reverse of side_terms (NONEQ = false, 2-D): cotangents of the side's
// contributions to W0, W0_n, W0_t -> cotangents of the side's W, Wn, Wt
// (added to gS).
template <typename T>
GKS_HD void side_vjp(const Side<T>& S, bool upper, const FluxParams<T>& P, const T* gW0, const T* gW0n,
                     const T* gW0t, Side<T>& gS)
{
    // ---- forward values
    const T r = S.W[0], ir = T(1) / r;
    const T U = S.W[1] * ir, V = S.W[2] * ir;
    const T p = P.gm1 * (S.W[3] - T(0.5) * r * (U * U + V * V));
    const T inv2l = p * ir;
    const T lam = T(0.5) / inv2l;
    const T sl = M<T>::sqrt_(lam);
    const T xi2 = P.K * inv2l, xi4 = P.K * (P.K + T(2)) * inv2l * inv2l;
    const T sg = upper ? T(1) : T(-1);
    const T z = sl * U;
    T u[5], v[5], h0, g;
    half_space_start<T>(z, sg, h0, g);
    const T c = T(0.28209479177387814);  // 1 / (2 sqrt(pi))
    u[0] = h0;
    u[1] = U * h0 + sg * c * g / sl;
#pragma unroll
    for (int n = 0; n < 3; ++n) u[n + 2] = U * u[n + 1] + T(n + 1) * inv2l * u[n];
    v[0] = T(1);
    v[1] = V;
#pragma unroll
    for (int n = 0; n < 3; ++n) v[n + 2] = V * v[n + 1] + T(n + 1) * inv2l * v[n];
    T bn[4], bt[4], an[4], at[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        bn[i] = S.Wn[i] * ir;
        bt[i] = S.Wt[i] * ir;
    }
    micro_slope<T, 2>(bn, U, V, lam, inv2l, P.ntot, P.inv_ntot, an);
    micro_slope<T, 2>(bt, U, V, lam, inv2l, P.ntot, P.inv_ntot, at);
    T H[10], tn[4], tt[4];
    hmat<0, 0, T, 2>(u, v, xi2, xi4, H);
    hmv<T, 2>(H, an, tn);
    hmv<T, 2>(H, at, tt);

    // ---- reverse: W0 += r H[0..3], W0n += r H an, W0t += r H at
    T gr = T(0), gH[10], gtn[4], gtt[4], gan[4] = {T(0), T(0), T(0), T(0)}, gat[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 10; ++i) gH[i] = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        gr += H[i] * gW0[i] + tn[i] * gW0n[i] + tt[i] * gW0t[i];
        gH[i] = r * gW0[i];
        gtn[i] = r * gW0n[i];
        gtt[i] = r * gW0t[i];
    }
    hmv_vjp(H, an, gtn, gH, gan);
    hmv_vjp(H, at, gtt, gH, gat);
    T gU = T(0), gV = T(0), glam = T(0), ginv2l = T(0);
    T gbn[4] = {T(0), T(0), T(0), T(0)}, gbt[4] = {T(0), T(0), T(0), T(0)};
    micro_slope_vjp(bn, U, V, lam, inv2l, P.ntot, P.inv_ntot, gan, gbn, gU, gV, glam, ginv2l);
    micro_slope_vjp(bt, U, V, lam, inv2l, P.ntot, P.inv_ntot, gat, gbt, gU, gV, glam, ginv2l);
    T gu[5] = {T(0), T(0), T(0), T(0), T(0)}, gv[5] = {T(0), T(0), T(0), T(0), T(0)};
    T gxi2 = T(0), gxi4 = T(0);
    hmat00_vjp(u, v, xi2, xi4, H, gH, gu, gv, gxi2, gxi4);
    // v recursion: v_{n+2} = V v_{n+1} + (n+1) inv2l v_n
#pragma unroll
    for (int n = 2; n >= 0; --n) {
        gV += v[n + 1] * gv[n + 2];
        gv[n + 1] += V * gv[n + 2];
        ginv2l += T(n + 1) * v[n] * gv[n + 2];
        gv[n] += T(n + 1) * inv2l * gv[n + 2];
    }
    gV += gv[1];
    // u recursion, then u1 = U h0 + sg c g / sl, u0 = h0
#pragma unroll
    for (int n = 2; n >= 0; --n) {
        gU += u[n + 1] * gu[n + 2];
        gu[n + 1] += U * gu[n + 2];
        ginv2l += T(n + 1) * u[n] * gu[n + 2];
        gu[n] += T(n + 1) * inv2l * gu[n + 2];
    }
    gU += h0 * gu[1];
    const T gh0 = gu[0] + U * gu[1];
    const T isl = T(1) / sl;
    const T gg = sg * c * isl * gu[1];
    T gsl = -sg * c * g * isl * isl * gu[1];
    // g = exp(-z^2); h0 = erfc(-sg z)/2, d h0/dz = sg exp(-z^2)/sqrt(pi)
    const T gz = -T(2) * z * g * gg + sg * g * T(0.56418958354775628) * gh0;
    gsl += U * gz;
    gU += sl * gz;
    // xi2 = K inv2l, xi4 = K (K+2) inv2l^2; sl = sqrt(lam); lam = 1/(2 inv2l)
    ginv2l += P.K * gxi2 + T(2) * P.K * (P.K + T(2)) * inv2l * gxi4;
    glam += T(0.5) * isl * gsl;
    ginv2l -= lam / inv2l * glam;
    // b = W_{n,t} / r
    T gir = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        gS.Wn[i] += ir * gbn[i];
        gS.Wt[i] += ir * gbt[i];
        gir += S.Wn[i] * gbn[i] + S.Wt[i] * gbt[i];
    }
    // inv2l = p / r; p = gm1 (W3 - r (U^2 + V^2)/2); U = W1/r, V = W2/r
    const T gp = ir * ginv2l;
    gir += p * ginv2l;
    gS.W[3] += P.gm1 * gp;
    gr -= T(0.5) * P.gm1 * (U * U + V * V) * gp;
    gU -= P.gm1 * r * U * gp;
    gV -= P.gm1 * r * V * gp;
    gS.W[1] += ir * gU;
    gS.W[2] += ir * gV;
    gir += S.W[1] * gU + S.W[2] * gV;
    gr -= ir * ir * gir;
    gS.W[0] += gr;
}

// Reverse of the equilibrium part of point_flux for tau = 0 (2-D):
// F = F0 (Euler flux of W0), dF = (dF/dW)(W0) W0_time with
// W0_time = -((dF/dW) W0_n + (dG/dW) W0_t).
template <typename T>
GKS_HD void equilibrium_vjp(const T* W0, const T* W0n, const T* W0t, T gm1, const T* gF, const T* gdF, T* gW0,
                            T* gW0n, T* gW0t)
{
    const T r0 = W0[0], ir0 = T(1) / r0;
    const T U0 = W0[1] * ir0, V0 = W0[2] * ir0;
    const T p0 = gm1 * (W0[3] - T(0.5) * r0 * (U0 * U0 + V0 * V0));
    const T h0 = (W0[3] + p0) * ir0;
    T X[4], Y[4], Wtime[4];
    euler_jvp<T, 2>(W0n, U0, V0, h0, gm1, X, nullptr);
    euler_jvp<T, 2>(W0t, U0, V0, h0, gm1, nullptr, Y);
#pragma unroll
    for (int i = 0; i < 4; ++i) Wtime[i] = -(X[i] + Y[i]);
    T gU = T(0), gV = T(0), gh = T(0), gWt[4] = {T(0), T(0), T(0), T(0)};
    euler_jvpF_vjp(Wtime, U0, V0, h0, gm1, gdF, gWt, gU, gV, gh);
#pragma unroll
    for (int i = 0; i < 4; ++i) gWt[i] = -gWt[i];
    euler_jvpF_vjp(W0n, U0, V0, h0, gm1, gWt, gW0n, gU, gV, gh);
    euler_jvpG_vjp(W0t, U0, V0, h0, gm1, gWt, gW0t, gU, gV, gh);
    // F0 = (W1, W1 U0 + p0, W1 V0, U0 (W3 + p0))
    T gp = gF[1] + U0 * gF[3];
    gW0[1] += gF[0] + U0 * gF[1] + V0 * gF[2];
    gU += W0[1] * gF[1] + (W0[3] + p0) * gF[3];
    gV += W0[1] * gF[2];
    gW0[3] += U0 * gF[3];
    // h0 = (W3 + p0) / r0
    gW0[3] += ir0 * gh;
    gp += ir0 * gh;
    T gir = (W0[3] + p0) * gh;
    // p0 = gm1 (W3 - r0 (U0^2 + V0^2)/2)
    gW0[3] += gm1 * gp;
    T gr = -T(0.5) * gm1 * (U0 * U0 + V0 * V0) * gp;
    gU -= gm1 * r0 * U0 * gp;
    gV -= gm1 * r0 * V0 * gp;
    // U0 = W1 / r0, V0 = W2 / r0
    gW0[1] += ir0 * gU;
    gW0[2] += ir0 * gV;
    gir += W0[1] * gU + W0[2] * gV;
    gr -= ir0 * ir0 * gir;
    gW0[0] += gr;
}

// Reverse of point_flux<T, 2, false, false> (tau = 0): cotangents of F and
// dF/dt at one Gauss point -> cotangents of both sides (added to gL, gR).
template <typename T>
GKS_HD void point_flux_vjp(const Side<T>& L, const Side<T>& R, const FluxParams<T>& P, const T* gF, const T* gdF,
                           Side<T>& gL, Side<T>& gR)
{
    T W0[4] = {T(0), T(0), T(0), T(0)}, W0n[4] = {T(0), T(0), T(0), T(0)}, W0t[4] = {T(0), T(0), T(0), T(0)};
    T d4[4], d5[4], d6[4], d7[4], d8[4], pl, pr;
    side_terms<T, 2, false, false>(L, true, P, W0, W0n, W0t, d4, d5, d6, d7, d8, pl);
    side_terms<T, 2, false, false>(R, false, P, W0, W0n, W0t, d4, d5, d6, d7, d8, pr);
    T gW0[4] = {T(0), T(0), T(0), T(0)}, gW0n[4] = {T(0), T(0), T(0), T(0)}, gW0t[4] = {T(0), T(0), T(0), T(0)};
    equilibrium_vjp(W0, W0n, W0t, P.gm1, gF, gdF, gW0, gW0n, gW0t);
    side_vjp(L, true, P, gW0, gW0n, gW0t, gL);
    side_vjp(R, false, P, gW0, gW0n, gW0t, gR);
}

}  // namespace gks
