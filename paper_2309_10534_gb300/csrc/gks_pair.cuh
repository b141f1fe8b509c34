// gks_pair.cuh -- packed float32 pairs for the reconstructions of the
// float32 kernels.
//
// GB300's FP32 units execute two-lane packed instructions (FFMA2, FADD2,
// FMUL2: one issue slot, two IEEE round-to-nearest results).  Where the same
// TENO-D arithmetic runs on two independent streams, the float32 kernels run
// them as one packed stream: in the 2-D sweep the normal reconstruction of
// variables (0, 1) and (2, 3) and the tangential reconstruction of a face
// side's value and normal-slope line averages; in the 1-D kernels the
// normal reconstruction of (rho, rho u).  (The flux's two sides were
// measured packed the same way and kept scalar: no gain.)  `f2` is a drop-in
// arithmetic type for the templated kernel arithmetic: a product stays
// unevaluated (`Prod`) until it is added, so `a * b + c` becomes one fused
// multiply-add, as the compiler's contraction does for scalar code.
// Divisions and comparisons run per lane.
#pragma once

#include "gks_device.cuh"

namespace gks {

struct __align__(8) f2 {
    float2 v;
    f2() = default;
    GKS_HD f2(float s) : v(make_float2(s, s)) {}
    GKS_HD f2(double s) : v(make_float2((float)s, (float)s)) {}
    GKS_HD f2(int s) : v(make_float2((float)s, (float)s)) {}
    GKS_HD f2(float a, float b) : v(make_float2(a, b)) {}
    GKS_HD explicit f2(float2 p) : v(p) {}
    GKS_HD float x() const { return v.x; }
    GKS_HD float y() const { return v.y; }
};

GKS_HD f2 pmul(f2 a, f2 b)
{
#ifdef __CUDA_ARCH__
    return f2(__fmul2_rn(a.v, b.v));
#else
    return f2(a.v.x * b.v.x, a.v.y * b.v.y);
#endif
}
GKS_HD f2 padd(f2 a, f2 b)
{
#ifdef __CUDA_ARCH__
    return f2(__fadd2_rn(a.v, b.v));
#else
    return f2(a.v.x + b.v.x, a.v.y + b.v.y);
#endif
}
GKS_HD f2 pfma(f2 a, f2 b, f2 c)
{
#ifdef __CUDA_ARCH__
    return f2(__ffma2_rn(a.v, b.v, c.v));
#else
    return f2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y));
#endif
}
GKS_HD f2 pneg(f2 a) { return f2(-a.v.x, -a.v.y); }

// an unevaluated product a * b
struct Prod {
    f2 a, b;
    GKS_HD operator f2() const { return pmul(a, b); }
};

GKS_HD Prod operator*(f2 a, f2 b) { return Prod{a, b}; }
GKS_HD Prod operator*(Prod p, f2 b) { return Prod{f2(p), b}; }
GKS_HD Prod operator*(f2 a, Prod p) { return Prod{a, f2(p)}; }
GKS_HD Prod operator*(Prod p, Prod q) { return Prod{f2(p), f2(q)}; }

GKS_HD f2 operator+(f2 a, f2 b) { return padd(a, b); }
GKS_HD f2 operator+(Prod p, f2 c) { return pfma(p.a, p.b, c); }
GKS_HD f2 operator+(f2 c, Prod p) { return pfma(p.a, p.b, c); }
GKS_HD f2 operator+(Prod p, Prod q) { return pfma(p.a, p.b, f2(q)); }

GKS_HD f2 operator-(f2 a) { return pneg(a); }
GKS_HD Prod operator-(Prod p) { return Prod{pneg(p.a), p.b}; }
GKS_HD f2 operator-(f2 a, f2 b) { return padd(a, pneg(b)); }
GKS_HD f2 operator-(Prod p, f2 c) { return pfma(p.a, p.b, pneg(c)); }
GKS_HD f2 operator-(f2 c, Prod p) { return pfma(pneg(p.a), p.b, c); }
GKS_HD f2 operator-(Prod p, Prod q) { return pfma(p.a, p.b, pneg(f2(q))); }

// per-lane division (the build's float division, as in scalar code)
GKS_HD f2 operator/(f2 a, f2 b) { return f2(a.v.x / b.v.x, a.v.y / b.v.y); }
GKS_HD f2 operator/(Prod p, f2 b) { return f2(p) / b; }

GKS_HD f2& operator+=(f2& a, f2 b) { return a = a + b; }
GKS_HD f2& operator+=(f2& a, Prod p) { return a = p + a; }
GKS_HD f2& operator-=(f2& a, f2 b) { return a = a - b; }
GKS_HD f2& operator*=(f2& a, f2 b) { return a = pmul(a, b); }

// TENO-D selection (Sec. 4.2, Eqs. 4.5-4.7 and 4.11-4.12) of two 5-cell
// stencils at once, one per lane, with the selection folded into the
// coefficients: a lane that keeps the large stencil has zero sub-stencil
// weights, a lane that keeps sub-stencils has zero quartic coefficients, so
// one formula evaluates either choice.  Same powers-of-ratios form as
// teno_select (no division by beta, nothing overflows).
struct TenoSel2 {
    f2 q2, b[3], c[3], u1, u2, u3, u4, w[3];
};

GKS_HD float lane_min4(float a, float b, float c, float d) { return fminf(fminf(a, b), fminf(c, d)); }

GKS_HD void teno_select_x2(const f2 q[5], const TenoT<float>& P, TenoSel2& S)
{
    TenoSel<f2> C;
    stencil_coeffs(q, C);
    f2 t[4];
    teno_indicators(C, f2(P.eps), t);
    const f2 m(lane_min4(t[0].x(), t[1].x(), t[2].x(), t[3].x()), lane_min4(t[0].y(), t[1].y(), t[2].y(), t[3].y()));
    f2 p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const f2 r = m * f2(1.0f / t[j].x(), 1.0f / t[j].y());
        if (P.q == 7) {
            const f2 r2 = r * r, r3 = r2 * r;
            p[j] = r3 * r3 * r;
        } else {
            p[j] = f2(ipow(r.x(), P.q), ipow(r.y(), P.q));
        }
    }
    const f2 s012 = p[0] + p[1] + p[2];
    const f2 lim = f2(P.ct1) * (s012 + p[3]);
    const float lx = (p[3].x() >= lim.x()) ? 1.0f : 0.0f, ly = (p[3].y() >= lim.y()) ? 1.0f : 0.0f;
    const f2 thr = f2(P.ct2) * s012;
    f2 d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        d[k] = f2(p[k].x() >= thr.x() ? 1.0f : 0.0f, p[k].y() >= thr.y() ? 1.0f : 0.0f);
    // at least one sub-stencil passes the second cut (its ratio is the
    // largest, >= s012 / 3 > C_T2 s012), so dsum >= 1
    const f2 dsum = d[0] + d[1] + d[2];
    const f2 inv = f2((1.0f - lx) / dsum.x(), (1.0f - ly) / dsum.y());  // 0 on large-stencil lanes
    const f2 lm(lx, ly);
    S.q2 = C.q2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        S.b[k] = C.b[k];
        S.c[k] = C.c[k];
        S.w[k] = d[k] * inv;
    }
    S.u1 = C.u1 * lm;
    S.u2 = C.u2 * lm;
    S.u3 = C.u3 * lm;
    S.u4 = C.u4 * lm;
}

// the selection of lane x (y) as 4 bits (bit 0: large stencil; bits 1-3:
// the kept sub-stencils): a lane that keeps sub-stencils has a positive weight
GKS_HD unsigned sel_code_x(const TenoSel2& S)
{
    const unsigned c = (S.w[0].x() > 0.0f ? 2u : 0u) | (S.w[1].x() > 0.0f ? 4u : 0u) | (S.w[2].x() > 0.0f ? 8u : 0u);
    return c ? c : 1u;
}
GKS_HD unsigned sel_code_y(const TenoSel2& S)
{
    const unsigned c = (S.w[0].y() > 0.0f ? 2u : 0u) | (S.w[1].y() > 0.0f ? 4u : 0u) | (S.w[2].y() > 0.0f ? 8u : 0u);
    return c ? c : 1u;
}

// values and xi-derivatives at the faces xi = +-1/2 of both lanes' selection:
// the quartic in the Legendre-type basis (P2(1/2) = 1/6, P3(1/2) = 1/20,
// P4(1/2) = 1/70; P2' = 1, P3' = 3/5, P4' = 2/7 at 1/2, odd ones change sign
// at -1/2), equal to Eqs. (4.8), (4.9) and their mirror, plus the
// sub-stencil blend of Eqs. (4.13), (4.14)
GKS_HD void teno_faces_x2(const TenoSel2& S, f2& vp, f2& dp, f2& vm, f2& dm)
{
    const f2 even = S.q2 + S.u2 * f2(1.0f / 6.0f) + S.u4 * f2(1.0f / 70.0f);
    const f2 odd = S.u1 * f2(0.5f) + S.u3 * f2(0.05f);
    const f2 deven = S.u1 + S.u3 * f2(0.6f);
    const f2 dodd = S.u2 + S.u4 * f2(2.0f / 7.0f);
    vp = even + odd;
    vm = even - odd;
    dp = deven + dodd;
    dm = deven - dodd;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const f2 bh = f2(0.5f) * S.b[k], c6 = S.c[k] * f2(1.0f / 6.0f);
        vp += S.w[k] * (bh + c6);
        vm += S.w[k] * (c6 - bh);
        dp += S.w[k] * (S.b[k] + S.c[k]);
        dm += S.w[k] * (S.b[k] - S.c[k]);
    }
}

// Normal reconstruction of one 1-D cell's three variables (rho, rho u, E):
// float32 TENO-D runs (rho, rho u) as one packed pair and E alone; otherwise
// variable by variable with the scheme's reconstruction.  Face values and
// xi-slopes at +1/2 (vp, dp) and -1/2 (vm, dm).
template <int REC, typename T>
GKS_HD void recon_cell3(const T q[3][5], const TenoT<T>& P, T* vp, T* dp, T* vm, T* dm)
{
    if constexpr (sizeof(T) == 4 && REC == 0) {
        f2 qq[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) qq[s] = f2(q[0][s], q[1][s]);
        TenoSel2 S2;
        teno_select_x2(qq, P, S2);
        f2 a, b, c, d;
        teno_faces_x2(S2, a, b, c, d);
        vp[0] = a.x(); vp[1] = a.y();
        dp[0] = b.x(); dp[1] = b.y();
        vm[0] = c.x(); vm[1] = c.y();
        dm[0] = d.x(); dm[1] = d.y();
        TenoSel<T> S;
        teno_select(q[2], P, S);
        teno_faces(q[2], S, vp[2], dp[2], vm[2], dm[2]);
    } else {
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            TenoSel<T> S;
            rec_select<REC>(q[v], P, S);
            rec_faces<REC>(q[v], S, vp[v], dp[v], vm[v], dm[v]);
        }
    }
}

// values and xi-derivatives at the two Gauss points xi = -g and xi = +g
// (g = 1/(2 sqrt 3)) of both lanes' selection.  At the Gauss points
// g^2 = 1/12, so P2 = 0, P3 = -xi/15, P4 = -1/180, P3' = 1/10, P4' = -2 xi/21
// for the quartic, and the quadratics reduce to q2 + b xi: every value is
// E + xi O and every derivative Ed + xi Od, with E, O, Ed, Od shared by the
// two points.
GKS_HD void teno_gauss_pm_x2(const TenoSel2& S, float g, f2& vm, f2& dm, f2& vp, f2& dp)
{
    f2 sb = S.w[0] * S.b[0], sc = S.w[0] * S.c[0];
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        sb += S.w[k] * S.b[k];
        sc += S.w[k] * S.c[k];
    }
    const f2 E = S.q2 - S.u4 * f2(1.0f / 180.0f);
    const f2 O = (S.u1 - S.u3 * f2(1.0f / 15.0f)) + sb;
    const f2 Ed = (S.u1 + S.u3 * f2(0.1f)) + sb;
    const f2 Od = (f2(2.0f) * S.u2 - S.u4 * f2(2.0f / 21.0f)) + f2(2.0f) * sc;
    const f2 G(g);
    vm = E - G * O;
    vp = E + G * O;
    dm = Ed - G * Od;
    dp = Ed + G * Od;
}

GKS_HD f2 fabs(f2 a) { return f2(fabsf(a.v.x), fabsf(a.v.y)); }

// the reconstruction parameters broadcast to both lanes (WENO5-AO)
GKS_HD TenoT<f2> pair_teno(const TenoT<float>& P)
{
    TenoT<f2> Q;
    Q.eps = f2(P.eps);
    Q.ct1 = f2(P.ct1);
    Q.ct2 = f2(P.ct2);
    Q.q = P.q;
#pragma unroll
    for (int k = 0; k < 4; ++k) Q.g[k] = f2(P.g[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Q.gr[k] = f2(P.gr[k]);
    Q.ig3 = f2(P.ig3);
    Q.eps_ao = f2(P.eps_ao);
    return Q;
}

// The scheme's reconstruction of two stencils at once: face values and
// xi-slopes (normal direction), or values and xi-derivatives at the two
// Gauss points (tangential).  REC 0: TENO-D with the folded selection above;
// REC 1: WENO5-AO through its templated arithmetic, whose weights have no
// branches.
template <int REC>
GKS_HD void packed_faces(const f2 q[5], const TenoT<float>& P, f2& vp, f2& dp, f2& vm, f2& dm)
{
    if constexpr (REC == 0) {
        TenoSel2 S;
        teno_select_x2(q, P, S);
        teno_faces_x2(S, vp, dp, vm, dm);
    } else {
        TenoSel<f2> S;
        ao_select(q, pair_teno(P), S);
        ao_faces(q, S, vp, dp, vm, dm);
    }
}
template <int REC>
GKS_HD void packed_gauss(const f2 q[5], const TenoT<float>& P, float gA, float gB, f2& va, f2& da, f2& vb, f2& db)
{
    if constexpr (REC == 0) {
        // the Gauss points are symmetric: gA = -gB
        TenoSel2 S;
        teno_select_x2(q, P, S);
        teno_gauss_pm_x2(S, gB, va, da, vb, db);
    } else {
        TenoSel<f2> S;
        ao_select(q, pair_teno(P), S);
        ao_gauss(S, f2(gA), va, da);
        ao_gauss(S, f2(gB), vb, db);
    }
}

}  // namespace gks
