// gks_device.cuh -- device arithmetic of the TENO-D gas-kinetic scheme.
//
// Everything here runs per cell or per interface point in registers:
//   * TENO-D reconstruction of one 5-cell stencil (paper Sec. 4.2), written
//     with the Legendre-type coefficients of the quartic and the (b, c)
//     coefficients of the three quadratics, evaluated at the cell faces
//     (xi = +-1/2) or at the Gauss points xi = +-1/(2 sqrt 3);
//   * Maxwellian moments, the closed-form micro-slope solve, kinetic merge
//     and the time-dependent BGK flux at one point (Sec. 2.1, Eqs. 2.5-2.9),
//     with the two time integrals of Sec. 2.2 folded into F and dF/dt.
// Templated on the arithmetic type T (float or double) and the dimension.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define GKS_HD __host__ __device__ __forceinline__

namespace gks {

// ------------------------------------------------------------------ math
template <typename T> struct M;
template <> struct M<float> {
    static GKS_HD float erfc_(float x) { return erfcf(x); }
    static GKS_HD float exp_(float x) { return expf(x); }
    static GKS_HD float sqrt_(float x) { return sqrtf(x); }
    static GKS_HD float rcp(float x) { return 1.0f / x; }
    static constexpr float tiny = 1.17549435e-38f;  // FLT_MIN: smallest eps kept normal
    static constexpr int nseries = 16;               // terms of the time-coefficient series
    static constexpr float s_series = 2.0f;          // series below, closed form above
    static constexpr float s_noexp = 48.0f;          // above: exp(-s/2) < 4e-11, below float32 resolution
};
template <> struct M<double> {
    static GKS_HD double erfc_(double x) { return erfc(x); }
    static GKS_HD double exp_(double x) { return exp(x); }
    static GKS_HD double sqrt_(double x) { return sqrt(x); }
    static GKS_HD double rcp(double x) { return 1.0 / x; }
    static constexpr double tiny = 0.0;
    static constexpr int nseries = 22;
    static constexpr double s_series = 1.0;
    static constexpr double s_noexp = 90.0;           // above: exp(-s/2) < 3e-20, below float64 resolution
};

// integer power by squaring (q of Eq. 4.5 is a small positive integer)
template <typename T>
GKS_HD T ipow(T x, int q)
{
    T r = T(1);
    while (q) {
        if (q & 1) r *= x;
        x *= x;
        q >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------ reconstruction parameters
// recon 0: TENO-D (Sec. 4.2); 1: WENO5-AO (Sec. 3.2), the reconstruction the
// paper compares against; 2: WENO5-Z and 3: TENO5, the conventional path
// (Sec. 3.1, 4.1; 1-D grids).
struct TenoParams {
    double eps;
    int q;
    double ct1, ct2;  // thresholds of the first / second selection
    int recon = 0;
    double d_hi = 0.85, d_lo = 0.85, eps_ao = 1e-8;  // WENO5-AO
};

// the same parameters in the arithmetic type of the kernel (no conversions
// from double inside the hot loop); eps is clamped to the smallest normal
// float in float32.  WENO5-AO: linear weights g[0..3] of the three
// sub-stencils and the large stencil, gr[k] = g[k]/g[3], and 1/g[3].
template <typename T> struct TenoT {
    T eps, ct1, ct2;
    int q;
    T g[4], gr[3], ig3, eps_ao;
};

template <typename T>
inline TenoT<T> teno_t(const TenoParams& P)
{
    TenoT<T> t;
    t.eps = (T)P.eps;
    if (t.eps < (T)M<T>::tiny) t.eps = (T)M<T>::tiny;
    t.ct1 = (T)P.ct1;
    t.ct2 = (T)P.ct2;
    t.q = P.q;
    const double g3 = P.d_hi, g1 = (1.0 - P.d_hi) * P.d_lo, g0 = 0.5 * (1.0 - P.d_hi) * (1.0 - P.d_lo);
    t.g[0] = (T)g0;
    t.g[1] = (T)g1;
    t.g[2] = (T)g0;
    t.g[3] = (T)g3;
    t.gr[0] = (T)(g0 / g3);
    t.gr[1] = (T)(g1 / g3);
    t.gr[2] = (T)(g0 / g3);
    t.ig3 = (T)(1.0 / g3);
    t.eps_ao = (T)P.eps_ao;
    return t;
}

// Result of the TENO-D selection on one 5-cell stencil: either the large
// stencil, or the equal-weight (d_k = 1/3) average of the kept sub-stencils.
template <typename T> struct TenoSel {
    T q2;               // centre cell average
    T b[3], c[3];       // quadratic k: p = q2 - c/12 + b xi + c xi^2
    T u1, u2, u3, u4;   // quartic in the Legendre-type basis
    T w[3];             // sub-stencil weights (0 when the large stencil is used)
    T w3;               // WENO5-AO: weight of the quartic (TENO-D: unused)
    bool large;
};

// beta_k of Eq. (3.7): quadratics b^2 + 13/3 c^2; the quartic in Balsara's
// Legendre form.  Selection of Eqs. (4.5)-(4.7) and (4.11)-(4.12) on powers
// normalised by the smallest beta + eps (below), without divisions and
// without (beta+eps)^-q, which would overflow in float32.
// the sub-stencil quadratics and the large-stencil quartic (Sec. 3.1),
// formed from the sums and differences of the cells at equal distance from
// the centre (the quartic's odd coefficients only see the differences, its
// even ones only the sums): every coefficient is one to three fused
// multiply-adds
template <typename T>
GKS_HD void stencil_coeffs(const T q[5], TenoSel<T>& S)
{
    const T q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3], q4 = q[4];
    const T s1 = q1 + q3, d1 = q3 - q1, s0 = q0 + q4, d0 = q4 - q0;
    S.q2 = q2;
    S.b[0] = T(1.5) * q2 + (T(0.5) * q0 - T(2) * q1);  // (q0 - 4 q1 + 3 q2) / 2
    S.c[0] = T(0.5) * (q0 + q2) - q1;                   // (q0 - 2 q1 + q2) / 2
    S.b[1] = T(0.5) * d1;                               // (q3 - q1) / 2
    S.c[1] = T(0.5) * s1 - q2;                          // (q1 - 2 q2 + q3) / 2
    S.b[2] = T(2) * q3 - (T(1.5) * q2 + T(0.5) * q4);   // (-3 q2 + 4 q3 - q4) / 2
    S.c[2] = T(0.5) * (q2 + q4) - q3;                   // (q2 - 2 q3 + q4) / 2
    S.u1 = T(82.0 / 120.0) * d1 - T(11.0 / 120.0) * d0;                       // (11 q0 - 82 q1 + 82 q3 - 11 q4) / 120
    S.u2 = T(40.0 / 56.0) * s1 - (T(3.0 / 56.0) * s0 + T(74.0 / 56.0) * q2);  // (-3 q0 + 40 q1 - 74 q2 + 40 q3 - 3 q4) / 56
    S.u3 = T(1.0 / 12.0) * d0 - T(1.0 / 6.0) * d1;                            // (-q0 + 2 q1 - 2 q3 + q4) / 12
    S.u4 = T(1.0 / 24.0) * s0 + (T(0.25) * q2 - T(1.0 / 6.0) * s1);          // (q0 - 4 q1 + 6 q2 - 4 q3 + q4) / 24
}

// smoothness indicators t_k = beta_k + eps of Eq. (3.7) (quadratics
// b^2 + 13/3 c^2; the quartic in Balsara's Legendre form), each a chain of
// fused multiply-adds onto eps
template <typename T>
GKS_HD void teno_indicators(const TenoSel<T>& S, T eps, T* t)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = S.b[k] * S.b[k] + (T(13.0 / 3.0) * S.c[k] * S.c[k] + eps);
    const T a = S.u1 + T(0.1) * S.u3, bq = S.u2 + T(123.0 / 455.0) * S.u4;
    t[3] = a * a + (T(13.0 / 3.0) * bq * bq + (T(781.0 / 20.0) * S.u3 * S.u3
                                              + (T(1421461.0 / 2275.0) * S.u4 * S.u4 + eps)));
}

// WENO5-AO (Sec. 3.2): beta by Eq. (3.7), global indicator
// tau = mean |beta_3 - beta_k|, weights gamma_k (1 + (tau/(beta_k + eps))^2)
// normalised over the four stencils, and the AO(5,3) polynomial
//   P = wbar_3/gamma_3 p_3 + sum_k (wbar_k - wbar_3 gamma_k/gamma_3) p_k,
// stored as the evaluation weights w3 (quartic) and w[k] (quadratics).
template <typename T>
GKS_HD void ao_select(const T q[5], const TenoT<T>& P, TenoSel<T>& S)
{
    stencil_coeffs(q, S);
    T beta[4];
#pragma unroll
    for (int k = 0; k < 3; ++k) beta[k] = S.b[k] * S.b[k] + T(13.0 / 3.0) * S.c[k] * S.c[k];
    {
        const T a = S.u1 + T(0.1) * S.u3, bq = S.u2 + T(123.0 / 455.0) * S.u4;
        beta[3] = a * a + T(13.0 / 3.0) * bq * bq + T(781.0 / 20.0) * S.u3 * S.u3
                + T(1421461.0 / 2275.0) * S.u4 * S.u4;
    }
    const T tau = (fabs(beta[3] - beta[0]) + fabs(beta[3] - beta[1]) + fabs(beta[3] - beta[2])) * T(1.0 / 3.0);
    T om[4], sum = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T r = tau / (beta[k] + P.eps_ao);
        om[k] = P.g[k] * (T(1) + r * r);
        sum += om[k];
    }
    const T is = T(1) / sum;
    const T w3 = om[3] * is;
    S.w3 = w3 * P.ig3;
#pragma unroll
    for (int k = 0; k < 3; ++k) S.w[k] = om[k] * is - w3 * P.gr[k];
    S.large = false;
}

template <typename T>
GKS_HD void teno_select(const T q[5], const TenoT<T>& P, TenoSel<T>& S)
{
    stencil_coeffs(q, S);
    T t[4];
    teno_indicators(S, P.eps, t);
    // chi_k = t_k^-q / sum_j t_j^-q.  With m = min_j t_j and r_j = m / t_j in
    // (0, 1], chi_k = r_k^q / sum_j r_j^q: nothing overflows, and an r^q that
    // underflows belongs to a chi far below any cut-off.  The same powers
    // serve both selections (the second normalises over k = 0..2 only).
    T m = t[0] < t[1] ? t[0] : t[1];
    m = m < t[2] ? m : t[2];
    m = m < t[3] ? m : t[3];
    T p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T r = m * (T(1) / t[j]);
        if (P.q == 7) {
            const T r2 = r * r, r3 = r2 * r;
            p[j] = r3 * r3 * r;
        } else {
            p[j] = ipow(r, P.q);
        }
    }
    const T s012 = p[0] + p[1] + p[2];
    // first selection (Eqs. 4.6, 4.7): keep the large stencil when chi_{3,1} >= C_T1
    S.large = (p[3] >= P.ct1 * (s012 + p[3]));
    if (S.large) {
        S.w[0] = S.w[1] = S.w[2] = T(0);
        return;
    }
    // second selection among the small stencils (Eqs. 4.11, 4.12), d_k = 1/3 cancels
    T d[3], dsum = T(0);
    const T thr = P.ct2 * s012;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = (p[k] >= thr) ? T(1) : T(0);
        dsum += d[k];
    }
    const T inv = T(1) / dsum;
#pragma unroll
    for (int k = 0; k < 3; ++k) S.w[k] = d[k] * inv;
}

// values and xi-derivatives at the faces xi = +1/2 (vp, dp) and -1/2 (vm, dm)
template <typename T>
GKS_HD void teno_faces(const T q[5], const TenoSel<T>& S, T& vp, T& dp, T& vm, T& dm)
{
    if (S.large) {  // Eqs. (4.8), (4.9) and their mirror at x_{i-1/2}
        vp = (T(2) * q[0] - T(13) * q[1] + T(47) * q[2] + T(27) * q[3] - T(3) * q[4]) * T(1.0 / 60.0);
        dp = (q[1] - T(15) * q[2] + T(15) * q[3] - q[4]) * T(1.0 / 12.0);
        vm = (T(-3) * q[0] + T(27) * q[1] + T(47) * q[2] - T(13) * q[3] + T(2) * q[4]) * T(1.0 / 60.0);
        dm = (q[0] - T(15) * q[1] + T(15) * q[2] - q[3]) * T(1.0 / 12.0);
        return;
    }
    // Eqs. (4.13), (4.14): p_k(+-1/2) = q2 +- b/2 + c/6, p_k'(+-1/2) = b +- c
    vp = dp = vm = dm = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T w = S.w[k], bh = T(0.5) * S.b[k], c6 = S.c[k] * T(1.0 / 6.0);
        vp += w * (bh + c6);
        vm += w * (c6 - bh);
        dp += w * (S.b[k] + S.c[k]);
        dm += w * (S.b[k] - S.c[k]);
    }
    vp += S.q2;
    vm += S.q2;
}

// one face of teno_faces: value and xi-derivative at xi = +1/2 (PLUS) or -1/2
template <bool PLUS, typename T>
GKS_HD void teno_face(const T q[5], const TenoSel<T>& S, T& v, T& d)
{
    if (S.large) {
        if (PLUS) {
            v = (T(2) * q[0] - T(13) * q[1] + T(47) * q[2] + T(27) * q[3] - T(3) * q[4]) * T(1.0 / 60.0);
            d = (q[1] - T(15) * q[2] + T(15) * q[3] - q[4]) * T(1.0 / 12.0);
        } else {
            v = (T(-3) * q[0] + T(27) * q[1] + T(47) * q[2] - T(13) * q[3] + T(2) * q[4]) * T(1.0 / 60.0);
            d = (q[0] - T(15) * q[1] + T(15) * q[2] - q[3]) * T(1.0 / 12.0);
        }
        return;
    }
    v = d = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T w = S.w[k], bh = T(0.5) * S.b[k], c6 = S.c[k] * T(1.0 / 6.0);
        if (PLUS) {
            v += w * (bh + c6);
            d += w * (S.b[k] + S.c[k]);
        } else {
            v += w * (c6 - bh);
            d += w * (S.b[k] - S.c[k]);
        }
    }
    v += S.q2;
}

// WENO5-AO values and xi-derivatives at the faces: the quartic's (Eqs. 4.8,
// 4.9 and mirror) and the quadratics' (Eqs. 4.13, 4.14) blended by S.w3, S.w
template <typename T>
GKS_HD void ao_faces(const T q[5], const TenoSel<T>& S, T& vp, T& dp, T& vm, T& dm)
{
    const T lvp = (T(2) * q[0] - T(13) * q[1] + T(47) * q[2] + T(27) * q[3] - T(3) * q[4]) * T(1.0 / 60.0);
    const T ldp = (q[1] - T(15) * q[2] + T(15) * q[3] - q[4]) * T(1.0 / 12.0);
    const T lvm = (T(-3) * q[0] + T(27) * q[1] + T(47) * q[2] - T(13) * q[3] + T(2) * q[4]) * T(1.0 / 60.0);
    const T ldm = (q[0] - T(15) * q[1] + T(15) * q[2] - q[3]) * T(1.0 / 12.0);
    T svp = T(0), sdp = T(0), svm = T(0), sdm = T(0), ws = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T w = S.w[k], bh = T(0.5) * S.b[k], c6 = S.c[k] * T(1.0 / 6.0);
        svp += w * (bh + c6);
        svm += w * (c6 - bh);
        sdp += w * (S.b[k] + S.c[k]);
        sdm += w * (S.b[k] - S.c[k]);
        ws += w;
    }
    vp = S.w3 * lvp + ws * S.q2 + svp;
    vm = S.w3 * lvm + ws * S.q2 + svm;
    dp = S.w3 * ldp + sdp;
    dm = S.w3 * ldm + sdm;
}

// WENO5-AO value and xi-derivative at the Gauss point xi = g (xi^2 = 1/12)
template <typename T>
GKS_HD void ao_gauss(const TenoSel<T>& S, T g, T& v, T& d)
{
    T sv = T(0), sd = T(0), ws = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sv += S.w[k] * S.b[k] * g;
        sd += S.w[k] * (S.b[k] + T(2) * S.c[k] * g);
        ws += S.w[k];
    }
    const T lv = S.q2 + S.u1 * g - S.u3 * g * T(1.0 / 15.0) - S.u4 * T(1.0 / 180.0);
    const T ld = S.u1 + T(2) * S.u2 * g + T(0.1) * S.u3 - T(2.0 / 21.0) * S.u4 * g;
    v = S.w3 * lv + ws * S.q2 + sv;
    d = S.w3 * ld + sd;
}

// value and xi-derivative at the Gauss point xi = g (g = +-1/(2 sqrt 3), xi^2 = 1/12)
template <typename T>
GKS_HD void teno_gauss(const TenoSel<T>& S, T g, T& v, T& d)
{
    if (S.large) {
        // P2(g) = 0, P3(g) = -g/15, P4(g) = -1/180; P3'(g) = 1/10, P4'(g) = -2g/21
        v = S.q2 + S.u1 * g - S.u3 * g * T(1.0 / 15.0) - S.u4 * T(1.0 / 180.0);
        d = S.u1 + T(2) * S.u2 * g + T(0.1) * S.u3 - T(2.0 / 21.0) * S.u4 * g;
        return;
    }
    v = S.q2;
    d = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v += S.w[k] * S.b[k] * g;
        d += S.w[k] * (S.b[k] + T(2) * S.c[k] * g);
    }
}

// teno_gauss at both Gauss points xi = -g (vm, dm) and xi = +g (vp, dp),
// g = 1/(2 sqrt 3): each value is E + xi O and each derivative Ed + xi Od,
// with E, O, Ed, Od formed once for the two points
template <typename T>
GKS_HD void teno_gauss_pm(const TenoSel<T>& S, T g, T& vm, T& dm, T& vp, T& dp)
{
    T E, O, Ed, Od;
    if (S.large) {
        E = S.q2 - S.u4 * T(1.0 / 180.0);
        O = S.u1 - S.u3 * T(1.0 / 15.0);
        Ed = S.u1 + T(0.1) * S.u3;
        Od = T(2) * S.u2 - T(2.0 / 21.0) * S.u4;
    } else {
        T sb = S.w[0] * S.b[0], sc = S.w[0] * S.c[0];
#pragma unroll
        for (int k = 1; k < 3; ++k) {
            sb += S.w[k] * S.b[k];
            sc += S.w[k] * S.c[k];
        }
        E = S.q2;
        O = sb;
        Ed = sb;
        Od = T(2) * sc;
    }
    vm = E - g * O;
    vp = E + g * O;
    dm = Ed - g * Od;
    dp = Ed + g * Od;
}

// The conventional path (Sec. 3.1, 4.1): WENO5-Z (REC 2) or TENO5 (REC 3)
// face values from the three quadratics, slopes from the quadratic through
// the cell average and the two face values (Eq. 3.11).  The selection keeps,
// per sub-stencil, the part of the weight that does not depend on the point:
// WENO-Z 1 + tau/(beta_k + eps) (Eq. 3.5, tau = |beta_0 - beta_2|), TENO5 the
// cut-off delta_k of Eq. (4.3).  TENO5's chi_k = gamma_k / sum gamma with
// gamma_k = (1 + tau/t_k)^q, t_k = beta_k + eps (Eqs. 4.1, 4.2), is formed
// from gamma_k / gamma_max = ((t_m / t_k) (t_k + tau)/(t_m + tau))^q, t_m the
// smallest t (the largest gamma), so nothing overflows in float32.
template <int REC, typename T>
GKS_HD void weno3_select(const T q[5], const TenoT<T>& P, TenoSel<T>& S)
{
    stencil_coeffs(q, S);
    T beta[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) beta[k] = S.b[k] * S.b[k] + T(13.0 / 3.0) * S.c[k] * S.c[k];
    const T tau = fabs(beta[0] - beta[2]);
    if constexpr (REC == 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) S.w[k] = T(1) + tau / (beta[k] + P.eps_ao);
    } else {
        T t[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) t[k] = beta[k] + P.eps;
        T m = t[0] < t[1] ? t[0] : t[1];
        m = m < t[2] ? m : t[2];
        const T imt = T(1) / (m + tau);
        T p[3], sum = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T r = (m / t[k]) * ((t[k] + tau) * imt);
            if (P.q == 6) {
                const T r3 = r * r * r;
                p[k] = r3 * r3;
            } else {
                p[k] = ipow(r, P.q);
            }
            sum += p[k];
        }
        const T thr = P.ct1 * sum;
#pragma unroll
        for (int k = 0; k < 3; ++k) S.w[k] = (p[k] >= thr) ? T(1) : T(0);
    }
    S.w3 = T(0);
    S.large = false;
}

// values at xi = +-1/2 with the linear weights of each face (d = 0.1, 0.6,
// 0.3 at +1/2, mirrored at -1/2), omega_k = d_k w_k / sum d_j w_j, and the
// xi-slopes of Eq. (3.11)
template <typename T>
GKS_HD void weno3_faces(const T q[5], const TenoSel<T>& S, T& vp, T& dp, T& vm, T& dm)
{
    const T dP[3] = {T(0.1), T(0.6), T(0.3)};
    T np = T(0), nm = T(0), sp = T(0), sm = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T bh = T(0.5) * S.b[k], c6 = S.c[k] * T(1.0 / 6.0);
        const T ap = dP[k] * S.w[k], am = dP[2 - k] * S.w[k];
        np += ap * (bh + c6);  // p_k(+1/2) - q2
        nm += am * (c6 - bh);  // p_k(-1/2) - q2
        sp += ap;
        sm += am;
    }
    const T ep = np / sp, em = nm / sm;
    vp = S.q2 + ep;
    vm = S.q2 + em;
    dp = T(2) * (em + T(2) * ep);
    dm = T(-2) * (T(2) * em + ep);
    (void)q;
}

// WENO5-Z / TENO5 value and xi-derivative at the Gauss point xi = g
// (g^2 = 1/12): the quadratics blended with the point's linear weights (from
// their definition, sum d_k p_k(g) = p_3(g): (210 + sqrt 3)/1080, 11/18,
// (210 - sqrt 3)/1080 at g = -1/(2 sqrt 3), mirrored at +), and the same
// blend's derivative (the tangential derivative of Step 3)
template <typename T>
GKS_HD void weno3_gauss(const TenoSel<T>& S, T g, T& v, T& d)
{
    const T r = T(1.7320508075688772 / 1080.0);
    const T sgn = (g < T(0)) ? T(1) : T(-1);
    const T dk[3] = {T(7.0 / 36.0) + sgn * r, T(11.0 / 18.0), T(7.0 / 36.0) - sgn * r};
    T num = T(0), dnum = T(0), den = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T a = dk[k] * S.w[k];
        num += a * (S.b[k] * g);                 // p_k(g) - q2 = b g + c (g^2 - 1/12)
        dnum += a * (S.b[k] + T(2) * S.c[k] * g);
        den += a;
    }
    const T iden = T(1) / den;
    v = S.q2 + num * iden;
    d = dnum * iden;
}

// the large-stencil quartic through five averages, value and xi-derivative
// at the Gauss point xi = g (the conventional path's linear reconstruction
// of the equilibrium line averages, Step 4)
template <typename T>
GKS_HD void quartic_gauss(const T q[5], T g, T& v, T& d)
{
    TenoSel<T> S;
    stencil_coeffs(q, S);
    v = S.q2 + S.u1 * g - S.u3 * g * T(1.0 / 15.0) - S.u4 * T(1.0 / 180.0);
    d = S.u1 + T(2) * S.u2 * g + T(0.1) * S.u3 - T(2.0 / 21.0) * S.u4 * g;
}

// the scheme's reconstruction: REC 0 = TENO-D, 1 = WENO5-AO, 2 = WENO5-Z and
// 3 = TENO5 (the conventional path)
template <int REC, typename T>
GKS_HD void rec_select(const T q[5], const TenoT<T>& P, TenoSel<T>& S)
{
    if constexpr (REC == 0) teno_select(q, P, S);
    else if constexpr (REC == 1) ao_select(q, P, S);
    else weno3_select<REC>(q, P, S);
}
template <int REC, typename T>
GKS_HD void rec_faces(const T q[5], const TenoSel<T>& S, T& vp, T& dp, T& vm, T& dm)
{
    if constexpr (REC == 0) teno_faces(q, S, vp, dp, vm, dm);
    else if constexpr (REC == 1) ao_faces(q, S, vp, dp, vm, dm);
    else weno3_faces(q, S, vp, dp, vm, dm);
}
template <int REC, typename T>
GKS_HD void rec_gauss(const TenoSel<T>& S, T g, T& v, T& d)
{
    if constexpr (REC == 0) teno_gauss(S, g, v, d);
    else if constexpr (REC == 1) ao_gauss(S, g, v, d);
    else weno3_gauss(S, g, v, d);
}

// the same at both Gauss points xi = -g (vm, dm) and xi = +g (vp, dp)
template <int REC, typename T>
GKS_HD void rec_gauss_pm(const TenoSel<T>& S, T g, T& vm, T& dm, T& vp, T& dp)
{
    if constexpr (REC == 0) {
        teno_gauss_pm(S, g, vm, dm, vp, dp);
    } else {
        rec_gauss<REC>(S, -g, vm, dm);
        rec_gauss<REC>(S, g, vp, dp);
    }
}

// ------------------------------------------------------------------ characteristic variables
// Sec. 3.1: for Euler systems the reconstructed quantities may be the
// characteristic variables.  Reconstruction code REC_TENO_CHAR is TENO-D on
// C = L W per face: L = R^-1, R the right eigenvectors of the Jacobian of the
// normal Euler flux in the face's local frame (normal velocity first),
// evaluated at the arithmetic mean of the two cells adjacent to the face;
// the reconstructed values and slopes are mapped back by R.  The tangential
// (Gauss-point) reconstruction of the 2-D sweep stays component-wise TENO-D.
constexpr int REC_TENO_CHAR = 4;
// the per-quantity reconstruction a kernel with code REC runs
__host__ __device__ constexpr int rec_base(int REC) { return REC == REC_TENO_CHAR ? 0 : REC; }
// WENO5-Z and TENO5: the conventional path (equilibrium state and slopes
// from their own linear reconstructions)
__host__ __device__ constexpr bool rec_conventional(int REC) { return REC == 2 || REC == 3; }

// Eigen-system of dF/dW at a state with velocity (U, V), sound speed c and
// total enthalpy H: eigenvalues U - c, U (entropy), U (shear; 2-D), U + c in
// slots 0..3 (1-D: slot 2 unused).  b1 = (gamma - 1)/c^2, k = |U|^2/2.
template <typename T> struct CharBasis {
    T U, V, c, ic, H, k, b1;
    bool ok;  // false: the mean state is not physical; projection = identity
};

// basis at the arithmetic mean of the conserved states wa, wb (4 slots,
// energy in slot 3)
template <typename T, int DIM>
GKS_HD void char_basis(const T* wa, const T* wb, T gm1, CharBasis<T>& B)
{
    const T r = T(0.5) * (wa[0] + wb[0]);
    const T ir = T(1) / r;
    B.U = T(0.5) * (wa[1] + wb[1]) * ir;
    B.V = (DIM == 2) ? T(0.5) * (wa[2] + wb[2]) * ir : T(0);
    const T E = T(0.5) * (wa[3] + wb[3]);
    B.k = T(0.5) * (B.U * B.U + B.V * B.V);
    const T p = gm1 * (E - r * B.k);
    B.ok = r > T(0) && p > T(0) && isfinite(p);
    const T c2 = (gm1 + T(1)) * p * ir;
    B.c = B.ok ? M<T>::sqrt_(c2) : T(1);
    B.ic = T(1) / B.c;
    B.H = (E + p) * ir;
    B.b1 = gm1 / c2;
}

// C = L q: with pt = b1 (q3 - U q1 - V q2 + k q0) and t = (q1 - U q0)/c,
// C = ((pt - t)/2, q0 - pt, q2 - V q0, (pt + t)/2)
template <typename T, int DIM>
GKS_HD void char_project(const CharBasis<T>& B, const T* q, T* C)
{
    if (!B.ok) {
#pragma unroll
        for (int i = 0; i < 4; ++i) C[i] = q[i];
        return;
    }
    const T q2 = (DIM == 2) ? q[2] : T(0);
    const T pt = B.b1 * (q[3] - B.U * q[1] - B.V * q2 + B.k * q[0]);
    const T t = B.ic * (q[1] - B.U * q[0]);
    C[0] = T(0.5) * (pt - t);
    C[1] = q[0] - pt;
    C[2] = (DIM == 2) ? q2 - B.V * q[0] : T(0);
    C[3] = T(0.5) * (pt + t);
}

// q = R C: the columns (1, U - c, V, H - U c), (1, U, V, k), (0, 0, 1, V),
// (1, U + c, V, H + U c)
template <typename T, int DIM>
GKS_HD void char_back(const CharBasis<T>& B, const T* C, T* q)
{
    if (!B.ok) {
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = C[i];
        return;
    }
    const T s = C[0] + C[3], d = C[3] - C[0];
    const T c2 = (DIM == 2) ? C[2] : T(0);
    q[0] = s + C[1];
    q[1] = B.U * q[0] + B.c * d;
    q[2] = (DIM == 2) ? B.V * q[0] + c2 : T(0);
    q[3] = B.H * s + B.U * B.c * d + B.k * C[1] + B.V * c2;
}

// Both sides of one face in characteristic variables: w[0..5] are the six
// cells i-2 .. i+3 around the face between cells i and i+1 (4 slots each;
// 1-D slot 2 = 0).  Left side: TENO-D of cells i-2 .. i+2 at xi = +1/2;
// right side: of cells i-1 .. i+3 at xi = -1/2; values and xi-derivatives
// back in conserved variables.
template <typename T, int DIM>
GKS_HD void char_face(const T (*w)[4], const TenoT<T>& P, T gm1, T* vl, T* dl, T* vr, T* dr)
{
    CharBasis<T> B;
    char_basis<T, DIM>(w[2], w[3], gm1, B);
    T C[6][4];
#pragma unroll
    for (int s = 0; s < 6; ++s) char_project<T, DIM>(B, w[s], C[s]);
    T cvl[4], cdl[4], cvr[4], cdr[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (DIM == 1 && k == 2) {
            cvl[k] = cdl[k] = cvr[k] = cdr[k] = T(0);
            continue;
        }
        T q[5];
        TenoSel<T> S;
#pragma unroll
        for (int s = 0; s < 5; ++s) q[s] = C[s][k];
        teno_select(q, P, S);
        teno_face<true>(q, S, cvl[k], cdl[k]);
#pragma unroll
        for (int s = 0; s < 5; ++s) q[s] = C[s + 1][k];
        teno_select(q, P, S);
        teno_face<false>(q, S, cvr[k], cdr[k]);
    }
    char_back<T, DIM>(B, cvl, vl);
    char_back<T, DIM>(B, cdl, dl);
    char_back<T, DIM>(B, cvr, vr);
    char_back<T, DIM>(B, cdr, dr);
}

// ------------------------------------------------------------------ kinetic layer
// Moments of a unit-mass Maxwellian: <u^n> (n = 0..6), <v^m> (m = 0..5),
// <xi^2>, <xi^4>.  In 1-D there is no v: <v^0> = 1, <v^m> = 0.
template <typename T, int DIM>
GKS_HD void u_recursion(T* u, T U, T inv2l)
{
#pragma unroll
    for (int n = 0; n < 5; ++n) u[n + 2] = U * u[n + 1] + T(n + 1) * inv2l * u[n];
}

template <typename T, int DIM>
GKS_HD void v_moments(T* v, T V, T inv2l)
{
    if constexpr (DIM == 2) {
        v[0] = T(1);
        v[1] = V;
#pragma unroll
        for (int n = 0; n < 4; ++n) v[n + 2] = V * v[n + 1] + T(n + 1) * inv2l * v[n];
    } else {
        v[0] = T(1);
#pragma unroll
        for (int n = 1; n < 6; ++n) v[n] = T(0);
    }
}

// Moment matrix H^(k,m)_ab = <u^k v^m psi_a psi_b>, psi = (1, u, v, (u^2+v^2+xi^2)/2),
// of a unit-mass Maxwellian from its moment tables; 10 unique entries
// (H00 H01 H02 H03 H11 H12 H13 H22 H23 H33).  <u^k v^m (a.psi) psi> = H a.
// 1-D: v == 0, so only m = 0 occurs and the v entries vanish.
template <int k, int m, typename T, int DIM>
GKS_HD void hmat(const T* u, const T* v, T xi2, T xi4, T* H)
{
    if constexpr (DIM == 2) {
        H[0] = u[k] * v[m];
        H[1] = u[k + 1] * v[m];
        H[2] = u[k] * v[m + 1];
        H[4] = u[k + 2] * v[m];
        H[5] = u[k + 1] * v[m + 1];
        H[7] = u[k] * v[m + 2];
        H[3] = T(0.5) * (H[4] + H[7] + H[0] * xi2);
        H[6] = T(0.5) * (u[k + 3] * v[m] + u[k + 1] * v[m + 2] + H[1] * xi2);
        H[8] = T(0.5) * (u[k + 2] * v[m + 1] + u[k] * v[m + 3] + H[2] * xi2);
        H[9] = T(0.25) * (u[k + 4] * v[m] + u[k] * v[m + 4] + H[0] * xi4
                          + T(2) * (u[k + 2] * v[m + 2] + (H[4] + H[7]) * xi2));
    } else {
        static_assert(m == 0, "1-D has no v moments");
        H[0] = u[k];
        H[1] = u[k + 1];
        H[4] = u[k + 2];
        H[3] = T(0.5) * (H[4] + H[0] * xi2);
        H[6] = T(0.5) * (u[k + 3] + H[1] * xi2);
        H[9] = T(0.25) * (u[k + 4] + H[0] * xi4 + T(2) * H[4] * xi2);
        H[2] = H[5] = H[7] = H[8] = T(0);
    }
}

// o = H a for the symmetric moment matrix of hmat
template <typename T, int DIM>
GKS_HD void hmv(const T* H, const T* a, T* o)
{
    if constexpr (DIM == 2) {
        o[0] = H[0] * a[0] + H[1] * a[1] + H[2] * a[2] + H[3] * a[3];
        o[1] = H[1] * a[0] + H[4] * a[1] + H[5] * a[2] + H[6] * a[3];
        o[2] = H[2] * a[0] + H[5] * a[1] + H[7] * a[2] + H[8] * a[3];
        o[3] = H[3] * a[0] + H[6] * a[1] + H[8] * a[2] + H[9] * a[3];
    } else {
        o[0] = H[0] * a[0] + H[1] * a[1] + H[3] * a[3];
        o[1] = H[1] * a[0] + H[4] * a[1] + H[6] * a[3];
        o[2] = T(0);
        o[3] = H[3] * a[0] + H[6] * a[1] + H[9] * a[3];
    }
}

// o += H a for the symmetric moment matrix of hmat, as fused multiply-add
// chains into the accumulator (no separate product and sum)
template <typename T, int DIM>
GKS_HD void hmv_acc(const T* H, const T* a, T* o)
{
    if constexpr (DIM == 2) {
        o[0] = fma(H[3], a[3], fma(H[2], a[2], fma(H[1], a[1], fma(H[0], a[0], o[0]))));
        o[1] = fma(H[6], a[3], fma(H[5], a[2], fma(H[4], a[1], fma(H[1], a[0], o[1]))));
        o[2] = fma(H[8], a[3], fma(H[7], a[2], fma(H[5], a[1], fma(H[2], a[0], o[2]))));
        o[3] = fma(H[9], a[3], fma(H[8], a[2], fma(H[6], a[1], fma(H[3], a[0], o[3]))));
    } else {
        o[0] = fma(H[3], a[3], fma(H[1], a[1], fma(H[0], a[0], o[0])));
        o[1] = fma(H[6], a[3], fma(H[4], a[1], fma(H[1], a[0], o[1])));
        o[3] = fma(H[9], a[3], fma(H[6], a[1], fma(H[3], a[0], o[3])));
    }
}

// Euler flux rho <u psi> of a Maxwellian state (local frame, normal first):
// (m, m U + p, m V, U (E + p))
template <typename T, int DIM>
GKS_HD void euler_flux(const T* W, T U, T p, T* F)
{
    F[0] = W[1];
    F[1] = W[1] * U + p;
    F[2] = (DIM == 2) ? W[1] * W[2] / W[0] : T(0);
    F[3] = U * (W[3] + p);
}

// Jacobian-vector products of the Euler fluxes.  For the micro slope a of a
// state derivative dW (<a psi> rho = dW), chain rule through the Maxwellian
// gives rho <u (a.psi) psi> = (dF/dW) dW and rho <v (a.psi) psi> = (dG/dW) dW,
// with F, G the normal and tangential Euler fluxes of an ideal gas whose
// gamma matches K.  h = (E + p)/rho.
template <typename T, int DIM>
GKS_HD void euler_jvp(const T* dW, T U, T V, T h, T gm1, T* dF, T* dG)
{
    const T q = T(0.5) * (U * U + V * V);
    if constexpr (DIM == 2) {
        const T dp = gm1 * (dW[3] - U * dW[1] - V * dW[2] + q * dW[0]);
        const T cross = V * dW[1] + U * dW[2] - U * V * dW[0];
        if (dF) {
            dF[0] = dW[1];
            dF[1] = T(2) * U * dW[1] - U * U * dW[0] + dp;
            dF[2] = cross;
            dF[3] = U * (dW[3] + dp) + h * (dW[1] - U * dW[0]);
        }
        if (dG) {
            dG[0] = dW[2];
            dG[1] = cross;
            dG[2] = T(2) * V * dW[2] - V * V * dW[0] + dp;
            dG[3] = V * (dW[3] + dp) + h * (dW[2] - V * dW[0]);
        }
    } else {
        const T dp = gm1 * (dW[3] - U * dW[1] + q * dW[0]);
        if (dF) {
            dF[0] = dW[1];
            dF[1] = T(2) * U * dW[1] - U * U * dW[0] + dp;
            dF[2] = T(0);
            dF[3] = U * (dW[3] + dp) + h * (dW[1] - U * dW[0]);
        }
        if (dG) dG[0] = dG[1] = dG[2] = dG[3] = T(0);
    }
}

// -rho <(a_n u + a_t v) psi> = -(dF/dW Wn + dG/dW Wt): the conserved time
// derivative that the compatibility condition <a_n u + a_t v + A> = 0 gives
template <typename T, int DIM>
GKS_HD void compat_time_derivative(const T* Wn, const T* Wt, T U, T V, T h, T gm1, T* Wtime)
{
    T x[4], y[4];
    euler_jvp<T, DIM>(Wn, U, V, h, gm1, x, nullptr);
    if constexpr (DIM == 2) {
        euler_jvp<T, DIM>(Wt, U, V, h, gm1, nullptr, y);
#pragma unroll
        for (int i = 0; i < 4; ++i) Wtime[i] = -(x[i] + y[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) Wtime[i] = -x[i];
    }
}

// Start of the half-space moments: h0 = 1/2 erfc(-sg z) (the mass fraction
// on the side sg of u = 0, z = sqrt(lambda) U) and g = exp(-z^2).
// float64: the math library's erfc and exp.  float32: erfc by Abramowitz &
// Stegun 7.1.26 (Hastings' rational approximation, |error| <= 1.5e-7 on
// x >= 0), which reuses g = exp(-z^2), so one exponential serves both.
template <typename T>
GKS_HD void half_space_start(T z, T sg, T& h0, T& g)
{
    h0 = T(0.5) * M<T>::erfc_(-sg * z);
    g = M<T>::exp_(-z * z);
}
template <>
GKS_HD void half_space_start<float>(float z, float sg, float& h0, float& g)
{
    const float x = fabsf(z);
#ifdef __CUDA_ARCH__
    g = __expf(-x * x);
    const float t = __frcp_rn(1.0f + 0.3275911f * x);
#else
    g = expf(-x * x);
    const float t = 1.0f / (1.0f + 0.3275911f * x);
#endif
    const float poly = t * (0.254829592f + t * (-0.284496736f + t * (1.421413741f + t * (-1.453152027f
                     + t * 1.061405429f))));
    const float h = 0.5f * poly * g;  // 1/2 erfc(|z|)
    h0 = (sg * z >= 0.0f) ? 1.0f - h : h;
}

// Micro slope: <a psi> = b with the full-space moments of a Maxwellian
// (Eq. 2.7), solved in closed form.  ntot = K + DIM degrees of freedom
// besides... (all translational + internal); inv2l = 1/(2 lambda).
template <typename T, int DIM>
GKS_HD void micro_slope(const T* b, T U, T V, T lam, T inv2l, T ntot, T inv_ntot, T* a)
{
    const T E = T(0.5) * (U * U + V * V + ntot * inv2l);
    const T R2 = b[1] - U * b[0];
    const T R3 = (DIM == 2) ? b[2] - V * b[0] : T(0);
    const T R4 = T(2) * (b[3] - E * b[0]);
    const T tl = T(2) * lam;
    a[3] = tl * tl * inv_ntot * (R4 - T(2) * U * R2 - T(2) * V * R3);
    a[2] = (DIM == 2) ? tl * R3 - V * a[3] : T(0);
    a[1] = tl * R2 - U * a[3];
    a[0] = b[0] - U * a[1] - V * a[2] - E * a[3];
}

// ------------------------------------------------------------------ time coefficients
// With s = dt/tau, the time integrals of Eq. (2.5) over [0, delta] are
// q_k = tau^{p_k} phi_k(delta/tau), p = (1,2,2,1,2,2).  The flux and its time
// derivative (Sec. 2.2) need F = (4 F(dt/2) - F(dt))/dt and
// dF = 4 (F(dt) - 2 F(dt/2))/dt^2, i.e. per coefficient
//   cF_k = (4 phi_k(s/2) - phi_k(s)) / s^{p_k}
//   cD_k = (phi_k(s) - 2 phi_k(s/2)) / s^{p_k}
// and then  qF_k = cF_k * dt^{p_k-1},  qD_k = 4 cD_k * dt^{p_k-2}.
// Small s: power series (coefficients generated at compile time from the
// Taylor series of exp, plus the 1/s terms of cF_4, cF_5); large s: closed
// forms in y = exp(-s/2) with the polynomial parts cancelled analytically.
template <typename E> struct SeriesTable {
    E c[12][24];
};

constexpr double cx_fact(int n) { return n <= 1 ? 1.0 : n * cx_fact(n - 1); }
constexpr double cx_pow2neg(int n) { return n == 0 ? 1.0 : 0.5 * cx_pow2neg(n - 1); }
// Taylor coefficient a_n of phi_k(x) = sum a_n x^n
constexpr double cx_phi(int k, int n)
{
    const double e = ((n % 2) ? -1.0 : 1.0) / cx_fact(n);  // (-1)^n / n!
    switch (k) {
    case 0: return n >= 2 ? e : 0.0;                   // x - 1 + e^-x
    case 1: return n >= 3 ? (n - 2) * e : 0.0;         // 2 - x - (x+2) e^-x
    case 2: return n >= 3 ? -e : 0.0;                  // x^2/2 - x + 1 - e^-x
    case 3: return n >= 1 ? -e : 0.0;                  // 1 - e^-x
    case 4: return n >= 1 ? (2 - n) * e : 0.0;         // -2 + (x+2) e^-x
    default: return n >= 1 ? e : 0.0;                  // -(1 - e^-x)
    }
}
constexpr int cx_p(int k) { return (k == 0 || k == 3) ? 1 : 2; }
template <typename E>
constexpr SeriesTable<E> make_series_table()
{
    SeriesTable<E> t{};
    for (int k = 0; k < 6; ++k)
        for (int m = 0; m < 24; ++m) {
            const int n = m + cx_p(k);  // coefficient of s^m after dividing by s^p
            const double w2 = cx_pow2neg(n);
            t.c[k][m] = (E)(cx_phi(k, n) * (4.0 * w2 - 1.0));       // cF_k
            t.c[6 + k][m] = (E)(cx_phi(k, n) * (1.0 - 2.0 * w2));   // cD_k
        }
    return t;
}
__constant__ SeriesTable<double> kSeriesD = make_series_table<double>();
__constant__ SeriesTable<float> kSeriesF = make_series_table<float>();
// host copies (operation counting, host replicas)
constexpr SeriesTable<double> kSeriesHostD = make_series_table<double>();
constexpr SeriesTable<float> kSeriesHostF = make_series_table<float>();

template <typename T> struct SeriesOf {
    static GKS_HD T c(int k, int m)
    {
#ifdef __CUDA_ARCH__
        return (T)kSeriesD.c[k][m];
#else
        return (T)kSeriesHostD.c[k][m];
#endif
    }
};
template <> struct SeriesOf<float> {
    static GKS_HD float c(int k, int m)
    {
#ifdef __CUDA_ARCH__
        return kSeriesF.c[k][m];
#else
        return kSeriesHostF.c[k][m];
#endif
    }
};

template <typename T>
GKS_HD void time_coeffs(T s, T* cF, T* cD)
{
    if (s < M<T>::s_series) {
        const int n = (s < T(0.25)) ? (M<T>::nseries / 2) : M<T>::nseries;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            T acc = T(0);
            for (int m = n - 1; m >= 0; --m) acc = acc * s + SeriesOf<T>::c(k, m);
            if (k < 6) cF[k] = acc; else cD[k - 6] = acc;
        }
        // phi_4 and phi_5 start at -x: their x^1 terms leave -1/s in cF_4, cF_5
        // (they cancel in cD); the table holds the powers s^0 and up.
        const T is = T(1) / s;
        cF[4] -= is;
        cF[5] -= is;
        return;
    }
    const T is = T(1) / s, is2 = is * is;
    if (s > M<T>::s_noexp) {
        // y = exp(-s/2) is below the working precision next to every other
        // term: the closed forms below with y = 0
        cF[0] = (s - T(3)) * is;
        cD[0] = is;
        cF[1] = (T(6) - s) * is2;
        cD[1] = T(-2) * is2;
        cF[2] = (T(3) - s) * is2;
        cD[2] = (T(0.25) * s * s - T(1)) * is2;
        cF[3] = T(3) * is;
        cD[3] = -is;
        cF[4] = T(-6) * is2;
        cD[4] = T(2) * is2;
        cF[5] = T(-3) * is2;
        cD[5] = is2;
        return;
    }
    const T y = M<T>::exp_(T(-0.5) * s), y2 = y * y;
    const T omy = T(1) - y;
    cF[0] = (s - T(3) + T(4) * y - y2) * is;
    cD[0] = omy * omy * is;
    cF[1] = (T(6) - s - (T(2) * s + T(8)) * y + (s + T(2)) * y2) * is2;
    cD[1] = (T(-2) + (s + T(4)) * y - (s + T(2)) * y2) * is2;
    cF[2] = (T(3) - s - T(4) * y + y2) * is2;
    cD[2] = (T(0.25) * s * s - T(1) + T(2) * y - y2) * is2;
    cF[3] = omy * (T(3) - y) * is;
    cD[3] = -omy * omy * is;
    cF[4] = (T(-6) + (T(2) * s + T(8)) * y - (s + T(2)) * y2) * is2;
    cD[4] = (T(2) - (s + T(4)) * y + (s + T(2)) * y2) * is2;
    cF[5] = -omy * (T(3) - y) * is2;
    cD[5] = omy * omy * is2;
}

// ------------------------------------------------------------------ flux at a point
template <typename T> struct FluxParams {
    T gm1;        // gamma - 1
    T K;          // internal degrees of freedom of this dimension
    T ntot;       // K + DIM
    T inv_ntot;   // 1 / ntot
    T dt;
    T c1, c2, mu; // collision time (Sec. 5)
    T prfac;      // 1/Pr - 1
    int tau_mode; // 0 zero, 1 Euler, 2 NS
    int merge = 0; // 0 kinetic weighting (Eqs. 3.25, 3.26), 1 arithmetic average of the sides
};

template <typename T> struct Side {  // one reconstructed side (local frame, 4 slots; 1-D slot 2 = 0)
    T W[4], Wn[4], Wt[4];
};

// Smallest internal-energy fraction (rho e / E) a float32 state may have.
// Below it the float32 pressure has no reliable digits: a reconstructed
// value carries an absolute rounding of ~1e-7 of its stencil's largest
// cell value, which is then a large part of E - rho |U|^2 / 2, and the micro
// slopes scale that error by lambda^2 = (rho / 2p)^2.  (Such points are
// reconstruction artefacts at strong shocks, e.g. a point with p = 7e-6
// beside a cell at p = 21 in the Mach 10 double Mach reflection, where the
// float32 flux came out -522 against 0.2 in float64.)  States of flows
// colder than that need the float64 path.
constexpr double kMinInternalFractionF32 = 1e-4;

// rho > 0 and p > 0 (finite); float32 states also need an internal energy
// of at least kMinInternalFractionF32 of E
template <typename T, int DIM>
GKS_HD bool physical(const T* W, T gm1)
{
    const T r = W[0];
    const T ke = (DIM == 2) ? (W[1] * W[1] + W[2] * W[2]) : W[1] * W[1];
    const T e = W[3] - T(0.5) * ke / r;  // internal energy per volume
    const T p = gm1 * e;
    bool ok = r > T(0) && p > T(0) && isfinite(p);
    if constexpr (sizeof(T) == 4) ok = ok && e >= T(kMinInternalFractionF32) * W[3];
    return ok;
}

// Kinetic merge of two states (values only; Eq. 3.25 with reading R2): the
// conventional path's line-averaged equilibrium state (Step 2).  Both sides
// must be physical.
template <typename T, int DIM>
GKS_HD void merge_values(const T* Wl, const T* Wr, const FluxParams<T>& P, T* W0)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) W0[i] = T(0);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const T* W = side ? Wr : Wl;
        const T sg = side ? T(-1) : T(1);
        const T r = W[0], ir = T(1) / r;
        const T U = W[1] * ir;
        const T V = (DIM == 2) ? W[2] * ir : T(0);
        const T p = P.gm1 * (W[3] - T(0.5) * r * (U * U + V * V));
        const T inv2l = p * ir;
        const T lam = T(0.5) / inv2l;
        const T sl = M<T>::sqrt_(lam);
        T u0, gexp;
        half_space_start<T>(sl * U, sg, u0, gexp);
        const T u1 = U * u0 + sg * T(0.28209479177387814) * gexp / sl;
        const T u2 = U * u1 + inv2l * u0;
        const T v2 = (DIM == 2) ? V * V + inv2l : T(0);
        W0[0] += r * u0;
        W0[1] += r * u1;
        if (DIM == 2) W0[2] += r * u0 * V;
        W0[3] += r * T(0.5) * (u2 + u0 * v2 + u0 * P.K * inv2l);
    }
}

// Accumulated contributions of the non-equilibrium side terms and of the
// equilibrium state, built side by side to keep few values alive.
template <typename T, int DIM, bool NONEQ, bool PRFIX>
GKS_HD void side_terms(const Side<T>& S, bool upper, const FluxParams<T>& P,
                       T* W0, T* W0n, T* W0t, T* S3, T* S4, T* S5, T* N4, T* N5, T& pside)
{
    const T r = S.W[0], ir = T(1) / r;
    const T U = S.W[1] * ir;
    const T V = (DIM == 2) ? S.W[2] * ir : T(0);
    const T p = P.gm1 * (S.W[3] - T(0.5) * r * (U * U + V * V));
    pside = p;
    const T inv2l = p * ir;           // 1/(2 lambda)
    const T lam = T(0.5) / inv2l;     // lambda = rho/(2p)
    const T sl = M<T>::sqrt_(lam);
    const T xi2 = P.K * inv2l, xi4 = P.K * (P.K + T(2)) * inv2l * inv2l;

    // half-space u-moments: upper = u > 0 (left state), else u < 0 (right state)
    T uh[7], v[6];
    const T sg = upper ? T(1) : T(-1);
    half_space_start<T>(sl * U, sg, uh[0], uh[1]);
    uh[1] = U * uh[0] + sg * T(0.28209479177387814) * uh[1] / sl;  // + e^{-lam U^2} / (2 sqrt(pi lam))
    u_recursion<T, DIM>(uh, U, inv2l);
    v_moments<T, DIM>(v, V, inv2l);

    // micro slopes, Eq. (2.7).  The solve is linear in its right-hand side,
    // so rho a = M^-1 W_d: the slopes are formed already multiplied by the
    // side's density, which every moment below carries (rho <(a.psi) psi>)
    T ran[4], rat[4] = {T(0), T(0), T(0), T(0)};
    micro_slope<T, DIM>(S.Wn, U, V, lam, inv2l, P.ntot, P.inv_ntot, ran);
    if constexpr (DIM == 2) micro_slope<T, DIM>(S.Wt, U, V, lam, inv2l, P.ntot, P.inv_ntot, rat);

    // kinetic merge, Eqs. (2.6), (3.25), (3.26): W0 += rho <psi>_half,
    // W0_n += rho <(a_n.psi) psi>_half, W0_t += rho <(a_t.psi) psi>_half
    T H[10];
    hmat<0, 0, T, DIM>(uh, v, xi2, xi4, H);
    W0[0] = fma(r, H[0], W0[0]);
    W0[1] = fma(r, H[1], W0[1]);
    W0[2] = fma(r, H[2], W0[2]);
    W0[3] = fma(r, H[3], W0[3]);
    hmv_acc<T, DIM>(H, ran, W0n);
    if constexpr (DIM == 2) hmv_acc<T, DIM>(H, rat, W0t);

    if constexpr (NONEQ) {
        // time derivative of the side's Maxwellian: <a_n u + a_t v + A> = 0
        const T h = (S.W[3] + p) * ir;
        T Wtime[4], rA[4];
        compat_time_derivative<T, DIM>(S.Wn, S.Wt, U, V, h, P.gm1, Wtime);
        micro_slope<T, DIM>(Wtime, U, V, lam, inv2l, P.ntot, P.inv_ntot, rA);
        if constexpr (PRFIX) hmv_acc<T, DIM>(H, rA, N5);  // density moments of the A and slope terms (heat flux)
        // flux moments of the side terms of Eq. (2.5) over the half space
        hmat<1, 0, T, DIM>(uh, v, xi2, xi4, H);
        S3[0] = fma(r, H[0], S3[0]);
        S3[1] = fma(r, H[1], S3[1]);
        S3[2] = fma(r, H[2], S3[2]);
        S3[3] = fma(r, H[3], S3[3]);
        hmv_acc<T, DIM>(H, rA, S5);
        if constexpr (PRFIX) {
            hmv_acc<T, DIM>(H, ran, N4);
            if constexpr (DIM == 2) {
                hmat<0, 1, T, DIM>(uh, v, xi2, xi4, H);
                hmv_acc<T, DIM>(H, rat, N4);
            }
        }
        hmat<2, 0, T, DIM>(uh, v, xi2, xi4, H);
        hmv_acc<T, DIM>(H, ran, S4);
        if constexpr (DIM == 2) {
            hmat<1, 1, T, DIM>(uh, v, xi2, xi4, H);
            hmv_acc<T, DIM>(H, rat, S4);
        }
    }
}

// F and dF/dt (per unit time; Sec. 2.2) at one interface point in the local
// frame.  Both sides must be physical (the caller applies the fallback).
// W0n_lin, W0_lin, W0t_lin: the conventional path's equilibrium normal
// slope (Eq. 3.12, in 2-D reconstructed to the point), state and tangential
// slope (2-D: linear reconstructions of line-averaged merges, Step 4),
// replacing the kinetic merge at the point; nullptr otherwise
template <typename T, int DIM, bool NONEQ, bool PRFIX>
GKS_HD void point_flux(const Side<T>& L, const Side<T>& R, const FluxParams<T>& P, T* F, T* dF,
                       const T* W0n_lin = nullptr, const T* W0_lin = nullptr, const T* W0t_lin = nullptr)
{
    T W0[4] = {0, 0, 0, 0}, W0n[4] = {0, 0, 0, 0}, W0t[4] = {0, 0, 0, 0};
    T S3[4] = {0, 0, 0, 0}, S4[4] = {0, 0, 0, 0}, S5[4] = {0, 0, 0, 0};
    T N4[4] = {0, 0, 0, 0}, N5[4] = {0, 0, 0, 0};
    T pl, pr;
    side_terms<T, DIM, NONEQ, PRFIX>(L, true, P, W0, W0n, W0t, S3, S4, S5, N4, N5, pl);
    side_terms<T, DIM, NONEQ, PRFIX>(R, false, P, W0, W0n, W0t, S3, S4, S5, N4, N5, pr);
    // the kinetic merge is also the density moment of the side terms (the
    // heat flux needs it even where W0 is replaced below)
    T W0k[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) W0k[i] = W0[i];
    if (P.merge == 1) {
        // arithmetic average of the two sides in place of the kinetic
        // weighting (Sec. 3.2, for smooth flow); the side terms stay
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            W0[i] = T(0.5) * (L.W[i] + R.W[i]);
            W0n[i] = T(0.5) * (L.Wn[i] + R.Wn[i]);
            W0t[i] = T(0.5) * (L.Wt[i] + R.Wt[i]);
        }
    }
    if (W0n_lin) {
#pragma unroll
        for (int i = 0; i < 4; ++i) W0n[i] = W0n_lin[i];
    }
    if (W0_lin) {
#pragma unroll
        for (int i = 0; i < 4; ++i) W0[i] = W0_lin[i];
    }
    if (W0t_lin) {
#pragma unroll
        for (int i = 0; i < 4; ++i) W0t[i] = W0t_lin[i];
    }

    // equilibrium state g0: rho0 <u psi>_0 is the Euler flux of W0 and
    // rho0 <u A0 psi>_0 = (dF/dW) W0_time with W0_time = rho0 <A0 psi>_0 from
    // the compatibility condition, so A0 itself is never formed
    const T r0 = W0[0], ir0 = T(1) / r0;
    const T U0 = W0[1] * ir0;
    const T V0 = (DIM == 2) ? W0[2] * ir0 : T(0);
    const T p0 = P.gm1 * (W0[3] - T(0.5) * r0 * (U0 * U0 + V0 * V0));
    const T h0 = (W0[3] + p0) * ir0;
    T F0[4], W0time[4], F2[4];
    euler_flux<T, DIM>(W0, U0, p0, F0);
    compat_time_derivative<T, DIM>(W0n, W0t, U0, V0, h0, P.gm1, W0time);
    euler_jvp<T, DIM>(W0time, U0, V0, h0, P.gm1, F2, nullptr);

    if (P.tau_mode == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            F[i] = F0[i];
            dF[i] = F2[i];
        }
        return;
    }
    // collision time and time coefficients
    T cF[6], cD[6];
    const T jump = fabs(pl - pr) / (pl + pr);
    T s;
    if (P.tau_mode == 1) s = T(1) / (P.c1 + P.c2 * jump);               // dt / tau
    else s = P.dt / (P.mu / p0 + P.c2 * jump * P.dt);
    time_coeffs<T>(s, cF, cD);

    T F1[4] = {T(0), T(0), T(0), T(0)};  // rho0 <u (a0n u + a0t v) psi>_0
    if constexpr (NONEQ) {
        const T inv2l = p0 * ir0, lam = T(0.5) / inv2l;
        const T xi2 = P.K * inv2l, xi4 = P.K * (P.K + T(2)) * inv2l * inv2l;
        // rho0 a0 = M^-1 W0_d (the solve is linear in its right-hand side)
        T u[7], v[6], ran[4], rat[4], H[10];
        u[0] = T(1);
        u[1] = U0;
        u_recursion<T, DIM>(u, U0, inv2l);
        v_moments<T, DIM>(v, V0, inv2l);
        micro_slope<T, DIM>(W0n, U0, V0, lam, inv2l, P.ntot, P.inv_ntot, ran);
        hmat<2, 0, T, DIM>(u, v, xi2, xi4, H);
        hmv_acc<T, DIM>(H, ran, F1);
        if constexpr (DIM == 2) {
            micro_slope<T, DIM>(W0t, U0, V0, lam, inv2l, P.ntot, P.inv_ntot, rat);
            hmat<1, 1, T, DIM>(u, v, xi2, xi4, H);
            hmv_acc<T, DIM>(H, rat, F1);
        }
    }
    const T dt = P.dt, idt = T(1) / dt;
    // qF_k = cF_k dt^{p_k - 1}, qD_k = 4 cD_k dt^{p_k - 2}
    const T qF0 = cF[0], qF1 = cF[1] * dt, qF2 = cF[2] * dt, qF3 = cF[3], qF4 = cF[4] * dt, qF5 = cF[5] * dt;
    const T qD0 = T(4) * cD[0] * idt, qD1 = T(4) * cD[1], qD2 = T(4) * cD[2], qD3 = T(4) * cD[3] * idt;
    const T qD4 = T(4) * cD[4], qD5 = T(4) * cD[5];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        F[i] = qF0 * F0[i] + qF1 * F1[i] + qF2 * F2[i] + qF3 * S3[i] + qF4 * S4[i] + qF5 * S5[i];
        dF[i] = qD0 * F0[i] + qD1 * F1[i] + qD2 * F2[i] + qD3 * S3[i] + qD4 * S4[i] + qD5 * S5[i];
    }
    if constexpr (PRFIX) {
        // Prandtl correction: F_E += (1/Pr - 1) q, q the heat flux relative to
        // (U0, V0) expanded in raw moments of the same time-dependent f.
        // Density moments: rho0 <psi>_0 = W0, rho0 <(a_n u + a_t v) psi>_0 =
        // -W0_time, rho0 <A0 psi>_0 = W0_time; side terms W0k (the kinetic
        // merge), N4, N5.
        const T ke = T(0.5) * (U0 * U0 + V0 * V0);
        const T cf = ke + U0 * U0;
        T MF[4], MD[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            MF[i] = qF0 * W0[i] + (qF2 - qF1) * W0time[i] + qF3 * W0k[i] + qF4 * N4[i] + qF5 * N5[i];
            MD[i] = qD0 * W0[i] + (qD2 - qD1) * W0time[i] + qD3 * W0k[i] + qD4 * N4[i] + qD5 * N5[i];
        }
        const T qh = F[3] - U0 * F[1] - V0 * F[2] + cf * F[0] + U0 * V0 * MF[2] - U0 * MF[3] - U0 * ke * MF[0];
        const T qd = dF[3] - U0 * dF[1] - V0 * dF[2] + cf * dF[0] + U0 * V0 * MD[2] - U0 * MD[3]
                   - U0 * ke * MD[0];
        F[3] += P.prfac * qh;
        dF[3] += P.prfac * qd;
    }
}

}  // namespace gks
