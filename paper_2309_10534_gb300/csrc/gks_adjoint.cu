// gks_adjoint.cu -- hand-written discrete adjoint of the 2-D S2O4 step
// (collision-free flux, tau = 0) with checkpointing (include/gks.h,
// gks_adjoint_* and gks_vjp_step).
//
// One step of the scheme (Sec. 2.2, dimension by dimension, fixed dt):
//   W*      = W^n - dt/h  d(F/2 + dt/8 dF)(W^n)     (both directions)
//   A       = W^n - dt/h  d(F + dt/6 dF)(W^n)
//   W^{n+1} = A   - dt/h  d(dt/3 dF)(W*)
// where d is the face difference and (F, dF) the Gauss-averaged face flux
// and its time derivative.  Given lam = dJ/dW^{n+1}, the adjoint step is
//   lam*  = [d dF/dW*]^T (dt^2/(3h) Delta lam)
//   lam^n = lam + lam* + [dF/dW^n]^T (dt/h Delta(lam + lam*/2))
//                      + [d dF/dW^n]^T (dt^2/h Delta(lam/6 + lam*/8))
// with Delta lam the difference of lam across a face (zero outside the
// interior).  The transposed flux Jacobian of one direction is applied by
// four kernels on the stage input:
//   k_adj_lines   normal TENO-D per cell -> face-line values and slopes
//                 (the forward sweep's phase 1)
//   k_adj_gauss   per face segment and Gauss point: tangential TENO-D to the
//                 Gauss point (forward), the reverse of the point flux, then
//                 the transposed tangential reconstruction; writes, per face
//                 segment, its contributions to the five line rows of its
//                 tangential stencil
//   k_adj_normal  per cell: gathers the line cotangents of its two faces and
//                 applies the transposed normal reconstruction; writes its
//                 contributions to the five cells of its stencil
//   k_adj_gather  per cell: sums the contributions it received
// and the ghost layers are folded back onto the interior cells they copy
// (the transpose of the ghost fill).  TENO-D selections are recomputed from
// the same stage inputs as in the forward pass, i.e. frozen at the forward
// pass's choice.  Every sum is a gather in a fixed order, so the result does
// not depend on scheduling (only the positivity fallback, which smooth flows
// do not take, adds with atomics).
//
// Checkpointing: gks_adjoint_forward keeps W every k steps; the backward pass
// recomputes each k-step segment from its checkpoint, stage by stage, keeping
// W and W* of every step, and runs the segment's adjoint steps in reverse.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/gks.h"
#include "gks_adjoint.cuh"
#include "gks_ctx.h"

using namespace gks;

namespace {

constexpr int NQ = 16;  // line quantities per face segment: [vL, sL, vR, sR] x 4 variables

// One direction of one stage.  Orientation: dirn 0 = faces normal to x
// (normal index = x, unit stride), dirn 1 = faces normal to y.  Scratch
// arrays are laid out with the unit-stride grid direction fastest.
struct AdjDir {
    const double* src;    // stage input, float64 path (ghosts filled)
    const float* srcf;    // stage input, float32 path (float32 shadow, ghosts filled)
    const double* lam1;   // cotangent fields (ghosted; interior used)
    const double* lam2;   // may be null
    double cF1, cD1, cF2, cD2;
    // float32 copies of the scalars, converted on the host (a float64 ->
    // float32 conversion in every thread would run on the slow float64 pipe)
    float fcF1, fcD1, fcF2, fcD2, fihn, fiht;
    void* lines;          // [NQ][faces nn+1][rows nt+4]
    void* contrib;        // [5][NQ][faces nn+1][rows nt]
    void* dcell;          // [5][4][cells nn+2][rows nt+4]
    double* gW;           // ghosted gradient accumulator
    int dirn, nn, nt;
    long long sn, st;     // element strides along normal / tangential
    double ihn, iht;
};

__device__ __forceinline__ int gvar_(int v, bool swap) { return (swap && (v == 1 || v == 2)) ? 3 - v : v; }

// scratch indices: faces f in [0, nn], line rows r in [-2, nt+2), Gauss rows
// in [0, nt), cells i in [-1, nn]
__device__ __forceinline__ long long lidx(const AdjDir& a, int f, int r)
{
    return a.dirn == 0 ? (long long)(r + 2) * (a.nn + 1) + f : (long long)f * (a.nt + 4) + (r + 2);
}
__device__ __forceinline__ long long cidx(const AdjDir& a, int f, int r)
{
    return a.dirn == 0 ? (long long)r * (a.nn + 1) + f : (long long)f * a.nt + r;
}
__device__ __forceinline__ long long didx(const AdjDir& a, int i, int r)
{
    return a.dirn == 0 ? (long long)(r + 2) * (a.nn + 2) + (i + 1) : (long long)(i + 1) * (a.nt + 4) + (r + 2);
}

// a direction scalar in the arithmetic type
template <typename T>
__device__ __forceinline__ T scal(double d, float f)
{
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}

template <typename T>
__device__ __forceinline__ T load_src(const AdjDir& a, long long gi)
{
    if constexpr (sizeof(T) == 4) return a.srcf[gi];
    else return a.src[gi];
}

// map the launch to (normal index, tangential index): the unit-stride grid
// direction runs along threadIdx.x
__device__ __forceinline__ void map2(const AdjDir& a, int& n, int& t, int n0, int t0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (a.dirn == 0) { n = n0 + x; t = t0 + y; }
    else { n = n0 + y; t = t0 + x; }
}

// frozen selection as 4 bits: large, and the kept small stencils
template <typename T>
__device__ __forceinline__ unsigned sel_code(const TenoSel<T>& S)
{
    if (S.large) return 1u;
    return (S.w[0] > T(0) ? 2u : 0u) | (S.w[1] > T(0) ? 4u : 0u) | (S.w[2] > T(0) ? 8u : 0u);
}

template <typename T>
__device__ __forceinline__ void sel_decode(unsigned c, TenoSel<T>& S)
{
    S.large = (c & 1u) != 0;
    const T d0 = (c & 2u) ? T(1) : T(0), d1 = (c & 4u) ? T(1) : T(0), d2 = (c & 8u) ? T(1) : T(0);
    const T dsum = d0 + d1 + d2;
    const T inv = S.large ? T(0) : T(1) / dsum;  // as teno_select: d_k / sum d
    S.w[0] = d0 * inv;
    S.w[1] = d1 * inv;
    S.w[2] = d2 * inv;
}

// The forward's TENO-D of two stencils (qa, qb) in the forward's arithmetic:
// the float32 sweep reconstructs variable pairs (0, 1), (2, 3) and, per face
// side, the value and normal-slope streams as packed pairs, so the same
// pairs here reproduce its values and selections bit for bit.  Returns the
// two selection codes (qa in bits 0-3, qb in bits 4-7).
template <typename T>
__device__ __forceinline__ unsigned fwd_faces2(const T qa[5], const T qb[5], const TenoT<T>& P, T* vp, T* dp, T* vm,
                                               T* dm)
{
    if constexpr (sizeof(T) == 4) {
        f2 qq[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) qq[s] = f2(qa[s], qb[s]);
        TenoSel2 S2;
        teno_select_x2(qq, P, S2);
        f2 a, b, c, d;
        teno_faces_x2(S2, a, b, c, d);
        vp[0] = a.x(); dp[0] = b.x(); vm[0] = c.x(); dm[0] = d.x();
        vp[1] = a.y(); dp[1] = b.y(); vm[1] = c.y(); dm[1] = d.y();
        return sel_code_x(S2) | (sel_code_y(S2) << 4);
    } else {
        unsigned code = 0;
        const T* q[2] = {qa, qb};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            TenoSel<T> S;
            teno_select(q[l], P, S);
            teno_faces(q[l], S, vp[l], dp[l], vm[l], dm[l]);
            code |= sel_code(S) << (4 * l);
        }
        return code;
    }
}
template <typename T>
__device__ __forceinline__ unsigned fwd_gauss2(const T qa[5], const T qb[5], const TenoT<T>& P, T gA, T gB, T* va,
                                               T* da, T* vb, T* db)
{
    if constexpr (sizeof(T) == 4) {
        f2 qq[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) qq[s] = f2(qa[s], qb[s]);
        TenoSel2 S2;
        teno_select_x2(qq, P, S2);
        f2 a, b, c, d;
        teno_gauss_pm_x2(S2, gB, a, b, c, d);  // gA = -gB
        va[0] = a.x(); da[0] = b.x(); vb[0] = c.x(); db[0] = d.x();
        va[1] = a.y(); da[1] = b.y(); vb[1] = c.y(); db[1] = d.y();
        return sel_code_x(S2) | (sel_code_y(S2) << 4);
    } else {
        unsigned code = 0;
        const T* q[2] = {qa, qb};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            TenoSel<T> S;
            teno_select(q[l], P, S);
            teno_gauss_pm(S, gB, va[l], da[l], vb[l], db[l]);  // gA = -gB, as the forward
            code |= sel_code(S) << (4 * l);
        }
        return code;
    }
}

// ---- phase 1: normal TENO-D of the stage input (as the forward sweep)
template <typename T>
__global__ void __launch_bounds__(256) k_adj_lines(GridDev g, AdjDir a, TenoT<T> tn)
{
    int i, r;
    map2(a, i, r, -1, -2);
    if (i > a.nn || r >= a.nt + 2) return;
    const bool swap = a.dirn != 0;
    const long long org = (long long)NG * g.pitch + NG;
    const long long LP = (long long)(a.nn + 1) * (a.nt + 4);
    T* L = static_cast<T*>(a.lines);
    const T ih = scal<T>(a.ihn, a.fihn);
    {
        const int vv = 2 * (int)blockIdx.z;  // variable pairs (0, 1), (2, 3), as the forward
        T q[2][5];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const long long base = (long long)gvar_(vv + l, swap) * g.plane + org + r * a.st;
#pragma unroll
            for (int s = 0; s < 5; ++s) q[l][s] = load_src<T>(a, base + (i - 2 + s) * a.sn);
        }
        T vp[2], dp[2], vm[2], dm[2];
        fwd_faces2(q[0], q[1], tn, vp, dp, vm, dm);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int v = vv + l;
            if (i + 1 <= a.nn) {
                L[(0 * 4 + v) * LP + lidx(a, i + 1, r)] = vp[l];
                L[(1 * 4 + v) * LP + lidx(a, i + 1, r)] = dp[l] * ih;
            }
            if (i >= 0) {
                L[(2 * 4 + v) * LP + lidx(a, i, r)] = vm[l];
                L[(3 * 4 + v) * LP + lidx(a, i, r)] = dm[l] * ih;
            }
        }
    }
}

// ---- Gauss points: forward tangential TENO-D, reverse point flux, transposed
// tangential TENO-D.  Two adjacent lanes hold the two Gauss points of one face
// segment; lane 0 finishes the left side's quantities, lane 1 the right's.
template <typename T>
__global__ void __launch_bounds__(128, (sizeof(T) == 4) ? 4 : 1) k_adj_gauss(GridDev g, AdjDir a, FluxParams<T> fp, TenoT<T> tt)
{
    const int gp = threadIdx.x & 1;
    const int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 1, y = blockIdx.y * blockDim.y + threadIdx.y;
    int f, r;
    if (a.dirn == 0) { f = x; r = y; }
    else { f = y; r = x; }
    const bool valid = f <= a.nn && r < a.nt;
    const int fc = valid ? f : 0, rc = valid ? r : 0;  // in-range indices for the idle lanes' loads
    const bool swap = a.dirn != 0;
    const long long org = (long long)NG * g.pitch + NG;
    const long long LP = (long long)(a.nn + 1) * (a.nt + 4);
    const long long CP = (long long)(a.nn + 1) * a.nt;
    const T* Lq = static_cast<const T*>(a.lines);
    const T gpos = gp ? T(0.28867513459481288) : T(-0.28867513459481288);
    const T iht = scal<T>(a.iht, a.fiht);

    // forward, as the forward sweep: lane gp reconstructs side gp (0: left,
    // 1: right) at both Gauss points, keeps its own point and hands the other
    // point's values to its partner
    Side<T> L, R;
    unsigned codes = 0;  // selections of the own side: 4 bits per quantity kk * 4 + v
    const T gA = T(-0.28867513459481288), gB = T(0.28867513459481288);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        // the side's value and normal-slope streams as one pair, as the forward
        T q[2][5];
        T va[2], da[2], vb[2], db[2];
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int s = 0; s < 5; ++s) q[l][s] = Lq[((2 * gp + l) * 4 + v) * LP + lidx(a, fc, rc - 2 + s)];
        const unsigned c2 = fwd_gauss2(q[0], q[1], tt, gA, gB, va, da, vb, db);
        codes |= (c2 & 15u) << (4 * v);
        codes |= (c2 >> 4) << (4 * (4 + v));
        T own = gp ? vb[0] : va[0], got = __shfl_xor_sync(0xffffffffu, gp ? va[0] : vb[0], 1);
        L.W[v] = gp ? got : own;
        R.W[v] = gp ? own : got;
        own = (gp ? db[0] : da[0]) * iht;
        got = __shfl_xor_sync(0xffffffffu, (gp ? da[0] : db[0]) * iht, 1);
        L.Wt[v] = gp ? got : own;
        R.Wt[v] = gp ? own : got;
        own = gp ? vb[1] : va[1];
        got = __shfl_xor_sync(0xffffffffu, gp ? va[1] : vb[1], 1);
        L.Wn[v] = gp ? got : own;
        R.Wn[v] = gp ? own : got;
    }
    // positivity fallback, as the forward: the adjacent cell average, zero slopes
    const bool fbL = valid && !physical<T, 2>(L.W, fp.gm1);
    const bool fbR = valid && !physical<T, 2>(R.W, fp.gm1);
    if (fbL || fbR) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const long long b = (long long)gvar_(v, swap) * g.plane + org + rc * a.st;
            if (fbL) { L.W[v] = load_src<T>(a, b + (fc - 1) * a.sn); L.Wn[v] = L.Wt[v] = T(0); }
            if (fbR) { R.W[v] = load_src<T>(a, b + fc * a.sn); R.Wn[v] = R.Wt[v] = T(0); }
        }
    }
    // face cotangents (each Gauss point carries weight 1/2).  The
    // differences are taken in float64, the rest in the working precision;
    // the two lanes of a face split the variables (lane gp: 2 gp, 2 gp + 1)
    // and exchange them, so each float64 difference (the float64 pipe is the
    // slow one) is formed once per face
    T gF[4], gdF[4];
    {
        const T cF1 = scal<T>(a.cF1, a.fcF1), cF2 = scal<T>(a.cF2, a.fcF2);
        const T cD1 = scal<T>(a.cD1, a.fcD1), cD2 = scal<T>(a.cD2, a.fcD2);
        T mF[2], mD[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int v = 2 * gp + h;
            const long long b = (long long)gvar_(v, swap) * g.plane + org + rc * a.st;
            // lam of the cells on either side (zero outside the interior);
            // one float64 subtraction per difference
            const double p1 = fc < a.nn ? a.lam1[b + fc * a.sn] : 0.0;
            const double m1 = fc >= 1 ? a.lam1[b + (fc - 1) * a.sn] : 0.0;
            T e1 = (T)(p1 - m1), e2 = T(0);
            if (a.lam2) {
                const double p2 = fc < a.nn ? a.lam2[b + fc * a.sn] : 0.0;
                const double m2 = fc >= 1 ? a.lam2[b + (fc - 1) * a.sn] : 0.0;
                e2 = (T)(p2 - m2);
            }
            mF[h] = T(0.5) * (cF1 * e1 + cF2 * e2);
            mD[h] = T(0.5) * (cD1 * e1 + cD2 * e2);
        }
        const T oF0 = __shfl_xor_sync(0xffffffffu, mF[0], 1), oF1 = __shfl_xor_sync(0xffffffffu, mF[1], 1);
        const T oD0 = __shfl_xor_sync(0xffffffffu, mD[0], 1), oD1 = __shfl_xor_sync(0xffffffffu, mD[1], 1);
        gF[0] = gp ? oF0 : mF[0];
        gF[1] = gp ? oF1 : mF[1];
        gF[2] = gp ? mF[0] : oF0;
        gF[3] = gp ? mF[1] : oF1;
        gdF[0] = gp ? oD0 : mD[0];
        gdF[1] = gp ? oD1 : mD[1];
        gdF[2] = gp ? mD[0] : oD0;
        gdF[3] = gp ? mD[1] : oD1;
    }
    Side<T> gL, gR;
#pragma unroll
    for (int v = 0; v < 4; ++v) gL.W[v] = gL.Wn[v] = gL.Wt[v] = gR.W[v] = gR.Wn[v] = gR.Wt[v] = T(0);
    if (valid) point_flux_vjp(L, R, fp, gF, gdF, gL, gR);
    if (fbL || fbR) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const long long b = (long long)gvar_(v, swap) * g.plane + org + rc * a.st;
            if (fbL) {
                atomicAdd(&a.gW[b + (fc - 1) * a.sn], (double)gL.W[v]);
                gL.W[v] = gL.Wn[v] = gL.Wt[v] = T(0);
            }
            if (fbR) {
                atomicAdd(&a.gW[b + fc * a.sn], (double)gR.W[v]);
                gR.W[v] = gR.Wn[v] = gR.Wt[v] = T(0);
            }
        }
    }
    // exchange: lane 0 keeps the left side (receives its + point), lane 1 the right
    Side<T>& mine = gp ? gR : gL;
    const Side<T>& other = gp ? gL : gR;
    T oW[4], oWn[4], oWt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        oW[v] = __shfl_xor_sync(0xffffffffu, other.W[v], 1);
        oWn[v] = __shfl_xor_sync(0xffffffffu, other.Wn[v], 1);
        oWt[v] = __shfl_xor_sync(0xffffffffu, other.Wt[v], 1);
    }
    if (!valid) return;
    const T gm = gA, gpl = gB;
    T* C = static_cast<T*>(a.contrib);
#pragma unroll 1
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * gp + kk;  // lane 0: k = 0, 1 (left), lane 1: k = 2, 3 (right)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int qi = k * 4 + v;
            TenoSel<T> S;
            sel_decode((codes >> (4 * (kk * 4 + v))) & 15u, S);
            // cotangents at the - point and the + point
            T gvm, gdm, gvp, gdp;
            if (kk == 0) {
                const T a0 = mine.W[v], d0 = mine.Wt[v] * iht, a1 = oW[v], d1 = oWt[v] * iht;
                gvm = gp ? a1 : a0; gdm = gp ? d1 : d0;
                gvp = gp ? a0 : a1; gdp = gp ? d0 : d1;
            } else {
                gvm = gp ? oWn[v] : mine.Wn[v];
                gvp = gp ? mine.Wn[v] : oWn[v];
                gdm = gdp = T(0);
            }
            T gq[5] = {T(0), T(0), T(0), T(0), T(0)};
            teno_gauss_T(S, gm, gvm, gdm, gq);
            teno_gauss_T(S, gpl, gvp, gdp, gq);
#pragma unroll
            for (int s = 0; s < 5; ++s) C[(long long)(s * NQ + qi) * CP + cidx(a, f, r)] = gq[s];
        }
    }
}

// ---- per cell: line cotangents of its faces -> transposed normal TENO-D
template <typename T>
__global__ void __launch_bounds__(256) k_adj_normal(GridDev g, AdjDir a, TenoT<T> tn)
{
    int i, r;
    map2(a, i, r, -1, -2);
    if (i > a.nn || r >= a.nt + 2) return;
    const bool swap = a.dirn != 0;
    const long long org = (long long)NG * g.pitch + NG;
    const long long CP = (long long)(a.nn + 1) * a.nt;
    const long long DP = (long long)(a.nn + 2) * (a.nt + 4);
    const T* C = static_cast<const T*>(a.contrib);
    T* D = static_cast<T*>(a.dcell);
    const T ih = scal<T>(a.ihn, a.fihn);
    // line row r receives from Gauss row r - s + 2 at stencil position s
    auto gline = [&](int q, int f) {
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int rg = r - s + 2;
            if (rg >= 0 && rg < a.nt) acc += C[(long long)(s * NQ + q) * CP + cidx(a, f, rg)];
        }
        return acc;
    };
    {
        const int vv = 2 * (int)blockIdx.z;  // variable pairs, as the forward's selection
        T q[2][5];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const long long base = (long long)gvar_(vv + l, swap) * g.plane + org + r * a.st;
#pragma unroll
            for (int s = 0; s < 5; ++s) q[l][s] = load_src<T>(a, base + (i - 2 + s) * a.sn);
        }
        T fvp[2], fdp[2], fvm[2], fdm[2];
        const unsigned c2 = fwd_faces2(q[0], q[1], tn, fvp, fdp, fvm, fdm);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int v = vv + l;
            T gvp = T(0), gdp = T(0), gvm = T(0), gdm = T(0);
            if (i + 1 <= a.nn) {
                gvp = gline(0 * 4 + v, i + 1);
                gdp = gline(1 * 4 + v, i + 1) * ih;
            }
            if (i >= 0) {
                gvm = gline(2 * 4 + v, i);
                gdm = gline(3 * 4 + v, i) * ih;
            }
            TenoSel<T> S;
            sel_decode((c2 >> (4 * l)) & 15u, S);  // the forward's selection
            T gq[5] = {T(0), T(0), T(0), T(0), T(0)};
            teno_faces_T(S, gvp, gdp, gvm, gdm, gq);
#pragma unroll
            for (int s = 0; s < 5; ++s) D[(long long)(s * 4 + v) * DP + didx(a, i, r)] = gq[s];
        }
    }
}

// ---- per cell: sum of the contributions of the cells whose stencil holds it
template <typename T>
__global__ void __launch_bounds__(256) k_adj_gather(GridDev g, AdjDir a)
{
    int j, r;
    map2(a, j, r, -3, -2);
    if (j > a.nn + 2 || r >= a.nt + 2) return;
    const bool swap = a.dirn != 0;
    const long long org = (long long)NG * g.pitch + NG;
    const long long DP = (long long)(a.nn + 2) * (a.nt + 4);
    const T* D = static_cast<const T*>(a.dcell);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int i = j + 2 - s;  // cell i's stencil position s is cell i - 2 + s = j
            if (i >= -1 && i <= a.nn) acc += D[(long long)(s * 4 + v) * DP + didx(a, i, r)];
        }
        a.gW[(long long)gvar_(v, swap) * g.plane + org + j * a.sn + r * a.st] += (double)acc;
    }
}

// ---- transpose of the ghost fill: y ghost rows first (over the full ghosted
// width), then the x ghost columns of the interior rows.  One thread per
// (column or row, variable) walks its six ghost cells in a fixed order.
__global__ void k_fold_y(GridDev g, double* gW)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gx = g.nx + 2 * NG;
    if (idx >= 4 * gx) return;
    const int v = idx / gx, i = idx % gx;
    double* P = gW + (long long)v * g.plane + i;
    for (int k = 0; k < 2 * NG; ++k) {
        const int j = k < NG ? k : g.ny + k;
        bool fn, fa;
        const int sj = ghost_src(g.bc[2 + (j >= NG + g.ny)], g.ny, j, fn, fa);
        const bool neg = (v == 2 && (fn || fa)) || (v == 1 && fa);
        const double x = P[(long long)j * g.pitch];
        P[(long long)sj * g.pitch] += neg ? -x : x;
        P[(long long)j * g.pitch] = 0.0;
    }
}

__global__ void k_fold_x(GridDev g, double* gW)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * g.ny) return;
    const int v = idx / g.ny, j = NG + idx % g.ny;
    double* P = gW + (long long)v * g.plane + (long long)j * g.pitch;
    for (int k = 0; k < 2 * NG; ++k) {
        const int i = k < NG ? k : g.nx + k;
        bool fn, fa;
        const int si = ghost_src(g.bc[(i >= NG + g.nx)], g.nx, i, fn, fa);
        const bool neg = (v == 1 && (fn || fa)) || (v == 2 && fa);
        const double x = P[i];
        P[si] += neg ? -x : x;
        P[i] = 0.0;
    }
}

// out = a + b + c (whole ghosted arrays)
__global__ void k_sum3(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                       double* __restrict__ out, long long n)
{
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += 256ll * gridDim.x) out[i] = a[i] + b[i] + c[i];
}

__global__ void k_shadow(const double* __restrict__ W, float* __restrict__ Wf, long long n)
{
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += 256ll * gridDim.x) Wf[i] = (float)W[i];
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

struct gks_adjoint {
    gks_ctx* c = nullptr;
    int k = 1;
    int nsteps = 0;
    double dt = 0.0;
    bool have_forward = false;
    std::vector<double*> ckpt;   // W at steps 0, k, 2k, ... (ghosted)
    std::vector<double*> seg;    // W of the segment being reversed
    std::vector<void*> segs;     // its W* (float32 on the float32 path), from the recomputation
    double* WN = nullptr;        // final state of the forward pass
    double *lam = nullptr, *lams = nullptr, *gacc = nullptr, *nxt = nullptr;
    void *lines = nullptr, *contrib = nullptr, *dcell = nullptr;
    long long launches = 0;
    // one full segment's recomputation and reverse sweep, captured once and
    // replayed for every full segment (fixed buffers; dt and the context's
    // parameters are baked in)
    cudaGraphExec_t seg_exec = nullptr;
    double seg_dt = 0.0;
    long long seg_version = -1, seg_kernels = 0, seg_ctx_kernels = 0;
    bool seg_eager = false;  // the segment does not return its buffers to place: no graph
};

namespace {

gks_status adj_alloc(gks_adjoint* A, double** p)
{
    gks_ctx* c = A->c;
    if (!*p) CK(cudaMalloc(p, c->arr_bytes));
    return GKS_OK;
}

gks_status adj_scratch(gks_adjoint* A)
{
    gks_ctx* c = A->c;
    if (A->lines) return GKS_OK;
    const long long nx = c->desc.nx, ny = c->desc.ny;
    const size_t es = c->desc.precision == GKS_FP32_FLUX ? 4 : 8;
    const long long lines = std::max((nx + 1) * (ny + 4), (ny + 1) * (nx + 4)) * NQ;
    const long long contrib = std::max((nx + 1) * ny, (ny + 1) * nx) * 5 * NQ;
    const long long dcell = std::max((nx + 2) * (ny + 4), (ny + 2) * (nx + 4)) * 20;
    CK(cudaMalloc(&A->lines, lines * es));
    CK(cudaMalloc(&A->contrib, contrib * es));
    CK(cudaMalloc(&A->dcell, dcell * es));
    gks_status s;
    if ((s = adj_alloc(A, &A->lam)) || (s = adj_alloc(A, &A->lams)) || (s = adj_alloc(A, &A->gacc)) ||
        (s = adj_alloc(A, &A->nxt)))
        return s;
    return GKS_OK;
}

// load a ghosted float64 state into the context's W (and its float32 shadow)
gks_status load_state(gks_adjoint* A, const double* Wg)
{
    gks_ctx* c = A->c;
    CK(cudaMemcpyAsync(c->W, Wg, c->arr_bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (c->Wf) {
        const long long n = (long long)c->nv * c->g.plane;
        k_shadow<<<blocks_for(n), 256, 0, c->stream>>>(c->W, c->Wf, n);
        CK(cudaGetLastError());
        ++A->launches;
    }
    return GKS_OK;
}

template <typename T>
gks_status sweep_vjp_t(gks_adjoint* A, AdjDir d)
{
    gks_ctx* c = A->c;
    const HostFlux hf = rt::host_flux(c);
    const FluxParams<T> fp = make_flux_params<T>(hf);
    const TenoT<T> tn = teno_t<T>(rt::teno_params(c, false)), tt = teno_t<T>(rt::teno_params(c, true));
    const GridDev& g = c->g;
    cudaStream_t st = c->stream;
    // launch shapes: x along the unit-stride direction
    auto grid_for = [&](int nnorm, int ntan, dim3 blk, int xmul) {
        const int ex = d.dirn == 0 ? nnorm : ntan, ey = d.dirn == 0 ? ntan : nnorm;
        return dim3((unsigned)((ex * xmul + blk.x - 1) / blk.x), (unsigned)((ey + blk.y - 1) / blk.y));
    };
    const dim3 b256(32, 8), b128(32, 4);
    // the per-cell kernels take the two variable pairs in blockIdx.z
    dim3 gcell = grid_for(d.nn + 2, d.nt + 4, b256, 1);
    gcell.z = 2;
    k_adj_lines<T><<<gcell, b256, 0, st>>>(g, d, tn);
    k_adj_gauss<T><<<grid_for(d.nn + 1, d.nt, b128, 2), b128, 0, st>>>(g, d, fp, tt);
    k_adj_normal<T><<<gcell, b256, 0, st>>>(g, d, tn);
    k_adj_gather<T><<<grid_for(d.nn + 6, d.nt + 4, b256, 1), b256, 0, st>>>(g, d);
    CK(cudaGetLastError());
    A->launches += 4;
    return GKS_OK;
}

// adds to A->gacc the transposed flux Jacobian of both directions at the
// stage input (src), with face cotangents from lam1, lam2
gks_status stage_vjp(gks_adjoint* A, bool stage2_input, const double* lam1, const double* lam2, double cF1,
                     double cD1, double cF2, double cD2)
{
    gks_ctx* c = A->c;
    const bool f32 = c->desc.precision == GKS_FP32_FLUX;
    for (int dirn = 0; dirn < 2; ++dirn) {
        AdjDir d{};
        d.src = stage2_input ? c->Ws : c->W;
        d.srcf = stage2_input ? c->Wsf : c->Wf;
        d.lam1 = lam1;
        d.lam2 = lam2;
        const double h = dirn == 0 ? c->g.dx : c->g.dy;
        d.cF1 = cF1 / h;
        d.cD1 = cD1 / h;
        d.cF2 = cF2 / h;
        d.cD2 = cD2 / h;
        d.lines = A->lines;
        d.contrib = A->contrib;
        d.dcell = A->dcell;
        d.gW = A->gacc;
        d.dirn = dirn;
        if (dirn == 0) {
            d.nn = c->desc.nx; d.nt = c->desc.ny; d.sn = 1; d.st = c->g.pitch;
            d.ihn = 1.0 / c->g.dx; d.iht = 1.0 / c->g.dy;
        } else {
            d.nn = c->desc.ny; d.nt = c->desc.nx; d.sn = c->g.pitch; d.st = 1;
            d.ihn = 1.0 / c->g.dy; d.iht = 1.0 / c->g.dx;
        }
        d.fcF1 = (float)d.cF1;
        d.fcD1 = (float)d.cD1;
        d.fcF2 = (float)d.cF2;
        d.fcD2 = (float)d.cD2;
        d.fihn = (float)d.ihn;
        d.fiht = (float)d.iht;
        gks_status s = f32 ? sweep_vjp_t<float>(A, d) : sweep_vjp_t<double>(A, d);
        if (s) return s;
    }
    const GridDev& g = c->g;
    k_fold_y<<<(4 * (g.nx + 2 * NG) + 127) / 128, 128, 0, c->stream>>>(g, A->gacc);
    k_fold_x<<<(4 * g.ny + 127) / 128, 128, 0, c->stream>>>(g, A->gacc);
    CK(cudaGetLastError());
    A->launches += 2;
    return GKS_OK;
}

size_t wstar_bytes(const gks_ctx* c)
{
    return (size_t)c->nv * c->g.plane * (c->Wsf ? sizeof(float) : sizeof(double));
}

// A->lam <- (dW^{n+1}/dW^n)^T A->lam at the ghosted state Wn with its stage
// state Ws (as the forward pass computed it)
gks_status adjoint_step(gks_adjoint* A, const double* Wn, const void* Ws)
{
    gks_ctx* c = A->c;
    const double dt = A->dt;
    gks_status s;
    if ((s = load_state(A, Wn))) return s;
    void* ws = c->Wsf ? static_cast<void*>(c->Wsf) : static_cast<void*>(c->Ws);
    CK(cudaMemcpyAsync(ws, Ws, wstar_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    if ((s = rt::enqueue_ghosts(c, c->W, c->stream))) return s;
    if ((s = rt::enqueue_ghosts(c, c->Ws, c->stream))) return s;
    // lam* = [d dF/dW*]^T (dt^2/(3h) Delta lam)
    CK(cudaMemsetAsync(A->gacc, 0, c->arr_bytes, c->stream));
    if ((s = stage_vjp(A, true, A->lam, nullptr, 0.0, dt * dt / 3.0, 0.0, 0.0))) return s;
    std::swap(A->lams, A->gacc);
    // stage 1 at W^n with the cotangents of A (lam) and of W* (lam*)
    CK(cudaMemsetAsync(A->gacc, 0, c->arr_bytes, c->stream));
    if ((s = stage_vjp(A, false, A->lam, A->lams, dt, dt * dt / 6.0, 0.5 * dt, dt * dt / 8.0))) return s;
    const long long n = (long long)c->nv * c->g.plane;
    k_sum3<<<blocks_for(n), 256, 0, c->stream>>>(A->lam, A->lams, A->gacc, A->nxt, n);
    CK(cudaGetLastError());
    ++A->launches;
    std::swap(A->lam, A->nxt);
    return GKS_OK;
}

// checkpoints for nsteps steps and the k segment states (W and W*), kept
// for the adjoint's lifetime
gks_status reserve(gks_adjoint* A, int nsteps)
{
    gks_ctx* c = A->c;
    const int ncp = (nsteps + A->k - 1) / A->k;
    while ((int)A->ckpt.size() < ncp) {
        double* p = nullptr;
        if (cudaMalloc(&p, c->arr_bytes) != cudaSuccess) {
            cudaGetLastError();
            return rt::fail(c, GKS_ENOMEM, "no device memory for %d checkpoints", ncp);
        }
        A->ckpt.push_back(p);
    }
    while ((int)A->seg.size() < A->k) {
        double* p = nullptr;
        void* q = nullptr;
        if (cudaMalloc(&p, c->arr_bytes) != cudaSuccess || cudaMalloc(&q, wstar_bytes(c)) != cudaSuccess) {
            cudaFree(p);
            cudaGetLastError();
            return rt::fail(c, GKS_ENOMEM, "no device memory for a %d-step segment", A->k);
        }
        A->seg.push_back(p);
        A->segs.push_back(q);
    }
    return GKS_OK;
}

gks_status check_supported(gks_ctx* c)
{
    if (c->desc.dim != 2) return rt::fail(c, GKS_EUNSUPPORTED, "the adjoint is built for 2-D grids");
    if (c->sch.tau_mode != GKS_TAU_ZERO)
        return rt::fail(c, GKS_EUNSUPPORTED, "the adjoint is built for the collision-free flux (tau_mode = zero)");
    if (c->sch.recon != GKS_RECON_TENO_D || c->sch.charvars)
        return rt::fail(c, GKS_EUNSUPPORTED,
                        "the adjoint is built for component-wise TENO-D (frozen stencil selection)");
    for (int k = 0; k < 4; ++k)
        if (c->desc.bc[k] > GKS_BC_REFLECT)
            return rt::fail(c, GKS_EUNSUPPORTED, "the adjoint is built for the copying boundary rules");
    if (c->sch.merge != GKS_MERGE_KINETIC)
        return rt::fail(c, GKS_EUNSUPPORTED, "the adjoint is built for the kinetic merge");
    return GKS_OK;
}

gks_status sync_check(gks_ctx* c)
{
    gks_diag d;
    return gks_get_diagnostics(c, &d);
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

gks_status gks_adjoint_create(gks_ctx* c, int checkpoint_every, gks_adjoint** out)
{
    if (!c || !out || checkpoint_every < 1) return GKS_EINVAL;
    *out = nullptr;
    gks_status s = check_supported(c);
    if (s) return s;
    gks_adjoint* A = new (std::nothrow) gks_adjoint();
    if (!A) return GKS_ENOMEM;
    A->c = c;
    A->k = checkpoint_every;
    if ((s = adj_scratch(A)) || (s = adj_alloc(A, &A->WN))) {
        gks_adjoint_destroy(A);
        cudaGetLastError();
        return s == GKS_ECUDA ? GKS_ENOMEM : s;
    }
    *out = A;
    return GKS_OK;
}

void gks_adjoint_destroy(gks_adjoint* A)
{
    if (!A) return;
    if (A->seg_exec) cudaGraphExecDestroy(A->seg_exec);
    for (double* p : A->ckpt) cudaFree(p);
    for (double* p : A->seg) cudaFree(p);
    for (void* p : A->segs) cudaFree(p);
    cudaFree(A->WN);
    cudaFree(A->lam);
    cudaFree(A->lams);
    cudaFree(A->gacc);
    cudaFree(A->nxt);
    cudaFree(A->lines);
    cudaFree(A->contrib);
    cudaFree(A->dcell);
    delete A;
}

gks_status gks_adjoint_forward(gks_adjoint* A, int nsteps, double dt)
{
    const NvtxRange range("gks_adjoint_forward");
    if (!A || nsteps < 1 || !(dt > 0.0) || !std::isfinite(dt)) return GKS_EINVAL;
    gks_ctx* c = A->c;
    gks_status s = check_supported(c);
    if (s) return s;
    if ((s = reserve(A, nsteps))) return s;
    A->have_forward = false;
    for (int n = 0; n < nsteps; ++n) {
        if (n % A->k == 0) CK(cudaMemcpyAsync(A->ckpt[n / A->k], c->W, c->arr_bytes, cudaMemcpyDeviceToDevice, c->stream));
        if ((s = gks_step(c, dt))) return s;
    }
    CK(cudaMemcpyAsync(A->WN, c->W, c->arr_bytes, cudaMemcpyDeviceToDevice, c->stream));
    if ((s = sync_check(c))) return s;
    A->nsteps = nsteps;
    A->dt = dt;
    A->have_forward = true;
    return GKS_OK;
}

namespace {

// recompute a segment of len steps from the state in the context, stage by
// stage (the same kernels and W as the forward pass's steps), keeping W and
// W* of every step, then reverse its steps
gks_status run_segment(gks_adjoint* A, int len)
{
    gks_ctx* c = A->c;
    gks_status s;
    const void* ws = c->Wsf ? static_cast<const void*>(c->Wsf) : static_cast<const void*>(c->Ws);
    for (int n = 0; n < len; ++n) {
        CK(cudaMemcpyAsync(A->seg[n], c->W, c->arr_bytes, cudaMemcpyDeviceToDevice, c->stream));
        if ((s = gks_stage(c, 1, A->dt))) return s;
        CK(cudaMemcpyAsync(A->segs[n], ws, wstar_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
        if (n + 1 < len && (s = gks_stage(c, 2, A->dt))) return s;
    }
    for (int n = len - 1; n >= 0; --n)
        if ((s = adjoint_step(A, A->seg[n], A->segs[n]))) return s;
    return GKS_OK;
}

// capture run_segment(k) as a graph (once per dt and context parameters);
// leaves seg_exec null where the segment's buffer rotation does not return
// to its start (odd k) so that replays would read the wrong buffers
gks_status segment_graph(gks_adjoint* A)
{
    gks_ctx* c = A->c;
    if (A->seg_eager) return GKS_OK;
    if (A->seg_exec && A->seg_dt == A->dt && A->seg_version == c->param_version) return GKS_OK;
    if (A->seg_exec) {
        cudaGraphExecDestroy(A->seg_exec);
        A->seg_exec = nullptr;
    }
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    double* const before[4] = {A->lam, A->lams, A->gacc, A->nxt};
    const long long L0 = A->launches, C0 = c->launches;
    cudaStream_t keep = c->stream;
    c->stream = c->cap_stream;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    gks_status s = run_segment(A, A->k);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->capturing = false;
    c->stream = keep;
    A->seg_kernels = A->launches - L0;
    A->seg_ctx_kernels = c->launches - C0;
    A->launches = L0;  // captured, not launched
    c->launches = C0;
    const bool in_place = A->lam == before[0] && A->lams == before[1] && A->gacc == before[2] && A->nxt == before[3];
    A->lam = before[0], A->lams = before[1], A->gacc = before[2], A->nxt = before[3];
    if (s != GKS_OK || e != cudaSuccess || !in_place) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (s != GKS_OK) return s;
        if (e != cudaSuccess) return rt::fail(c, GKS_ECUDA, "capturing the adjoint segment: %s", cudaGetErrorString(e));
        A->seg_eager = true;
        return GKS_OK;
    }
    e = cudaGraphInstantiate(&A->seg_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    A->seg_dt = A->dt;
    A->seg_version = c->param_version;
    return GKS_OK;
}

}  // namespace

gks_status gks_adjoint_backward(gks_adjoint* A, const double* gWN, double* gW0, int on_device)
{
    const NvtxRange range("gks_adjoint_backward");
    if (!A || !gWN || !gW0) return GKS_EINVAL;
    gks_ctx* c = A->c;
    if (!A->have_forward) return rt::fail(c, GKS_EINVAL, "gks_adjoint_backward needs a completed forward pass");
    gks_status s;
    if ((s = reserve(A, A->nsteps))) return s;
    CK(cudaMemsetAsync(A->lam, 0, c->arr_bytes, c->stream));
    if ((s = rt::copy_interior(c, A->lam, gWN, on_device, true))) return s;
    const int ncp = (A->nsteps + A->k - 1) / A->k;
    for (int sgi = ncp - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * A->k, n1 = std::min(n0 + A->k, A->nsteps);
        const NvtxRange seg_range("adjoint segment");
        if ((s = load_state(A, A->ckpt[sgi]))) return s;
        if (n1 - n0 == A->k) {
            if ((s = segment_graph(A))) return s;
            if (A->seg_exec) {
                CK(cudaGraphLaunch(A->seg_exec, c->stream));
                A->launches += A->seg_kernels;
                c->launches += A->seg_ctx_kernels;
                continue;
            }
        }
        if ((s = run_segment(A, n1 - n0))) return s;
    }
    if ((s = rt::copy_interior(c, A->lam, gW0, on_device, false))) return s;
    // leave the context at the forward pass's final state
    if ((s = load_state(A, A->WN))) return s;
    return sync_check(c);
}

long long gks_adjoint_launches(const gks_adjoint* A) { return A ? A->launches : 0; }

gks_status gks_adjoint_reserve(gks_adjoint* A, int nsteps)
{
    if (!A || nsteps < 1) return GKS_EINVAL;
    return reserve(A, nsteps);
}

gks_status gks_vjp_step(gks_ctx* c, const double* W, const double* gout, double* gin, double dt, int on_device)
{
    if (!c || !W || !gout || !gin || !(dt > 0.0) || !std::isfinite(dt)) return GKS_EINVAL;
    gks_adjoint* A = nullptr;
    gks_status s = gks_adjoint_create(c, 1, &A);
    if (s) return s;
    if (!(s = gks_set_state(c, W, on_device)) && !(s = gks_adjoint_forward(A, 1, dt)))
        s = gks_adjoint_backward(A, gout, gin, on_device);
    gks_adjoint_destroy(A);
    return s;
}

}  // extern "C"
