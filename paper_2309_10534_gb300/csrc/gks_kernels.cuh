// gks_kernels.cuh -- kernels of one S2O4 step of the TENO-D gas-kinetic scheme.
//
// Data layout (HBM): conserved variables, float64, SoA with three ghost
// layers: W[v][j][i], v < nvar, j < gy = ny + 6 (1-D: gy = 1), i < pitch
// (pitch >= nx + 6, a multiple of 16 doubles).  Interior cell (0, 0) sits at
// (j, i) = (3, 3) (1-D: i = 3).  Three such arrays live on the device:
//   W  -- the state W^n (and W^{n+1} after stage 2)
//   Ws -- the stage state W*
//   Ac -- the stage accumulator W^n - dt/dx d(F + dt/6 dF)   (Sec. 2.2)
// Kernels of one step (2-D): ghost(W), sweep-x s1, sweep-y s1, ghost(Ws),
// sweep-x s2, sweep-y s2 (+ CFL reduction), commit.  1-D: ghost, stage 1,
// ghost, stage 2, commit.  A sweep computes every face flux of its tile
// once, in shared memory, so both neighbours of a face apply bit-identical
// values and the update is conservative.
#pragma once

#include "gks_device.cuh"
#include "gks_pair.cuh"

namespace gks {

constexpr int NG = 3;

struct DevState {
    double t, dt, t_end, cfl;
    unsigned long long sigma;      // max over cells of the signal rate, as ordered bits
    unsigned long long fallbacks;  // positivity fallbacks taken
    long long steps, max_steps;
    unsigned int err;              // bit 0 non-physical update, bit 1 fallback failed
    unsigned int done;             // 1: t_end or max_steps reached; kernels return early
    unsigned int fixed_dt;         // 1: keep dt (caller-given), 0: CFL time step
    unsigned int pad;
};

// state-setting boundary rules: conserved states (energy in slot 3) and the
// moving oblique shock x_s(y, t) = x0 + (y - oy) cot + vx t
struct BcStates {
    double in[4], pre[4];
    double x0, cot, vx;
};

struct GridDev {
    int dim, nx, ny, pitch, gy;
    long long plane;   // elements per variable plane = gy * pitch
    double dx, dy;
    int bc[4];
    double gamma, mu;
    double ox, oy;     // domain origin (cell centres at ox + (i + 1/2) dx)
    BcStates bs;
};

constexpr int BC_INFLOW = 5, BC_WALL_AFTER_X0 = 6, BC_MOVING_SHOCK = 7;

// the state a state-setting rule gives the ghost centred at (x, y) at time t,
// or nullptr where the rule copies from the interior
__device__ __forceinline__ const double* ghost_state(const GridDev& g, int bc, double x, double y, double t)
{
    if (bc == BC_INFLOW) return g.bs.in;
    if (bc == BC_WALL_AFTER_X0) return (x < g.bs.x0) ? g.bs.in : nullptr;
    if (bc == BC_MOVING_SHOCK) return (x < g.bs.x0 + (y - g.oy) * g.bs.cot + g.bs.vx * t) ? g.bs.in : g.bs.pre;
    return nullptr;
}

// ------------------------------------------------------------------ ghosts
// source index of ghost position g (ghosted coordinate) along a line of n
// interior cells, and the velocity flips the rule implies
__device__ __forceinline__ int ghost_src(int bc, int n, int g, bool& flip_n, bool& flip_all)
{
    flip_n = flip_all = false;
    if (g >= NG && g < NG + n) return g;
    const bool low = g < NG;
    switch (bc) {
    case 0:  // periodic
        return NG + (((g - NG) % n) + n) % n;
    case 1:  // zero gradient
        return low ? NG : NG + n - 1;
    case 3:  // no-slip adiabatic wall
        flip_all = true;
        return low ? 2 * NG - 1 - g : 2 * (NG + n) - 1 - g;
    default:  // symmetry / reflect
        flip_n = true;
        return low ? 2 * NG - 1 - g : 2 * (NG + n) - 1 - g;
    }
}

// ------------------------------------------------------------------ CFL rate
// sigma = max((|U| + a)/h, 4 nu / h^2), dt = cfl / sigma  (Sec. 5), in the
// kernel's arithmetic type (the float32 path takes its time step in float32;
// only the state and its accumulation are float64)
// U^2 + V^2 with both products rounded before the sum (no fused
// multiply-add): the same bits for (U, V) and (V, U), so a sweep that holds
// the state in its local frame and the grid-order reduction pick the same
// time step
template <typename T>
__device__ __forceinline__ T speed2(T U, T V)
{
    if constexpr (sizeof(T) == 4) return __fmul_rn(U, U) + __fmul_rn(V, V);
    else return __dmul_rn(U, U) + __dmul_rn(V, V);
}

// division and square root rounded to nearest whatever the unit's float
// flags: the sweeps' units take fast float32 division and square root, the
// reduction before a call's first step (k_sigma) does not, and both must
// form the same time step
template <typename T>
__device__ __forceinline__ T div_rn(T a, T b)
{
    if constexpr (sizeof(T) == 4) return __fdiv_rn(a, b);
    else return __ddiv_rn(a, b);
}
template <typename T>
__device__ __forceinline__ T sqrt_rn(T a)
{
    if constexpr (sizeof(T) == 4) return __fsqrt_rn(a);
    else return __dsqrt_rn(a);
}

template <typename T, typename WT = double>
__device__ __forceinline__ T cell_sigma(const WT* w, int dim, T gamma, T mu, T h, unsigned int& err)
{
    const T r = (T)w[0], ir = div_rn(T(1), r);
    const T U = (T)w[1] * ir, V = (dim == 2) ? (T)w[2] * ir : T(0);
    const T E = (T)(dim == 2 ? w[3] : w[2]);  // no dynamic index: keeps w in registers
    const T q = speed2(U, V);
    const T p = (gamma - T(1)) * (E - T(0.5) * r * q);
    if (!(r > T(0) && p > T(0) && isfinite(p))) err |= 1u;
    const T a = sqrt_rn(gamma * p * ir);
    const T ih = div_rn(T(1), h);
    T s = (sqrt_rn(q) + a) * ih;
    if (mu > T(0)) s = fmax(s, T(4) * mu * ir * ih * ih);
    return s;
}

// Block reduction of the CFL rate (only when with_sigma), the error word and
// the fallback count; one atomic of each per block.
template <int NT, typename T>
__device__ __forceinline__ void block_commit(T s, bool with_sigma, unsigned int err, unsigned int nfb, DevState* ds)
{
    __shared__ T red_s[NT / 32];
    __shared__ unsigned int red_e[NT / 32], red_f[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (with_sigma) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        err |= __shfl_xor_sync(0xffffffffu, err, o);
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red_s[w] = s; red_e[w] = err; red_f[w] = nfb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < NT / 32; ++k) {
            if (with_sigma) s = fmax(s, red_s[k]);
            err |= red_e[k];
            nfb += red_f[k];
        }
        const double sd = (double)s;
        if (with_sigma && (sd > 0.0 || sd != sd))
            atomicMax(&ds->sigma, (unsigned long long)__double_as_longlong(sd));
        if (err) atomicOr(&ds->err, err);
        if (nfb) atomicAdd(&ds->fallbacks, (unsigned long long)nfb);
    }
}

// ------------------------------------------------------------------ stage arithmetic
// Stage combinations of the face flux F and its time derivative dF
// (Sec. 2.2): stage 1: g0 = F/2 + dt/8 dF (for W*), g1 = F + dt/6 dF (for the
// accumulator); stage 2: g0 = dt/3 dF.  Explicit fused multiply-adds, here
// and in the updates below, give every kernel the same rounding.
template <typename T>
__device__ __forceinline__ void stage_comb(int stage, T F, T dF, T dt, T& g0, T& g1)
{
    if (stage == 1) {
        g0 = fma(T(0.125) * dt, dF, T(0.5) * F);
        g1 = fma(dt * T(1.0 / 6.0), dF, F);
    } else {
        g0 = (dt * T(1.0 / 3.0)) * dF;
        g1 = T(0);
    }
}
// float64 path: W* = W - cx dG0, A = W - cx dG1; stage 2: W = A - cx dG0
__device__ __forceinline__ double upd64(double w, double cx, double dG) { return fma(-cx, dG, w); }
// float32 path: W* = W - cx dG0 and the increment cx dG1 in float32; stage 2:
// W = W - (increment + cx dG0), the sum in float32, the update in float64
__device__ __forceinline__ float wstar32(float w, float cx, float dG) { return fmaf(-cx, dG, w); }
__device__ __forceinline__ double wnew32(double w, float inc, float cx, float dG)
{
    return w - (double)fmaf(cx, dG, inc);
}

// ------------------------------------------------------------------ 1-D stage
// float64 path: W* and the accumulator A are float64 arrays.
// float32 path (as the 2-D one): W* is only the stage-2 reconstruction input,
// so it is formed and kept in float32, and the accumulator is kept as the
// float32 increment dt/dx d(F + dt/6 dF); the only float64 arithmetic is the
// final update W^{n+1} = W^n - (increment + dt/dx d(dt/3 dF*)).
struct Stage1DArgs {
    const double* src;   // float64 reconstruction input (W; float64 path stage 2: W*), ghosts filled
    const float* srcf;   // float32 path: stage 1 the float32 shadow of W (or nullptr: src,
                         // converted), stage 2 W* (float32); ghosts filled
    double* out0;        // float64 path stage 1: W*; stage 2: the new state
    double* out1;        // float64 path stage 1: accumulator A
    const double* acc;   // float64 path stage 2: accumulator A
    float* out0f;        // float32 path stage 1: W*; stage 2: the new state's float32
                         // shadow (or nullptr)
    float* out1f;        // float32 path stage 1: accumulator increment
    const float* accf;   // float32 path stage 2: accumulator increment
    const double* base;  // float32 path stage 2: W^n
    int stage;
    int with_sigma;      // stage 2: reduce the CFL rate of the new state
    double idx;          // 1 / dx
};

template <typename T, bool NONEQ, bool PRFIX, int TN, int REC = 0>
__global__ void __launch_bounds__(TN + 2) k1d_stage(GridDev g, Stage1DArgs a, FluxParams<T> fp, TenoT<T> tn,
                                                    DevState* ds)
{
    if (ds->done) return;
    // TN cells per block, TN + 2 threads: the TN + 2 reconstructed cells,
    // TN + 1 faces and TN updated cells each take one pass of the block
    constexpr int NT = TN + 2;
    const double dt = ds->dt;
    // dt and dt/dx in the arithmetic type, converted once per block (a
    // float64 -> float32 conversion runs on the slow float64 pipe)
    __shared__ T s_scal[6];  // dt, dt/dx, 1/dx, gamma, mu, dx
    if (threadIdx.x == 0) {
        s_scal[0] = (T)dt;
        s_scal[1] = (T)(dt * a.idx);
        s_scal[2] = (T)a.idx;
        s_scal[3] = (T)g.gamma;
        s_scal[4] = (T)g.mu;
        s_scal[5] = (T)g.dx;
    }
    __shared__ T sq[3][TN + 6];
    __shared__ T sL[3][2][TN + 1], sR[3][2][TN + 1];  // [var][value, slope][face]
    __shared__ T sG[2][3][TN + 1];                     // face fluxes for the update
    const int i0 = blockIdx.x * TN;
    const int tid = threadIdx.x;
    const int gx = g.nx + 2 * NG;
    const int slot[3] = {0, 1, 3};

    const int pl = (int)g.plane;  // a 1-D plane is one ghosted row
    // one loop per source type: a per-element choice between the float32
    // and the converted float64 source was compiled as both, and every
    // element then paid a float64 -> float32 conversion on the slow float64
    // pipe whichever source it took
    auto load = [&](auto src) {
        for (int k = tid; k < 3 * (TN + 6); k += NT) {
            const int v = k / (TN + 6), c = k % (TN + 6);
            const int gi = i0 + c;  // ghosted index of cell i0 - 3 + c
            sq[v][c] = gi < gx ? (T)src[v * pl + gi] : T(0);
        }
    };
    if constexpr (sizeof(T) == 4) {
        if (a.srcf) load(a.srcf);
        else load(a.src);
    } else {
        load(a.src);
    }
    __syncthreads();
    fp.dt = s_scal[0];
    const T idx_ = s_scal[2];
    if constexpr (REC == REC_TENO_CHAR) {
        // phase 1 in characteristic variables: per face f (between interior
        // i0 + f - 1 and i0 + f), the six cells around it projected with the
        // face's basis, both sides reconstructed
        for (int f = tid; f <= TN; f += NT) {
            T w[6][4], vl[4], dl[4], vr[4], dr[4];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                w[c][0] = sq[0][f + c];
                w[c][1] = sq[1][f + c];
                w[c][2] = T(0);
                w[c][3] = sq[2][f + c];
            }
            char_face<T, 1>(w, tn, fp.gm1, vl, dl, vr, dr);
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                sL[v][0][f] = vl[slot[v]];
                sL[v][1][f] = dl[slot[v]] * idx_;
                sR[v][0][f] = vr[slot[v]];
                sR[v][1][f] = dr[slot[v]] * idx_;
            }
        }
    } else {
        // phase 1: reconstruction per cell c (interior i0 - 1 + c), both faces
        for (int c = tid; c < TN + 2; c += NT) {
            T q[3][5], vp[3], dp[3], vm[3], dm[3];
#pragma unroll
            for (int v = 0; v < 3; ++v)
#pragma unroll
                for (int s = 0; s < 5; ++s) q[v][s] = sq[v][c + s];
            recon_cell3<REC>(q, tn, vp, dp, vm, dm);
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                if (c <= TN) { sL[v][0][c] = vp[v]; sL[v][1][c] = dp[v] * idx_; }
                if (c >= 1) { sR[v][0][c - 1] = vm[v]; sR[v][1][c - 1] = dm[v] * idx_; }
            }
        }
    }
    __syncthreads();
    // phase 2: flux at face f (between interior i0+f-1 and i0+f)
    unsigned int nfb = 0, err = 0;
    for (int f = tid; f <= TN; f += NT) {
        if (i0 + f > g.nx) continue;  // padding past the last face
        Side<T> L, R;
#pragma unroll
        for (int k = 0; k < 4; ++k) { L.W[k] = L.Wn[k] = L.Wt[k] = R.W[k] = R.Wn[k] = R.Wt[k] = T(0); }
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            L.W[slot[v]] = sL[v][0][f];
            L.Wn[slot[v]] = sL[v][1][f];
            R.W[slot[v]] = sR[v][0][f];
            R.Wn[slot[v]] = sR[v][1][f];
        }
        if (!physical<T, 1>(L.W, fp.gm1)) {
#pragma unroll
            for (int v = 0; v < 3; ++v) { L.W[slot[v]] = sq[v][f + 2]; L.Wn[slot[v]] = T(0); }
            ++nfb;
            if (!physical<T, 1>(L.W, fp.gm1)) err |= 2u;
        }
        if (!physical<T, 1>(R.W, fp.gm1)) {
#pragma unroll
            for (int v = 0; v < 3; ++v) { R.W[slot[v]] = sq[v][f + 3]; R.Wn[slot[v]] = T(0); }
            ++nfb;
            if (!physical<T, 1>(R.W, fp.gm1)) err |= 2u;
        }
        T F[4], dF[4];
        if constexpr (rec_conventional(REC)) {
            // conventional path: equilibrium slope from the cell averages
            // i-1 .. i+2 around the face by the linear Eq. (3.12)
            T w0n[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int v = 0; v < 3; ++v)
                w0n[slot[v]] = (T(1.25) * (sq[v][f + 3] - sq[v][f + 2]) - T(1.0 / 12.0) * (sq[v][f + 4] - sq[v][f + 1]))
                             * idx_;
            point_flux<T, 1, NONEQ, PRFIX>(L, R, fp, F, dF, w0n);
        } else {
            point_flux<T, 1, NONEQ, PRFIX>(L, R, fp, F, dF);
        }
        const T tdt = s_scal[0];
#pragma unroll
        for (int v = 0; v < 3; ++v) stage_comb<T>(a.stage, F[slot[v]], dF[slot[v]], tdt, sG[0][v][f], sG[1][v][f]);
    }
    __syncthreads();
    // phase 3: update
    T sig = T(0);
    const double cx = dt * a.idx;
    const T cxt = s_scal[1];
    for (int c = tid; c < TN; c += NT) {
        const int i = i0 + c;
        if (i >= g.nx) continue;
        const int o = i + NG;
        if constexpr (sizeof(T) == 4) {
            if (a.stage == 1) {
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    a.out0f[v * pl + o] = wstar32(sq[v][c + 3], cxt, sG[0][v][c + 1] - sG[0][v][c]);
                    a.out1f[v * pl + o] = cxt * (sG[1][v][c + 1] - sG[1][v][c]);
                }
            } else {
                T w[3];
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int gi = v * pl + o;
                    const double r = wnew32(a.base[gi], a.accf[gi], cxt, sG[0][v][c + 1] - sG[0][v][c]);
                    a.out0[gi] = r;
                    w[v] = (T)r;
                    if (a.out0f) a.out0f[gi] = w[v];
                }
                if (a.with_sigma) sig = fmax(sig, cell_sigma<T, T>(w, 1, s_scal[3], s_scal[4], s_scal[5], err));
            }
        } else if (a.stage == 1) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const double w = a.src[v * pl + o];
                a.out0[v * pl + o] = upd64(w, cx, (double)(sG[0][v][c + 1] - sG[0][v][c]));
                a.out1[v * pl + o] = upd64(w, cx, (double)(sG[1][v][c + 1] - sG[1][v][c]));
            }
        } else {
            double w[4];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const double r = upd64(a.acc[v * pl + o], cx, (double)(sG[0][v][c + 1] - sG[0][v][c]));
                a.out0[v * pl + o] = r;
                w[v] = r;
            }
            if (a.with_sigma) sig = fmax(sig, cell_sigma<T>(w, 1, s_scal[3], s_scal[4], s_scal[5], err));
        }
    }
    if (NT % 32 == 0) block_commit<NT, T>(sig, a.with_sigma != 0, err, nfb, ds);
}

// ------------------------------------------------------------------ 2-D sweep
// One stage = x sweep (pass 0) then y sweep (pass 1).  The x sweep stores its
// flux-divergence increments dt/dx dG in the kernel's arithmetic type (inc0,
// inc1); the y sweep adds its own.
// float64 path (one float64 update per value):
//   stage 1: W* = W - (inc0 + dt/dy dG1),  A = W - (inc1 + dt/dy dG2)
//   stage 2: W  = A - (inc0 + dt/dy dG)
// float32 path: W* is only the stage-2 reconstruction input, so it is formed
// in float32 from the float32 shadow of W, and the accumulator stays an
// increment; the only float64 arithmetic is the final update of W:
//   stage 1: W*f = Wf - (inc0 + dt/dy dG1),  inc1 <- inc1 + dt/dy dG2
//   stage 2: W   = W - (inc1 + inc0 + dt/dy dG)   (and its shadow Wf)
struct SweepArgs {
    const double* src;   // reconstruction input (W or W*), ghosts filled
    const float* srcf;   // float32 path: float32 shadow of src (ghosts filled)
    const float* basef;  // float32 path, y sweep of stage 1: float32 shadow of W
    const double* base;  // y sweep: W (stage 1) or A (stage 2)
    double* out0;        // y sweep, stage 1: W*; stage 2: W
    float* out0f;        // float32 path, y sweep: float32 shadow of out0
    double* out1;        // y sweep, stage 1: A
    void* inc0;          // increments, arithmetic type, same ghosted layout
    void* inc1;          // (stage 1 only)
    int stage, pass;     // pass 0: x sweep (first), 1: y sweep (second)
    int dirn;            // 0: faces normal to x, 1: faces normal to y
    int nn, nt;          // cells along the normal / tangential direction
    long long sn, st;    // element strides along normal / tangential
    double ihn, iht;     // inverse cell sizes along normal / tangential
    double hmin;         // min(dx, dy) for the CFL rate
    int with_sigma;
};

// global variable index of local variable v (swap: faces normal to y)
__device__ __forceinline__ int gvar(int v, bool swap) { return (swap && (v == 1 || v == 2)) ? 3 - v : v; }

template <typename T, int TN, int TT, bool CONV = false> struct SweepSmem {
    T w[4][TT + 4][TN + 6];           // cells: tangential rows t0-2.., normal n0-3..
    T rec[4][4][TT + 4][TN + 1];      // [vL, sL, vR, sR][var][row][face]
    T flux[8 * (TN + 1) * (TT + 1)];  // face fluxes for the update (layout: sfi)
    // conventional path: line-averaged equilibrium state and its normal
    // slope per face and row (Step 2)
    T w0[CONV ? 2 : 1][4][CONV ? TT + 4 : 1][CONV ? TN + 1 : 1];
};

template <typename T, bool NONEQ, bool PRFIX, int TN, int TT, int REC = 0>
__global__ void __launch_bounds__(TT * (TN + 1), (sizeof(T) == 4) ? 1024 / (TT * (TN + 1)) : 1)
k2d_sweep(GridDev g, SweepArgs a, FluxParams<T> fp, TenoT<T> tnn, TenoT<T> tnt, DevState* ds)
{
    if (ds->done) return;
    constexpr int NT = TT * (TN + 1);    // one thread per (face, row) pair
    constexpr int NF = TN + 1;           // faces per tile row
    constexpr int NP = TT * NF;          // (face, row) pairs
    static_assert(NP == NT, "one (face,row) pair per thread");
    constexpr bool CONV = rec_conventional(REC);
    constexpr int RB = rec_base(REC);  // the tangential (per-quantity) reconstruction
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem<T, TN, TT, CONV>& sm = *reinterpret_cast<SweepSmem<T, TN, TT, CONV>*>(smem_raw);
    // face fluxes for the update: [k][row][face] for x faces; [k][face][row]
    // (rows padded) for y faces, so that phase 3 runs along the unit-stride x
    // direction in both sweeps
    T* sF = sm.flux;
    const bool fy = a.dirn != 0;
    auto sfi = [&](int k, int r, int f) { return fy ? (k * NF + f) * (TT + 1) + r : (k * TT + r) * NF + f; };

    const int tid = threadIdx.x;
    // the stage's scalars in the arithmetic type, converted once per block
    // (a float64 -> float32 conversion runs on the slow float64 pipe):
    // dt, dt/h_n, 1/h_n, 1/h_t, gamma, mu, min(h_n, h_t); visible after the
    // load phase's barrier
    __shared__ T s_scal[7];
    if (tid == 0) {
        const double dt = ds->dt;
        s_scal[0] = (T)dt;
        s_scal[1] = (T)(dt * a.ihn);
        s_scal[2] = (T)a.ihn;
        s_scal[3] = (T)a.iht;
        s_scal[4] = (T)g.gamma;
        s_scal[5] = (T)g.mu;
        s_scal[6] = (T)a.hmin;
    }
    const int n0 = blockIdx.x * TN, t0 = blockIdx.y * TT;
    // local frame: normal momentum first; y faces swap the two momentum components
    const bool swap = a.dirn != 0;
    // offsets within one variable plane fit in 32 bits; each variable's plane
    // is reached through its own base pointer
    const int org = NG * g.pitch + NG;  // interior (0,0)
    const int sn = (int)a.sn, st = (int)a.st;
    const long long pv1 = (long long)gvar(1, swap) * g.plane, pv2 = (long long)gvar(2, swap) * g.plane;
    const long long pv3 = 3 * g.plane;

    // load cells (normal n0-3 .. n0+TN+2, tangential t0-2 .. t0+TT+1); the
    // thread index runs fastest along the unit-stride direction
    {
        constexpr int CN = TN + 6, CT = TT + 4, NCELL = CN * CT;
        for (int k = tid; k < 4 * NCELL; k += NT) {
            const int v = k / NCELL, e = k % NCELL;
            int cn, ct;
            if (a.dirn == 0) { ct = e / CN; cn = e % CN; } else { cn = e / CT; ct = e % CT; }
            const int in = n0 - 3 + cn, it = t0 - 2 + ct;
            T val = T(0);
            if (in < a.nn + 3 && it < a.nt + 2) {  // ghosted extent (negative side is covered by ghosts)
                const long long pv = v == 0 ? 0 : (v == 1 ? pv1 : (v == 2 ? pv2 : pv3));
                const int off = org + in * sn + it * st;
                if constexpr (sizeof(T) == 4) val = (a.srcf + pv)[off];
                else val = (a.src + pv)[off];
            }
            sm.w[v][ct][cn] = val;
        }
    }
    __syncthreads();
    fp.dt = s_scal[0];

    // phase 1: normal TENO-D per (cell, row, var): cell c <-> normal n0-1+c
    if constexpr (REC == REC_TENO_CHAR) {
        // characteristic variables: per (face, row), the six cells around
        // face f (between normal n0-1+f and n0+f) projected with the face's
        // basis, both sides reconstructed
        const T ih = s_scal[2];
        constexpr int NR = TT + 4;
        for (int k = tid; k < NF * NR; k += NT) {
            const int r = k / NF, f = k % NF;
            T w[6][4], vl[4], dl[4], vr[4], dr[4];
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int v = 0; v < 4; ++v) w[c][v] = sm.w[v][r][f + c];
            char_face<T, 2>(w, tnn, fp.gm1, vl, dl, vr, dr);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                sm.rec[0][v][r][f] = vl[v];
                sm.rec[1][v][r][f] = dl[v] * ih;
                sm.rec[2][v][r][f] = vr[v];
                sm.rec[3][v][r][f] = dr[v] * ih;
            }
        }
    } else if constexpr (sizeof(T) == 4 && REC <= 1) {
        // float32 TENO-D / WENO5-AO: variables (0, 1) and (2, 3) as packed pairs
        const float ih = s_scal[2];
        constexpr int NC = TN + 2, NR = TT + 4;
        for (int k = tid; k < 2 * NC * NR; k += NT) {
            const int vv = 2 * (k / (NC * NR)), e = k % (NC * NR);
            const int r = e / NC, c = e % NC;
            f2 q[5];
#pragma unroll
            for (int s = 0; s < 5; ++s) q[s] = f2(sm.w[vv][r][c + s], sm.w[vv + 1][r][c + s]);
            f2 vp, dp, vm, dm;
            packed_faces<REC>(q, tnn, vp, dp, vm, dm);
            const f2 dpi = dp * f2(ih), dmi = dm * f2(ih);
            if (c <= TN) {
                sm.rec[0][vv][r][c] = vp.x(); sm.rec[0][vv + 1][r][c] = vp.y();
                sm.rec[1][vv][r][c] = dpi.x(); sm.rec[1][vv + 1][r][c] = dpi.y();
            }
            if (c >= 1) {
                sm.rec[2][vv][r][c - 1] = vm.x(); sm.rec[2][vv + 1][r][c - 1] = vm.y();
                sm.rec[3][vv][r][c - 1] = dmi.x(); sm.rec[3][vv + 1][r][c - 1] = dmi.y();
            }
        }
    } else {
        const T ih = s_scal[2];
        constexpr int NC = TN + 2, NR = TT + 4;
        for (int k = tid; k < 4 * NC * NR; k += NT) {
            const int v = k / (NC * NR), e = k % (NC * NR);
            const int r = e / NC, c = e % NC;
            T q[5];
#pragma unroll
            for (int s = 0; s < 5; ++s) q[s] = sm.w[v][r][c + s];
            TenoSel<T> S;
            rec_select<REC>(q, tnn, S);
            T vp, dp, vm, dm;
            rec_faces<REC>(q, S, vp, dp, vm, dm);
            if (c <= TN) { sm.rec[0][v][r][c] = vp; sm.rec[1][v][r][c] = dp * ih; }
            if (c >= 1) { sm.rec[2][v][r][c - 1] = vm; sm.rec[3][v][r][c - 1] = dm * ih; }
        }
    }
    __syncthreads();

    unsigned int nfb = 0, err = 0;
    if constexpr (CONV) {
        // phase 1b (conventional path, Step 2): per face and row, the
        // line-averaged equilibrium state by the kinetic merge of the face
        // values (a non-physical side takes its adjacent cell average), and
        // its normal slope by Eq. (3.12) on the row's cell averages
        const T ih = s_scal[2];
        for (int k = tid; k < NF * (TT + 4); k += NT) {
            const int r = k / NF, f = k % NF;
            // faces n0+f <= nn on rows t0-2+r <= nt+1 (ghosted extent) exist;
            // the rest of the tile is padding that no Gauss point reads
            if (n0 + f > a.nn || t0 - 2 + r > a.nt + 1) continue;
            T wl[4], wr[4], w0[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) { wl[v] = sm.rec[0][v][r][f]; wr[v] = sm.rec[2][v][r][f]; }
            if (!physical<T, 2>(wl, fp.gm1)) {
#pragma unroll
                for (int v = 0; v < 4; ++v) wl[v] = sm.w[v][r][f + 2];
                if (!physical<T, 2>(wl, fp.gm1)) err |= 2u;
            }
            if (!physical<T, 2>(wr, fp.gm1)) {
#pragma unroll
                for (int v = 0; v < 4; ++v) wr[v] = sm.w[v][r][f + 3];
                if (!physical<T, 2>(wr, fp.gm1)) err |= 2u;
            }
            merge_values<T, 2>(wl, wr, fp, w0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                sm.w0[0][v][r][f] = w0[v];
                sm.w0[1][v][r][f] = (T(1.25) * (sm.w[v][r][f + 3] - sm.w[v][r][f + 2])
                                     - T(1.0 / 12.0) * (sm.w[v][r][f + 4] - sm.w[v][r][f + 1])) * ih;
            }
        }
        __syncthreads();
    }

    // phase 2: per (face segment, Gauss point): tangential TENO-D of the line
    // averages to the Gauss point, then merge + flux.  The two lanes of a face
    // segment split the work: lane gpi reconstructs side gpi (0: left, 1:
    // right) at both Gauss points, keeps its own point and hands the other
    // point's values to its partner; after the flux they average (weights 1/2).
    const T tdt = s_scal[0];
    const T iht = s_scal[3];
    const T gA = T(-0.28867513459481288), gB = T(0.28867513459481288);  // -+1/(2 sqrt 3)
#pragma unroll 1
    for (int task = tid; task < 2 * NP; task += NT) {
        const int pair = task >> 1, gpi = task & 1;
        const int r = pair / NF, f = pair % NF;
        // faces n0+f <= nn on rows t0+r < nt exist; the rest of the tile is padding
        const bool valid = (n0 + f <= a.nn) && (t0 + r < a.nt);
        Side<T> L, R;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            // line averages of the side's value (W) and normal slope (Wn) at
            // the two Gauss points: value and tangential derivative of W,
            // value of Wn
            T wa, wda, wb, wdb, na, nb;
            if constexpr (sizeof(T) == 4 && RB <= 1) {
                // both streams as one packed pair (x: W, y: Wn)
                f2 q[5];
#pragma unroll
                for (int s = 0; s < 5; ++s) q[s] = f2(sm.rec[2 * gpi][v][r + s][f], sm.rec[2 * gpi + 1][v][r + s][f]);
                f2 va, da, vb, db;
                packed_gauss<RB>(q, tnt, gA, gB, va, da, vb, db);
                wa = va.x(), wda = da.x(), wb = vb.x(), wdb = db.x(), na = va.y(), nb = vb.y();
            } else {
                T q[5];
                TenoSel<T> S;
                T dn;
#pragma unroll
                for (int s = 0; s < 5; ++s) q[s] = sm.rec[2 * gpi][v][r + s][f];
                rec_select<RB>(q, tnt, S);
                rec_gauss_pm<RB>(S, gB, wa, wda, wb, wdb);  // gA = -gB
#pragma unroll
                for (int s = 0; s < 5; ++s) q[s] = sm.rec[2 * gpi + 1][v][r + s][f];
                rec_select<RB>(q, tnt, S);
                rec_gauss_pm<RB>(S, gB, na, dn, nb, dn);
            }
            // own side at own point; the partner's point goes to the partner
            T own = gpi ? wb : wa, got = __shfl_xor_sync(0xffffffffu, gpi ? wa : wb, 1);
            L.W[v] = gpi ? got : own;
            R.W[v] = gpi ? own : got;
            own = (gpi ? wdb : wda) * iht;
            got = __shfl_xor_sync(0xffffffffu, (gpi ? wda : wdb) * iht, 1);
            L.Wt[v] = gpi ? got : own;
            R.Wt[v] = gpi ? own : got;
            own = gpi ? nb : na;
            got = __shfl_xor_sync(0xffffffffu, gpi ? na : nb, 1);
            L.Wn[v] = gpi ? got : own;
            R.Wn[v] = gpi ? own : got;
        }
        T F[4] = {T(0), T(0), T(0), T(0)}, dF[4] = {T(0), T(0), T(0), T(0)};
        if (valid) {
            if (!physical<T, 2>(L.W, fp.gm1)) {
#pragma unroll
                for (int v = 0; v < 4; ++v) { L.W[v] = sm.w[v][r + 2][f + 2]; L.Wn[v] = L.Wt[v] = T(0); }
                ++nfb;
                if (!physical<T, 2>(L.W, fp.gm1)) err |= 2u;
            }
            if (!physical<T, 2>(R.W, fp.gm1)) {
#pragma unroll
                for (int v = 0; v < 4; ++v) { R.W[v] = sm.w[v][r + 2][f + 3]; R.Wn[v] = R.Wt[v] = T(0); }
                ++nfb;
                if (!physical<T, 2>(R.W, fp.gm1)) err |= 2u;
            }
            if constexpr (CONV) {
                // Step 4: the equilibrium state and slopes at this lane's Gauss
                // point, linear (quartic) reconstructions of the rows' merges
                T w0g[4], w0t[4], w0n[4];
                const T gme = gpi ? gB : gA;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    T q[5], dd;
#pragma unroll
                    for (int s = 0; s < 5; ++s) q[s] = sm.w0[0][v][r + s][f];
                    quartic_gauss(q, gme, w0g[v], dd);
                    w0t[v] = dd * iht;
#pragma unroll
                    for (int s = 0; s < 5; ++s) q[s] = sm.w0[1][v][r + s][f];
                    quartic_gauss(q, gme, w0n[v], dd);
                }
                // a non-physical linear state (the quartic across a
                // discontinuity) falls back to the kinetic merge at the point
                if (physical<T, 2>(w0g, fp.gm1)) {
                    point_flux<T, 2, NONEQ, PRFIX>(L, R, fp, F, dF, w0n, w0g, w0t);
                } else {
                    ++nfb;
                    point_flux<T, 2, NONEQ, PRFIX>(L, R, fp, F, dF);
                }
            } else {
                point_flux<T, 2, NONEQ, PRFIX>(L, R, fp, F, dF);
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            F[v] = T(0.5) * (F[v] + __shfl_xor_sync(0xffffffffu, F[v], 1));
            dF[v] = T(0.5) * (dF[v] + __shfl_xor_sync(0xffffffffu, dF[v], 1));
        }
        if (gpi == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T g0, g1;
                stage_comb<T>(a.stage, F[v], dF[v], tdt, g0, g1);
                sF[sfi(v, r, f)] = g0;
                if (a.stage == 1) sF[sfi(4 + v, r, f)] = g1;
            }
        }
    }
    __syncthreads();

    // phase 3: flux divergence; the y sweep updates the float64 state
    T sig = T(0);
    const T cn = s_scal[1];
    if (tid < TN * TT) {
        // x faces: the normal (x) index fastest; y faces: the tangential (x) index
        const int r = fy ? tid % TT : tid / TN, c = fy ? tid / TT : tid % TN;
        const int in = n0 + c, it = t0 + r;
        if (in < a.nn && it < a.nt) {
            const int o = org + in * sn + it * st;
            T* inc0 = static_cast<T*>(a.inc0);
            T* inc1 = static_cast<T*>(a.inc1);
            double wn[4];
            T wf[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const long long go = (v == 0 ? 0 : (v == 1 ? pv1 : (v == 2 ? pv2 : pv3))) + o;
                const T d0 = cn * (sF[sfi(v, r, c + 1)] - sF[sfi(v, r, c)]);
                const T d1 = (a.stage == 1)
                           ? cn * (sF[sfi(4 + v, r, c + 1)] - sF[sfi(4 + v, r, c)])
                           : T(0);
                if (a.pass == 0) {
                    inc0[go] = d0;
                    if (a.stage == 1) inc1[go] = d1;
                } else if constexpr (sizeof(T) == 4) {
                    if (a.stage == 1) {
                        a.out0f[go] = a.basef[go] - (inc0[go] + d0);
                        inc1[go] = inc1[go] + d1;
                    } else {
                        const double res = a.base[go] - (double)(inc1[go] + inc0[go] + d0);
                        a.out0[go] = res;
                        wf[v] = (float)res;  // local order; the CFL rate only needs |U|
                        a.out0f[go] = wf[v];
                    }
                } else if (a.stage == 1) {
                    const double w = a.base[go];
                    a.out0[go] = w - (double)(inc0[go] + d0);
                    a.out1[go] = w - (double)(inc1[go] + d1);
                } else {
                    const double res = a.base[go] - (double)(inc0[go] + d0);
                    a.out0[go] = res;
                    wn[v] = res;  // local order; the CFL rate only needs |U|
                }
            }
            if (a.with_sigma) {
                if constexpr (sizeof(T) == 4) sig = cell_sigma<T, T>(wf, 2, s_scal[4], s_scal[5], s_scal[6], err);
                else sig = cell_sigma<T>(wn, 2, s_scal[4], s_scal[5], s_scal[6], err);
            }
        }
    }
    block_commit<NT, T>(sig, a.with_sigma != 0, err, nfb, ds);
}

}  // namespace gks
