// gks_aux.cuh -- small kernels of the step loop: ghost-layer filling, the
// CFL-rate reduction of a state, and the device-side time commit.  Included
// by the runtime translation unit only.
#pragma once

#include "gks_kernels.cuh"

namespace gks {

// ------------------------------------------------------------------ ghosts
// One thread per ghost cell.  x ghosts of interior rows use the x rule; rows
// of y ghosts use the y rule to pick an interior row, then the x rule for
// x-ghost columns (the same values as filling x first, then y over the full
// ghosted width).
// State-setting rules (inflow, wall after x0, moving shock) write their state;
// toff: the array's time is t + toff dt (0 for W, 1/2 for W*).
template <typename E>
__global__ void k_fill_ghosts(GridDev g, E* __restrict__ W, const DevState* ds, double toff)
{
    if (ds && ds->done) return;
    const int gx = g.nx + 2 * NG;
    const int nv = g.dim + 2;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int i, j;
    if (g.dim == 1) {
        if (idx >= 2 * NG) return;
        j = 0;
        i = idx < NG ? idx : g.nx + idx;  // 0,1,2 and nx+3.. nx+5
    } else {
        const int band = 2 * NG * gx;
        if (idx < band) {
            j = idx / gx;
            i = idx % gx;
            if (j >= NG) j = g.ny + j;  // rows ny+3 .. ny+5
        } else {
            idx -= band;
            if (idx >= 2 * NG * g.ny) return;
            j = NG + idx / (2 * NG);
            int k = idx % (2 * NG);
            i = k < NG ? k : g.nx + k;
        }
    }
    bool fxn = false, fxa = false, fyn = false, fya = false;
    const double t = ds ? ds->t + toff * ds->dt : 0.0;
    const double xc = g.ox + (i - NG + 0.5) * g.dx, yc = g.oy + (j - NG + 0.5) * g.dy;
    int sj = j;
    if (g.dim == 2 && (j < NG || j >= NG + g.ny)) {
        const int by = g.bc[2 + (j >= NG + g.ny)];
        const double* st = ghost_state(g, by, xc, yc, t);
        if (st) {
            for (int v = 0; v < nv; ++v)
                W[(long long)v * g.plane + (long long)j * g.pitch + i] = (E)st[v == nv - 1 ? 3 : v];
            return;
        }
        sj = ghost_src(by, g.ny, j, fyn, fya);
    }
    int si = i;
    const double* sx = nullptr;  // x ghost column under an inflow rule
    if (i < NG || i >= NG + g.nx) {
        const int bx = g.bc[(i >= NG + g.nx)];
        sx = ghost_state(g, bx, xc, yc, t);
        if (!sx) si = ghost_src(bx, g.nx, i, fxn, fxa);
    }
    for (int v = 0; v < nv; ++v) {
        E val = sx ? (E)sx[v == nv - 1 ? 3 : v] : W[(long long)v * g.plane + (long long)sj * g.pitch + si];
        // x rule flips the x velocity (v=1) for symmetry, both for no-slip
        const int vx = 1, vy = (g.dim == 2) ? 2 : -1;
        bool neg = false;
        if (v == vx && (fxn || fxa)) neg = !neg;
        if (v == vy && fxa) neg = !neg;
        if (v == vy && (fyn || fya)) neg = !neg;
        if (v == vx && fya) neg = !neg;
        W[(long long)v * g.plane + (long long)j * g.pitch + i] = neg ? -val : val;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sigma(GridDev g, const double* __restrict__ W, DevState* ds)
{
    T s = T(0);
    unsigned int err = 0;
    const int nv = g.dim + 2;
    const double h = (g.dim == 2) ? fmin(g.dx, g.dy) : g.dx;
    const long long ncell = (long long)g.nx * (g.dim == 2 ? g.ny : 1);
    for (long long c = blockIdx.x * 256ll + threadIdx.x; c < ncell; c += 256ll * gridDim.x) {
        const int i = (int)(c % g.nx), j = (int)(c / g.nx);
        const long long off = (long long)(g.dim == 2 ? j + NG : 0) * g.pitch + i + NG;
        double w[4];
        for (int v = 0; v < nv; ++v) w[v] = W[(long long)v * g.plane + off];
        s = fmax(s, cell_sigma<T>(w, g.dim, (T)g.gamma, (T)g.mu, (T)h, err));
    }
    block_commit<256, T>(s, true, err, 0u, ds);
}

// float32 shadow of a float64 array (same layout)
__global__ void k_to_float(const double* __restrict__ W, float* __restrict__ Wf, long long n)
{
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += 256ll * gridDim.x) Wf[i] = (float)W[i];
}

// float64 views of the float32 path's stage buffers (gks_get_buffer):
// W* from its float32 form, the accumulator from W and its increment
__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, long long n)
{
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += 256ll * gridDim.x) dst[i] = (double)src[i];
}
__global__ void k_accumulator(const double* __restrict__ W, const float* __restrict__ inc, double* __restrict__ A,
                              long long n)
{
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += 256ll * gridDim.x) A[i] = W[i] - (double)inc[i];
}

// After the last kernel of a step: advance t by dt, pick the next dt
// (CFL from the reduced sigma, clipped to t_end), detect completion.
// init = 1: only pick dt from sigma (before the first step).
__global__ void k_commit(DevState* ds, int init)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (ds->done) return;
    if (!init) {
        ds->t += ds->dt;
        ds->steps += 1;
    }
    const double sig = __longlong_as_double((long long)ds->sigma);
    ds->sigma = 0ull;
    double dt = ds->fixed_dt ? ds->dt : ds->cfl / sig;
    if (ds->t + dt > ds->t_end) dt = ds->t_end - ds->t;
    ds->dt = dt;
    if (!(ds->t < ds->t_end) || (ds->max_steps > 0 && ds->steps >= ds->max_steps)) ds->done = 1u;
}

}  // namespace gks
