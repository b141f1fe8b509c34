// gks_flips.cu -- gks_selection_flips: the TENO-D stencil selections
// (Eqs. 4.7, 4.12 of Sec. 4.2) that the float32 path's arithmetic makes
// differently from the float64 path's on the same state.
//
// TENO-D chooses between the large stencil and the sub-stencils by
// thresholds on ratios of smoothness indicators, so the float32 path, whose
// reconstruction runs on the state rounded to float32 and in float32
// arithmetic, can take another (equally valid) choice than the float64 path
// where a ratio lies within rounding of a cut-off.  This diagnostic counts
// such choices on one state.  Both precisions run the kernels' own code: the
// float64 selection of the float64 kernels and the float32 selection of the
// float32 kernels (packed variable pairs in the normal direction, packed
// value / slope streams in the tangential one, 1-D (rho, rho u) packed), and
// this unit is compiled with the float32 kernels' arithmetic flags, so every
// choice is the one the kernels make.
#include <cuda_runtime.h>

#include "../../include/gks.h"
#include "gks_ctx.h"
#include "gks_pair.cuh"

namespace {

using namespace gks;

// A stencil whose data vary by less than 2^-16 of their magnitude (about 100
// float32 ulps) is below float32 resolution: where float32 rounding makes
// it constant any choice reproduces the constant, and where the float64 data
// vary at round-off level the float64 choice follows that noise.  Flips on
// such stencils change no value beyond rounding; they are counted apart.
// scale: the magnitude of the quantity the stencil's data resolve (cell and
// line averages: their own largest magnitude; line-averaged normal slopes:
// the largest magnitude of the values they are the slope of, over dx).
__device__ double magnitude(const double* q)
{
    double mx = fabs(q[0]);
#pragma unroll
    for (int s = 1; s < 5; ++s) mx = fmax(mx, fabs(q[s]));
    return mx;
}
__device__ bool resolved(const double* q, double scale)
{
    double lo = q[0], hi = q[0];
#pragma unroll
    for (int s = 1; s < 5; ++s) {
        lo = fmin(lo, q[s]);
        hi = fmax(hi, q[s]);
    }
    return hi - lo > ldexp(scale, -16);
}

// the selection as 4 bits: bit 0 large stencil, bits 1-3 kept sub-stencils
template <typename T>
__device__ unsigned sel_code(const TenoSel<T>& S)
{
    if (S.large) return 1u;
    return (S.w[0] > T(0) ? 2u : 0u) | (S.w[1] > T(0) ? 4u : 0u) | (S.w[2] > T(0) ? 8u : 0u);
}

// counters: normal flips, normal selections, tangential flips, tangential
// selections, unresolved flips (both kinds)
constexpr int NCOUNT = 5;

__device__ void add_counts(unsigned long long* out, unsigned (&c)[NCOUNT])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NCOUNT; ++k) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NCOUNT; ++k)
            if (c[k]) atomicAdd(out + k, (unsigned long long)c[k]);
}

// one compared selection: a flip on a resolved stencil counts in slot k,
// on an unresolved one in slot 4
__device__ void tally(unsigned (&c)[NCOUNT], int k, unsigned code64, unsigned code32, const double* q,
                      double scale)
{
    c[k + 1] += 1;
    if (code64 != code32) c[resolved(q, scale) ? k : 4] += 1;
}

// 1-D: per cell, the normal selection of (rho, rho u, E)
__global__ void k_flips1d(GridDev g, const double* __restrict__ W, TenoT<double> pd, TenoT<float> pf,
                          unsigned long long* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // interior cell
    unsigned cnt[NCOUNT] = {0, 0, 0, 0, 0};
    if (i < g.nx) {
        const int pl = (int)g.plane;
        double q[3][5];
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int s = 0; s < 5; ++s) q[v][s] = W[v * pl + NG + i - 2 + s];
        unsigned cd[3], cf[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            TenoSel<double> S;
            teno_select(q[v], pd, S);
            cd[v] = sel_code(S);
        }
        f2 qq[5];
        float qe[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            qq[s] = f2((float)q[0][s], (float)q[1][s]);
            qe[s] = (float)q[2][s];
        }
        TenoSel2 S2;
        teno_select_x2(qq, pf, S2);
        cf[0] = sel_code_x(S2);
        cf[1] = sel_code_y(S2);
        TenoSel<float> S;
        teno_select(qe, pf, S);
        cf[2] = sel_code(S);
#pragma unroll
        for (int v = 0; v < 3; ++v) tally(cnt, 0, cd[v], cf[v], q[v], magnitude(q[v]));
    }
    add_counts(out, cnt);
}

// 2-D, one direction: per (face, row) of the interior.  Cell f (f < nn):
// the normal selection of its four variables; face f (between cells f-1 and
// f): the tangential selections of both sides' value and normal-slope line
// averages over rows t-2 .. t+2, each precision on its own line averages.
__global__ void k_flips2d(GridDev g, const double* __restrict__ W, int dirn, TenoT<double> nd, TenoT<float> nf,
                          TenoT<double> td, TenoT<float> tf, double ihn, unsigned long long* out)
{
    const int nn = dirn ? g.ny : g.nx, nt = dirn ? g.nx : g.ny;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned cnt[NCOUNT] = {0, 0, 0, 0, 0};
    if (idx < (long long)(nn + 1) * nt) {
        const int f = (int)(idx % (nn + 1)), t = (int)(idx / (nn + 1));
        // variable v of the local frame (normal momentum first) at normal
        // index n, tangential index tt (interior coordinates; ghosts at -3..)
        auto at = [&](int v, int n, int tt) -> double {
            const int gv = (dirn && (v == 1 || v == 2)) ? 3 - v : v;
            const int i = dirn ? tt : n, j = dirn ? n : tt;
            return W[(long long)gv * g.plane + (long long)(j + NG) * g.pitch + (i + NG)];
        };
        const float ihf = (float)ihn;
#pragma unroll 1
        for (int vp = 0; vp < 4; vp += 2) {  // the float32 sweep's variable pairs (0, 1), (2, 3)
            if (f < nn) {
                double q[2][5];
                f2 qq[5];
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    q[0][s] = at(vp, f - 2 + s, t);
                    q[1][s] = at(vp + 1, f - 2 + s, t);
                    qq[s] = f2((float)q[0][s], (float)q[1][s]);
                }
                TenoSel2 S2;
                teno_select_x2(qq, nf, S2);
                const unsigned cf0 = sel_code_x(S2), cf1 = sel_code_y(S2);
                TenoSel<double> S;
                teno_select(q[0], nd, S);
                tally(cnt, 0, sel_code(S), cf0, q[0], magnitude(q[0]));
                teno_select(q[1], nd, S);
                tally(cnt, 0, sel_code(S), cf1, q[1], magnitude(q[1]));
            }
            // line averages of the two sides (side 0: cell f-1 at +1/2,
            // side 1: cell f at -1/2), rows t-2 .. t+2, per precision
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                double lv[2][5], ls[2][5];
                f2 fv[5], fs[5];  // lanes: variables vp, vp + 1
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const int c = f - 1 + side, row = t - 2 + r;
                    double q[2][5];
                    f2 qq[5];
#pragma unroll
                    for (int s = 0; s < 5; ++s) {
                        q[0][s] = at(vp, c - 2 + s, row);
                        q[1][s] = at(vp + 1, c - 2 + s, row);
                        qq[s] = f2((float)q[0][s], (float)q[1][s]);
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        TenoSel<double> S;
                        teno_select(q[k], nd, S);
                        double a, b, cc, d;
                        teno_faces(q[k], S, a, b, cc, d);
                        lv[k][r] = side ? cc : a;
                        ls[k][r] = (side ? d : b) * ihn;
                    }
                    TenoSel2 S2;
                    teno_select_x2(qq, nf, S2);
                    f2 a, b, cc, d;
                    teno_faces_x2(S2, a, b, cc, d);
                    fv[r] = side ? cc : a;
                    fs[r] = (side ? d : b) * f2(ihf);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    // float32: one packed selection of the (value, slope) streams
                    f2 qq[5];
#pragma unroll
                    for (int r = 0; r < 5; ++r) qq[r] = k ? f2(fv[r].y(), fs[r].y()) : f2(fv[r].x(), fs[r].x());
                    TenoSel2 S2;
                    teno_select_x2(qq, tf, S2);
                    TenoSel<double> S;
                    teno_select(lv[k], td, S);
                    const double mv = magnitude(lv[k]);
                    tally(cnt, 2, sel_code(S), sel_code_x(S2), lv[k], mv);
                    teno_select(ls[k], td, S);
                    tally(cnt, 2, sel_code(S), sel_code_y(S2), ls[k], mv * ihn);
                }
            }
        }
    }
    add_counts(out, cnt);
}

}  // namespace

extern "C" gks_status gks_selection_flips(gks_ctx* c, gks_flip_count* out)
{
    if (!c || !out) return GKS_EINVAL;
    if (c->sch.recon != GKS_RECON_TENO_D || c->sch.charvars)
        return rt::fail(c, GKS_EUNSUPPORTED, "selection flips are counted for component-wise TENO-D");
    const TenoParams tn = rt::teno_params(c, false), tt = rt::teno_params(c, true);
    unsigned long long* d = nullptr;
    unsigned long long h[NCOUNT] = {0, 0, 0, 0, 0};
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) return rt::fail(c, GKS_ENOMEM, "cudaMalloc of 40 bytes failed");
    gks_status st = GKS_OK;
    do {
        if (cudaMemsetAsync(d, 0, sizeof h, c->stream) != cudaSuccess) { st = GKS_ECUDA; break; }
        if ((st = rt::fill_ghosts_f64(c, c->W, c->stream)) != GKS_OK) break;
        if (c->desc.dim == 1) {
            k_flips1d<<<(c->desc.nx + 255) / 256, 256, 0, c->stream>>>(c->g, c->W, teno_t<double>(tn),
                                                                     teno_t<float>(tn), d);
            ++c->launches;
        } else {
            for (int dir = 0; dir < 2; ++dir) {
                const int nn = dir ? c->desc.ny : c->desc.nx, nt = dir ? c->desc.nx : c->desc.ny;
                const long long n = (long long)(nn + 1) * nt;
                const double ihn = 1.0 / (dir ? c->g.dy : c->g.dx);
                k_flips2d<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                    c->g, c->W, dir, teno_t<double>(tn), teno_t<float>(tn), teno_t<double>(tt), teno_t<float>(tt),
                    ihn, d);
                ++c->launches;
            }
        }
        if (cudaGetLastError() != cudaSuccess) { st = GKS_ECUDA; break; }
        if (cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            st = GKS_ECUDA;
    } while (0);
    cudaFree(d);
    if (st == GKS_ECUDA) return rt::fail(c, st, "selection flip count failed");
    if (st) return st;
    out->normal_flips = (long long)h[0];
    out->normal_selections = (long long)h[1];
    out->tangential_flips = (long long)h[2];
    out->tangential_selections = (long long)h[3];
    out->unresolved_flips = (long long)h[4];
    return GKS_OK;
}
