// gks_ensemble.cu -- a batch of independent 1-D problems advanced in ONE
// persistent launch (include/gks.h, gks_batch_*).
//
// Every block pops the next problem from an atomic queue (problems ordered by
// decreasing estimated cost n^2 * s_max, longest-processing-time first),
// advances it to t_end with its own CFL steps, writes it back and pops the
// next.  The whole problem stays with one block, so the stage barrier is a
// __syncthreads and blocks never wait on each other.  A stage sweeps the
// problem in chunks of NT-6 cells with the same per-cell and per-face
// arithmetic as the single-grid 1-D kernel (zero-gradient ends by clamped
// indices).  The launch (queue reset + kernel) is captured once as a CUDA
// graph per (t_end, max_steps, launch shape); a small autotuner times the
// candidate launch shapes on a short horizon and caches the winner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <iomanip>
#include <new>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/gks.h"
#include "gks_launch.h"
#include "gks_nvtx.h"

using namespace gks;

namespace {

struct BatchDev {
    double* W;                    // packed [3][total] state
    float* Wf;                    // float32 path: float32 shadow of W, written by the
                                  // kernel (converted when a block takes a problem,
                                  // kept with every update); float64 path: unused
    void *Ws, *A;                 // W* and the accumulator: float64 arrays on the
                                  // float64 path; on the float32 path W* in float32
                                  // and the accumulator increment in float32
    long long total;              // cells of all problems
    const long long* off;         // first cell of each problem
    const int* n;                 // cells per problem
    const double* dx;             // cell size per problem
    const int* order;             // LPT order of problem indices
    double* t;                    // per-problem time
    long long* steps;             // per-problem step count
    unsigned int* err;            // per-problem error word
    unsigned long long* fallbacks;
    int* queue;
    int count;
    double t_end, cfl;
    long long max_steps;          // per problem and call; <= 0: none
    double gamma, mu;
};

template <typename T, int NT>
__device__ __forceinline__ T block_max(T v, T* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T r = red[0];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) r = fmax(r, red[k]);
    return r;
}

__device__ __forceinline__ unsigned int block_or(unsigned int v, unsigned int* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned int r = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r |= red[k];
    return r;
}

// A chunk holds TN = NT - 6 cells, so that its TN + 6 stencil cells, TN + 2
// reconstructed cells and TN + 1 faces each take one pass of the block.
template <typename T, int NT> struct ChunkSmem {
    T q[3][NT];                 // cells c0-3 .. c0+TN+2
    T L[3][2][NT], R[3][2][NT]; // face states [var][value, slope][face]
    T G[2][3][NT];              // face fluxes for the update
};

// The stage's scalars: dt and dt/dx in float64 (the float64 updates) and in
// the arithmetic type, 1/dx in the arithmetic type; formed once per step by
// one thread (a float64 operation in a float32 kernel runs on the slow
// float64 pipe)
template <typename T> struct StepScalars {
    double dt, cx;
    T tdt, cxt, ih;
};

// One stage over cells [c0, c0+TN) of a problem: load (clamped indices =
// zero-gradient ghosts), TENO-D per cell, flux per face, update.  The update
// follows the single-grid 1-D kernel: float64 W* and accumulator on the
// float64 path; on the float32 path W* and the accumulator increment in
// float32 and one float64 update of W per value and step, its float32
// shadow Wf (the stage-1 input) written beside it.
template <typename T, int NT, bool NONEQ, bool PRFIX>
__device__ void stage_chunk(ChunkSmem<T, NT>& sm, double* W, float* Wf, T* Ws, T* A, long long vstride, int n,
                            int c0, int stage, const StepScalars<T>& sc, const FluxParams<T>& fp, const TenoT<T>& tn,
                            T& sig, unsigned int& err, unsigned int& nfb, T gamma, T mu, T hcell)
{
    constexpr int TN = NT - 6;
    const int tid = threadIdx.x;
    const int slot[3] = {0, 1, 3};
    __syncthreads();  // shared memory of the previous chunk is free
    // each variable's array through its own base pointer; cell offsets in 32 bits
    double* Wv[3] = {W, W + vstride, W + 2 * vstride};
    float* Wfv[3] = {Wf, Wf + vstride, Wf + 2 * vstride};
    T* Wsv[3] = {Ws, Ws + vstride, Ws + 2 * vstride};
    T* Av[3] = {A, A + vstride, A + 2 * vstride};
    for (int k = tid; k < 3 * (TN + 6); k += NT) {
        const int v = k / (TN + 6), c = k % (TN + 6);
        int i = c0 - 3 + c;
        i = i < 0 ? 0 : (i >= n ? n - 1 : i);
        if (stage == 2) sm.q[v][c] = (v == 0 ? Ws : (v == 1 ? Wsv[1] : Wsv[2]))[i];
        else if constexpr (sizeof(T) == 4) sm.q[v][c] = (v == 0 ? Wf : (v == 1 ? Wfv[1] : Wfv[2]))[i];
        else sm.q[v][c] = (v == 0 ? W : (v == 1 ? Wv[1] : Wv[2]))[i];
    }
    __syncthreads();
    const T ih = sc.ih;
    for (int c = tid; c < TN + 2; c += NT) {  // cell c0-1+c
        T q[3][5], vp[3], dp[3], vm[3], dm[3];
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int s = 0; s < 5; ++s) q[v][s] = sm.q[v][c + s];
        recon_cell3<0>(q, tn, vp, dp, vm, dm);  // the single-grid 1-D kernel's arithmetic
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            if (c <= TN) { sm.L[v][0][c] = vp[v]; sm.L[v][1][c] = dp[v] * ih; }
            if (c >= 1) { sm.R[v][0][c - 1] = vm[v]; sm.R[v][1][c - 1] = dm[v] * ih; }
        }
    }
    __syncthreads();
    const T tdt = sc.tdt;
    for (int f = tid; f <= TN; f += NT) {  // face between cells c0+f-1 and c0+f
        if (c0 + f > n) continue;
        Side<T> L, R;
#pragma unroll
        for (int k = 0; k < 4; ++k) L.W[k] = L.Wn[k] = L.Wt[k] = R.W[k] = R.Wn[k] = R.Wt[k] = T(0);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            L.W[slot[v]] = sm.L[v][0][f];
            L.Wn[slot[v]] = sm.L[v][1][f];
            R.W[slot[v]] = sm.R[v][0][f];
            R.Wn[slot[v]] = sm.R[v][1][f];
        }
        if (!physical<T, 1>(L.W, fp.gm1)) {
#pragma unroll
            for (int v = 0; v < 3; ++v) { L.W[slot[v]] = sm.q[v][f + 2]; L.Wn[slot[v]] = T(0); }
            ++nfb;
            if (!physical<T, 1>(L.W, fp.gm1)) err |= 2u;
        }
        if (!physical<T, 1>(R.W, fp.gm1)) {
#pragma unroll
            for (int v = 0; v < 3; ++v) { R.W[slot[v]] = sm.q[v][f + 3]; R.Wn[slot[v]] = T(0); }
            ++nfb;
            if (!physical<T, 1>(R.W, fp.gm1)) err |= 2u;
        }
        T F[4], dF[4];
        point_flux<T, 1, NONEQ, PRFIX>(L, R, fp, F, dF);
#pragma unroll
        for (int v = 0; v < 3; ++v) stage_comb<T>(stage, F[slot[v]], dF[slot[v]], tdt, sm.G[0][v][f], sm.G[1][v][f]);
    }
    __syncthreads();
    const double cx = sc.cx;
    const T cxt = sc.cxt;
    for (int c = tid; c < TN; c += NT) {
        const int i = c0 + c;
        if (i >= n) continue;
        if constexpr (sizeof(T) == 4) {
            if (stage == 1) {
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    Wsv[v][i] = wstar32(sm.q[v][c + 3], cxt, sm.G[0][v][c + 1] - sm.G[0][v][c]);
                    Av[v][i] = cxt * (sm.G[1][v][c + 1] - sm.G[1][v][c]);
                }
            } else {
                T w[3];
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const double r = wnew32(Wv[v][i], Av[v][i], cxt, sm.G[0][v][c + 1] - sm.G[0][v][c]);
                    Wv[v][i] = r;
                    w[v] = (T)r;
                    Wfv[v][i] = w[v];
                }
                sig = fmax(sig, cell_sigma<T, T>(w, 1, gamma, mu, hcell, err));
            }
        } else if (stage == 1) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const double w = Wv[v][i];
                Wsv[v][i] = upd64(w, cx, (double)(sm.G[0][v][c + 1] - sm.G[0][v][c]));
                Av[v][i] = upd64(w, cx, (double)(sm.G[1][v][c + 1] - sm.G[1][v][c]));
            }
        } else {
            double w[3];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                w[v] = upd64(Av[v][i], cx, (double)(sm.G[0][v][c + 1] - sm.G[0][v][c]));
                Wv[v][i] = w[v];
            }
            sig = fmax(sig, cell_sigma<T>(w, 1, gamma, mu, hcell, err));
        }
    }
}

template <typename T, int NT, bool NONEQ, bool PRFIX>
__global__ void __launch_bounds__(NT) k_batch(BatchDev b, FluxParams<T> fp, TenoT<T> tn)
{
    __shared__ ChunkSmem<T, NT> sm;
    __shared__ T red[NT / 32];
    __shared__ unsigned int redu[NT / 32];
    __shared__ int s_prob, s_go;
    __shared__ StepScalars<T> s_sc;
    constexpr int TN = NT - 6;
    const int tid = threadIdx.x;
    const T gamma = (T)b.gamma, mu = (T)b.mu;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_prob = atomicAdd(b.queue, 1);
        __syncthreads();
        const int qi = s_prob;
        if (qi >= b.count) return;
        const int p = b.order[qi];
        const int n = b.n[p];
        const long long off = b.off[p];
        const double dx = b.dx[p], idx = 1.0 / dx;
        const T hcell = (T)dx;
        double* W = b.W + off;
        float* Wf = b.Wf ? b.Wf + off : nullptr;
        T* Ws = static_cast<T*>(b.Ws) + off;
        T* A = static_cast<T*>(b.A) + off;
        double t = b.t[p];          // thread 0 keeps the time and step count
        long long steps = 0;
        unsigned int err = 0, nfb = 0;
        // CFL rate of the starting state (float32 path: from the state rounded
        // to float32, which becomes the shadow the stage-1 loads read)
        T sig = T(0);
        for (int i = tid; i < n; i += NT) {
            const T w0[3] = {(T)W[i], (T)W[b.total + i], (T)W[2 * b.total + i]};
            if constexpr (sizeof(T) == 4) {
                Wf[i] = w0[0];
                Wf[b.total + i] = w0[1];
                Wf[2 * b.total + i] = w0[2];
            }
            sig = fmax(sig, cell_sigma<T, T>(w0, 1, gamma, mu, hcell, err));
        }
        sig = block_max<T, NT>(sig, red);
        err = block_or(err, redu);
        for (;;) {
            if (tid == 0) {
                const int go = t < b.t_end && (b.max_steps <= 0 || steps < b.max_steps) && !err;
                if (go) {
                    double dt = b.cfl / (double)sig;
                    if (t + dt > b.t_end) dt = b.t_end - t;
                    s_sc.dt = dt;
                    s_sc.cx = dt * idx;
                    s_sc.tdt = (T)dt;
                    s_sc.cxt = (T)(dt * idx);
                    s_sc.ih = (T)idx;
                }
                s_go = go;
            }
            __syncthreads();
            if (!s_go) break;
            const StepScalars<T>& sc = s_sc;  // read where used: no registers held across the chunks
            FluxParams<T> f = fp;
            f.dt = sc.tdt;
            for (int c0 = 0; c0 < n; c0 += TN)
                stage_chunk<T, NT, NONEQ, PRFIX>(sm, W, Wf, Ws, A, b.total, n, c0, 1, sc, f, tn, sig, err, nfb, gamma,
                                                 mu, hcell);
            T s2 = T(0);
            for (int c0 = 0; c0 < n; c0 += TN)
                stage_chunk<T, NT, NONEQ, PRFIX>(sm, W, Wf, Ws, A, b.total, n, c0, 2, sc, f, tn, s2, err, nfb, gamma,
                                                 mu, hcell);
            sig = block_max<T, NT>(s2, red);
            err = block_or(err, redu);
            if (tid == 0) {
                t += sc.dt;
                ++steps;
            }
        }
        if (nfb) atomicAdd(b.fallbacks, (unsigned long long)nfb);
        if (tid == 0) {
            b.t[p] = t;
            b.steps[p] += steps;
            b.err[p] |= err;
        }
    }
}

// per-problem maximum signal speed of the stored state (for the LPT order)
__global__ void k_batch_speed(BatchDev b, double* speed)
{
    const int p = blockIdx.x;
    const int n = b.n[p];
    const double* W = b.W + b.off[p];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = W[i], U = W[b.total + i] / r, E = W[2 * b.total + i];
        const double pr = (b.gamma - 1.0) * (E - 0.5 * r * U * U);
        const double a = (r > 0.0 && pr > 0.0) ? sqrt(b.gamma * pr / r) : 0.0;
        s = fmax(s, fabs(U) + a);
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) s = fmax(s, red[k]);
        speed[p] = s;
    }
}

// ------------------------------------------------------------------ launch shapes
using KernFn = void (*)(BatchDev, FluxParams<float>, TenoT<float>);
using KernFnD = void (*)(BatchDev, FluxParams<double>, TenoT<double>);

template <typename T>
struct KernTable {
    using Fn = void (*)(BatchDev, FluxParams<T>, TenoT<T>);
    static Fn get(int threads, int variant)
    {
        // variant 0: tau = 0; 1: with non-equilibrium terms; 2: plus Prandtl fix
        if (threads == 128) {
            if (variant == 0) return k_batch<T, 128, false, false>;
            if (variant == 1) return k_batch<T, 128, true, false>;
            return k_batch<T, 128, true, true>;
        }
        if (variant == 0) return k_batch<T, 256, false, false>;
        if (variant == 1) return k_batch<T, 256, true, false>;
        return k_batch<T, 256, true, true>;
    }
};

}  // namespace

struct gks_batch {
    int count = 0, precision = 0;
    long long total = 0;
    std::vector<int> n;
    std::vector<double> len;
    std::vector<long long> off;
    double* W = nullptr;
    float* Wf = nullptr;  // float32 path: float32 shadow of W (maintained by the kernel)
    void *Ws = nullptr, *A = nullptr;
    long long* d_off = nullptr;
    int *d_n = nullptr, *d_order = nullptr, *d_queue = nullptr;
    double *d_dx = nullptr, *d_t = nullptr, *d_speed = nullptr;
    long long* d_steps = nullptr;
    unsigned int* d_err = nullptr;
    unsigned long long* d_fb = nullptr;
    gks_gas gas{1.4, 0.0, 1.0};
    gks_scheme sch{};
    cudaStream_t stream = nullptr, cap = nullptr;
    int threads = 256, blocks_per_sm = 2, sms = 0;
    cudaGraphExec_t graph = nullptr;
    double g_t_end = -1.0;
    long long g_max = -1;
    int g_threads = 0, g_bps = 0;
    unsigned long long g_version = 0, version = 1;
    long long launches = 0;
    std::string err;
};

namespace {

gks_status bfail(gks_batch* b, gks_status s, const char* fmt, ...)
{
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->err = buf;
    }
    return s;
}

#define BCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return bfail(b, GKS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

BatchDev dev_view(gks_batch* b, double t_end, long long max_steps)
{
    BatchDev d;
    d.W = b->W;
    d.Wf = b->Wf;
    d.Ws = b->Ws;
    d.A = b->A;
    d.total = b->total;
    d.off = b->d_off;
    d.n = b->d_n;
    d.dx = b->d_dx;
    d.order = b->d_order;
    d.t = b->d_t;
    d.steps = b->d_steps;
    d.err = b->d_err;
    d.fallbacks = b->d_fb;
    d.queue = b->d_queue;
    d.count = b->count;
    d.t_end = t_end;
    d.cfl = b->sch.cfl;
    d.max_steps = max_steps;
    d.gamma = b->gas.gamma;
    d.mu = b->gas.mu;
    return d;
}

int variant_of(const gks_batch* b)
{
    if (b->sch.tau_mode == GKS_TAU_ZERO) return 0;
    if (b->sch.tau_mode == GKS_TAU_NS && b->gas.Pr != 1.0) return 2;
    return 1;
}

HostFlux host_flux_1d(const gks_batch* b)
{
    HostFlux h;
    h.gamma = b->gas.gamma;
    h.K = (3.0 - b->gas.gamma) / (b->gas.gamma - 1.0);
    h.ntot = h.K + 1.0;
    h.c1 = b->sch.c1;
    h.c2 = b->sch.c2;
    h.mu = b->gas.mu;
    h.prfac = (b->sch.tau_mode == GKS_TAU_NS) ? 1.0 / b->gas.Pr - 1.0 : 0.0;
    h.tau_mode = b->sch.tau_mode;
    h.merge = b->sch.merge;
    return h;
}

gks_status enqueue_batch(gks_batch* b, double t_end, long long max_steps, int threads, int bps, cudaStream_t st)
{
    BCK(cudaMemsetAsync(b->d_queue, 0, sizeof(int), st));
    const BatchDev d = dev_view(b, t_end, max_steps);
    const HostFlux hf = host_flux_1d(b);
    const TenoParams tp{b->sch.eps, b->sch.q, b->sch.ct1, b->sch.ct2};
    const int grid = std::max(1, std::min(b->count, b->sms * bps));
    const int var = variant_of(b);
    if (b->precision == GKS_FP32_FLUX)
        KernTable<float>::get(threads, var)<<<grid, threads, 0, st>>>(d, make_flux_params<float>(hf), teno_t<float>(tp));
    else
        KernTable<double>::get(threads, var)<<<grid, threads, 0, st>>>(d, make_flux_params<double>(hf), teno_t<double>(tp));
    BCK(cudaGetLastError());
    return GKS_OK;
}

gks_status run_batch(gks_batch* b, double t_end, long long max_steps, int threads, int bps)
{
    if (!b->graph || b->g_t_end != t_end || b->g_max != max_steps || b->g_threads != threads || b->g_bps != bps ||
        b->g_version != b->version) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        if (!b->cap) BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        gks_status s = enqueue_batch(b, t_end, max_steps, threads, bps, b->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (s) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        BCK(e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(e);
        b->g_t_end = t_end;
        b->g_max = max_steps;
        b->g_threads = threads;
        b->g_bps = bps;
        b->g_version = b->version;
    }
    BCK(cudaGraphLaunch(b->graph, b->stream));
    b->launches += 1;
    return GKS_OK;
}

// longest-processing-time order from n^2 * (max signal speed)
gks_status order_problems(gks_batch* b)
{
    const BatchDev d = dev_view(b, 0.0, 0);
    k_batch_speed<<<b->count, 128, 0, b->stream>>>(d, b->d_speed);
    BCK(cudaGetLastError());
    std::vector<double> speed(b->count);
    BCK(cudaMemcpyAsync(speed.data(), b->d_speed, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    std::vector<int> order(b->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const double cx = (double)b->n[x] * b->n[x] / b->len[x] * speed[x];
        const double cy = (double)b->n[y] * b->n[y] / b->len[y] * speed[y];
        return cx > cy;
    });
    BCK(cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return GKS_OK;
}

std::string cache_path()
{
    const char* p = getenv("GKS_TUNE_CACHE");
    if (p && *p) return p;
    const char* home = getenv("HOME");
    return std::string(home ? home : ".") + "/.cache/gks_batch_tune.txt";
}

std::string cache_key(const gks_batch* b)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream k;
    k << prop.name << "|sm" << prop.multiProcessorCount << "|p" << b->precision << "|v" << variant_of(b) << "|c"
      << b->count << "|n" << b->total;
    std::string s = k.str();
    for (auto& ch : s)
        if (ch == ' ') ch = '_';
    return s;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

gks_status gks_batch_create(int count, const int* ncells, const double* lengths, int precision, gks_batch** out)
{
    if (!out || count < 1 || !ncells || !lengths) return GKS_EINVAL;
    *out = nullptr;
    if (precision != GKS_FP64 && precision != GKS_FP32_FLUX) return GKS_EINVAL;
    gks_batch* b = new (std::nothrow) gks_batch();
    if (!b) return GKS_ENOMEM;
    b->count = count;
    b->precision = precision;
    b->n.assign(ncells, ncells + count);
    b->len.assign(lengths, lengths + count);
    b->off.resize(count);
    long long tot = 0;
    for (int k = 0; k < count; ++k) {
        if (b->n[k] < 3 || !(b->len[k] > 0.0)) {
            delete b;
            return GKS_EINVAL;
        }
        b->off[k] = tot;
        tot += b->n[k];
    }
    b->total = tot;
    b->sch = {0.5, 0.01, 1.0, 1e-7, 1e-5, 1e-7, 1e-5, 1e-40, 7, GKS_TAU_EULER, 1, GKS_RECON_TENO_D, 0.85, 0.85, 1e-8};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t arr = sizeof(double) * 3 * (size_t)tot;
    const size_t warr = (precision == GKS_FP32_FLUX ? sizeof(float) : sizeof(double)) * 3 * (size_t)tot;
    std::vector<double> dx(count);
    for (int k = 0; k < count; ++k) dx[k] = b->len[k] / b->n[k];
    bool ok = cudaMalloc(&b->W, arr) == cudaSuccess && cudaMalloc(&b->Ws, warr) == cudaSuccess &&
              (precision != GKS_FP32_FLUX || cudaMalloc(&b->Wf, warr) == cudaSuccess) &&
              cudaMalloc(&b->A, warr) == cudaSuccess && cudaMalloc(&b->d_off, sizeof(long long) * count) == cudaSuccess &&
              cudaMalloc(&b->d_n, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_order, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_queue, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_dx, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_t, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_speed, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_steps, sizeof(long long) * count) == cudaSuccess &&
              cudaMalloc(&b->d_err, sizeof(unsigned int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_fb, sizeof(unsigned long long)) == cudaSuccess;
    if (ok) {
        std::vector<int> order(count);
        std::iota(order.begin(), order.end(), 0);
        ok = cudaMemcpy(b->d_off, b->off.data(), sizeof(long long) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_n, b->n.data(), sizeof(int) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_dx, dx.data(), sizeof(double) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(b->d_t, 0, sizeof(double) * count) == cudaSuccess &&
             cudaMemset(b->d_steps, 0, sizeof(long long) * count) == cudaSuccess &&
             cudaMemset(b->d_err, 0, sizeof(unsigned int) * count) == cudaSuccess &&
             cudaMemset(b->d_fb, 0, sizeof(unsigned long long)) == cudaSuccess;
    }
    if (!ok) {
        gks_batch_destroy(b);
        cudaGetLastError();
        return GKS_ENOMEM;
    }
    *out = b;
    return GKS_OK;
}

void gks_batch_destroy(gks_batch* b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->W);
    cudaFree(b->Wf);
    cudaFree(b->Ws);
    cudaFree(b->A);
    cudaFree(b->d_off);
    cudaFree(b->d_n);
    cudaFree(b->d_order);
    cudaFree(b->d_queue);
    cudaFree(b->d_dx);
    cudaFree(b->d_t);
    cudaFree(b->d_speed);
    cudaFree(b->d_steps);
    cudaFree(b->d_err);
    cudaFree(b->d_fb);
    delete b;
}

const char* gks_batch_last_error(const gks_batch* b) { return b ? b->err.c_str() : "null batch"; }

gks_status gks_batch_set_gas(gks_batch* b, const gks_gas* gas)
{
    if (!b || !gas) return GKS_EINVAL;
    if (!(gas->gamma > 1.0 && gas->gamma < 3.0) || !(gas->mu >= 0.0) || !(gas->Pr > 0.0))
        return bfail(b, GKS_EINVAL, "gas parameters out of range");
    b->gas = *gas;
    ++b->version;
    return GKS_OK;
}

gks_status gks_batch_set_scheme(gks_batch* b, const gks_scheme* s)
{
    if (!b || !s) return GKS_EINVAL;
    gks_status code = GKS_OK;
    if (const char* why = gks::scheme_problem(s, 1, &code)) return bfail(b, code, "%s", why);
    if (s->recon != GKS_RECON_TENO_D || s->charvars)
        return bfail(b, GKS_EUNSUPPORTED, "batches reconstruct with component-wise TENO-D only");
    b->sch = *s;
    ++b->version;
    return GKS_OK;
}

gks_status gks_batch_set_stream(gks_batch* b, void* stream)
{
    if (!b) return GKS_EINVAL;
    b->stream = (cudaStream_t)stream;
    return GKS_OK;
}

gks_status gks_batch_set_state(gks_batch* b, const double* W, int on_device)
{
    if (!b || !W || (on_device != GKS_HOST_MEMORY && on_device != GKS_DEVICE_MEMORY)) return GKS_EINVAL;
    BCK(cudaMemcpyAsync(b->W, W, sizeof(double) * 3 * (size_t)b->total,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemsetAsync(b->d_t, 0, sizeof(double) * b->count, b->stream));
    BCK(cudaMemsetAsync(b->d_steps, 0, sizeof(long long) * b->count, b->stream));
    BCK(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned int) * b->count, b->stream));
    BCK(cudaMemsetAsync(b->d_fb, 0, sizeof(unsigned long long), b->stream));
    return order_problems(b);
}

gks_status gks_batch_get_state(gks_batch* b, double* W, int on_device)
{
    if (!b || !W || (on_device != GKS_HOST_MEMORY && on_device != GKS_DEVICE_MEMORY)) return GKS_EINVAL;
    BCK(cudaMemcpyAsync(W, b->W, sizeof(double) * 3 * (size_t)b->total,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return GKS_OK;
}

gks_status gks_batch_set_launch(gks_batch* b, int threads, int blocks_per_sm)
{
    if (!b || (threads != 128 && threads != 256) || blocks_per_sm < 1 || blocks_per_sm > 16) return GKS_EINVAL;
    b->threads = threads;
    b->blocks_per_sm = blocks_per_sm;
    return GKS_OK;
}

gks_status gks_batch_advance_to(gks_batch* b, double t_end, long long max_steps)
{
    const NvtxRange range("gks_batch_advance_to");
    if (!b || !std::isfinite(t_end)) return GKS_EINVAL;
    gks_status s = run_batch(b, t_end, max_steps, b->threads, b->blocks_per_sm);
    if (s) return s;
    BCK(cudaStreamSynchronize(b->stream));
    std::vector<unsigned int> err(b->count);
    BCK(cudaMemcpy(err.data(), b->d_err, sizeof(unsigned int) * b->count, cudaMemcpyDeviceToHost));
    int bad = 0, first = -1;
    for (int k = 0; k < b->count; ++k)
        if (err[k]) {
            if (first < 0) first = k;
            ++bad;
        }
    if (bad)
        return bfail(b, GKS_ENONPHYSICAL, "%d problem(s) stopped on a non-physical state (first: problem %d, error word %u)",
                     bad, first, err[first]);
    return GKS_OK;
}

gks_status gks_batch_get_progress(gks_batch* b, double* t, long long* steps, unsigned int* err,
                                  long long* fallbacks)
{
    if (!b) return GKS_EINVAL;
    BCK(cudaStreamSynchronize(b->stream));
    if (t) BCK(cudaMemcpy(t, b->d_t, sizeof(double) * b->count, cudaMemcpyDeviceToHost));
    if (steps) BCK(cudaMemcpy(steps, b->d_steps, sizeof(long long) * b->count, cudaMemcpyDeviceToHost));
    if (err) BCK(cudaMemcpy(err, b->d_err, sizeof(unsigned int) * b->count, cudaMemcpyDeviceToHost));
    if (fallbacks) {
        unsigned long long f = 0;
        BCK(cudaMemcpy(&f, b->d_fb, sizeof f, cudaMemcpyDeviceToHost));
        *fallbacks = (long long)f;
    }
    return GKS_OK;
}

gks_status gks_batch_tune(gks_batch* b, double t_probe, int use_cache, int* threads, int* blocks_per_sm,
                          double* best_ms)
{
    if (!b || !(t_probe > 0.0)) return GKS_EINVAL;
    const std::string key = cache_key(b), path = cache_path();
    if (use_cache) {
        std::ifstream in(path);
        std::string k;
        int th, bp;
        double ms;
        while (in >> k >> th >> bp >> ms)
            if (k == key && gks_batch_set_launch(b, th, bp) == GKS_OK) {
                if (threads) *threads = th;
                if (blocks_per_sm) *blocks_per_sm = bp;
                if (best_ms) *best_ms = ms;
                return GKS_OK;
            }
    }
    // time every candidate on the first t_probe of the stored state, then
    // restore it (state, times, steps, errors)
    const size_t arr = sizeof(double) * 3 * (size_t)b->total;
    double* save = nullptr;
    BCK(cudaMalloc(&save, arr));
    BCK(cudaMemcpyAsync(save, b->W, arr, cudaMemcpyDeviceToDevice, b->stream));
    std::vector<double> t0(b->count);
    BCK(cudaMemcpyAsync(t0.data(), b->d_t, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand_threads[2] = {128, 256};
    const int cand_bps[4] = {1, 2, 4, 8};
    int best_t = b->threads, best_b = b->blocks_per_sm;
    double best = 1e300;
    gks_status st = GKS_OK;
    for (int ti = 0; ti < 2 && st == GKS_OK; ++ti)
        for (int bi = 0; bi < 4 && st == GKS_OK; ++bi) {
            cudaMemcpyAsync(b->W, save, arr, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(b->d_t, t0.data(), sizeof(double) * b->count, cudaMemcpyHostToDevice, b->stream);
            cudaEventRecord(e0, b->stream);
            st = run_batch(b, t_probe, 0, cand_threads[ti], cand_bps[bi]);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = GKS_ECUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == GKS_OK && ms < best) {
                best = ms;
                best_t = cand_threads[ti];
                best_b = cand_bps[bi];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(b->W, save, arr, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->d_t, t0.data(), sizeof(double) * b->count, cudaMemcpyHostToDevice, b->stream);
    cudaMemsetAsync(b->d_steps, 0, sizeof(long long) * b->count, b->stream);
    cudaMemsetAsync(b->d_err, 0, sizeof(unsigned int) * b->count, b->stream);
    cudaMemsetAsync(b->d_fb, 0, sizeof(unsigned long long), b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(save);
    if (st) return st;
    gks_batch_set_launch(b, best_t, best_b);
    if (threads) *threads = best_t;
    if (blocks_per_sm) *blocks_per_sm = best_b;
    if (best_ms) *best_ms = best;
    std::ofstream o(path, std::ios::app);
    if (o) o << key << " " << best_t << " " << best_b << " " << std::setprecision(17) << best << "\n";
    return GKS_OK;
}

long long gks_batch_launches(const gks_batch* b) { return b ? b->launches : 0; }

}  // extern "C"
