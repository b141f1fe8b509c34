// gks_api.cu -- host runtime and C ABI (include/gks.h) of the TENO-D
// gas-kinetic scheme library.
//
// The context owns three ghosted float64 device arrays (state W, stage state
// W*, stage accumulator A), a device-resident DevState (t, dt, CFL rate,
// error word, counters) and, once advance_to has run, a CUDA graph of
// GRAPH_STEPS consecutive S2O4 steps.  Time, time step and completion live
// on the device, so a replayed graph needs no host round trip per step;
// the host reads the completion flag once per replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gks.h"
#include "gks_aux.cuh"
#include "gks_ctx.h"
#include "gks_launch.h"

using namespace gks;

namespace {
constexpr int GRAPH_STEPS = 8;

// interior [nv][ny][nx] <-> ghosted layout (1-D: ny = 1, no ghost rows)
__device__ __forceinline__ long long ghosted_index(const GridDev& g, long long k)
{
    const int ny = (g.dim == 2) ? g.ny : 1;
    const long long per_v = (long long)g.nx * ny;
    const int v = (int)(k / per_v);
    const long long r = k - v * per_v;
    const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
    return (long long)v * g.plane + (long long)((g.dim == 2 ? NG : 0) + j) * g.pitch + NG + i;
}
__global__ void k_unpack(GridDev g, const double* __restrict__ src, double* __restrict__ arr, long long n)
{
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < n; k += 256ll * gridDim.x) arr[ghosted_index(g, k)] = src[k];
}
__global__ void k_pack(GridDev g, const double* __restrict__ arr, double* __restrict__ dst, long long n)
{
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < n; k += 256ll * gridDim.x) dst[k] = arr[ghosted_index(g, k)];
}
}  // namespace


namespace gks {
namespace rt {

gks_status fail(gks_ctx* c, gks_status s, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

}  // namespace rt
}  // namespace gks

using gks::rt::fail;

namespace {

double internal_dof(int dim, double gamma)
{
    // 2-D: K = (5 - 3 gamma)/(gamma - 1) + 1 (Sec. 2.1); 1-D: K = (3 - gamma)/(gamma - 1)
    return dim == 2 ? (5.0 - 3.0 * gamma) / (gamma - 1.0) + 1.0 : (3.0 - gamma) / (gamma - 1.0);
}

}  // namespace

namespace gks {
namespace rt {

HostFlux host_flux(const gks_ctx* c)
{
    HostFlux h;
    h.gamma = c->gas.gamma;
    h.K = internal_dof(c->desc.dim, c->gas.gamma);
    h.ntot = h.K + c->desc.dim;
    h.c1 = c->sch.c1;
    h.c2 = c->sch.c2;
    h.mu = c->gas.mu;
    h.prfac = (c->sch.tau_mode == GKS_TAU_NS) ? 1.0 / c->gas.Pr - 1.0 : 0.0;
    h.tau_mode = c->sch.tau_mode;
    h.merge = c->sch.merge;
    return h;
}

}  // namespace rt
}  // namespace gks
using gks::rt::host_flux;

namespace {

}  // namespace

namespace gks {
namespace rt {

TenoParams teno_params(const gks_ctx* c, bool tangential)
{
    TenoParams t;
    t.eps = c->sch.eps;
    t.q = c->sch.q;
    t.ct1 = tangential ? c->sch.ct1_t : c->sch.ct1;
    t.ct2 = tangential ? c->sch.ct2_t : c->sch.ct2;
    t.recon = c->sch.charvars ? REC_TENO_CHAR : c->sch.recon;
    t.d_hi = c->sch.d_hi;
    t.d_lo = c->sch.d_lo;
    t.eps_ao = c->sch.eps_ao;
    return t;
}

}  // namespace rt
}  // namespace gks
using gks::rt::teno_params;

namespace {

bool prepared_f32 = false, prepared_f64 = false;

// ---------------------------------------------------------------- profiling
// Returns the index of an event pair whose start was recorded, or -1.
int prof_begin(gks_ctx* c, cudaStream_t st, int kind)
{
    if (!c->prof || c->capturing) return -1;
    if (c->ev_used == c->ev.size()) {
        if (c->ev.size() >= 8192) return -1;
        gks_ctx::EvPair p{};
        if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return -1;
        c->ev.push_back(p);
    }
    gks_ctx::EvPair& p = c->ev[c->ev_used];
    p.kind = kind;
    if (cudaEventRecord(p.a, st) != cudaSuccess) return -1;
    return (int)c->ev_used++;
}

void prof_end(gks_ctx* c, cudaStream_t st, int idx)
{
    if (idx >= 0) cudaEventRecord(c->ev[idx].b, st);
}

// fold the recorded pairs into per-kind totals and recycle the events
cudaError_t prof_harvest(gks_ctx* c)
{
    if (!c->ev_used) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1].b);
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k < c->ev_used; ++k) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->ev[k].a, c->ev[k].b);
        if (e != cudaSuccess) return e;
        c->prof_n[c->ev[k].kind] += 1;
        c->prof_ms[c->ev[k].kind] += ms;
    }
    c->ev_used = 0;
    return cudaSuccess;
}

// ---------------------------------------------------------------- launches
// Ghost layers of W or W*.  On the float32 path the stage kernels read W* in
// float32 (and, in 2-D, W through its float32 shadow), so those ghosts are
// filled instead of the float64 ones.
}  // namespace

namespace gks {
namespace rt {

gks_status enqueue_ghosts(gks_ctx* c, double* arr, cudaStream_t st)
{
    const int gx = c->desc.nx + 2 * NG;
    const int n = (c->desc.dim == 1) ? 2 * NG : 2 * NG * gx + 2 * NG * c->desc.ny;
    const int pi = prof_begin(c, st, 1);
    float* shadow = (arr == c->Ws) ? c->Wsf : (arr == c->W ? c->Wf : nullptr);
    const double toff = (arr == c->Ws) ? 0.5 : 0.0;  // W* belongs to t + dt/2
    if (shadow) k_fill_ghosts<float><<<(n + 127) / 128, 128, 0, st>>>(c->g, shadow, c->ds, toff);
    else k_fill_ghosts<double><<<(n + 127) / 128, 128, 0, st>>>(c->g, arr, c->ds, toff);
    CK(cudaGetLastError());
    prof_end(c, st, pi);
    ++c->launches;
    return GKS_OK;
}

gks_status fill_ghosts_f64(gks_ctx* c, double* arr, cudaStream_t st)
{
    const int gx = c->desc.nx + 2 * NG;
    const int n = (c->desc.dim == 1) ? 2 * NG : 2 * NG * gx + 2 * NG * c->desc.ny;
    k_fill_ghosts<double><<<(n + 127) / 128, 128, 0, st>>>(c->g, arr, c->ds, 0.0);
    CK(cudaGetLastError());
    ++c->launches;
    return GKS_OK;
}

}  // namespace rt
}  // namespace gks
using gks::rt::enqueue_ghosts;

namespace {

gks_status enqueue_stage(gks_ctx* c, int stage, int with_sigma, cudaStream_t st)
{
    const HostFlux hf = host_flux(c);
    const TenoParams tn = teno_params(c, false), tt = teno_params(c, true);
    const bool f32 = c->desc.precision == GKS_FP32_FLUX;
    if (c->desc.dim == 1) {
        Stage1DArgs a{};
        a.stage = stage;
        a.with_sigma = with_sigma;
        a.idx = 1.0 / c->g.dx;
        if (f32) {
            // float32 W* (Wsf) and accumulator increment (inc1)
            float* inc = static_cast<float*>(c->inc1);
            if (stage == 1) { a.src = c->W; a.srcf = c->Wf; a.out0f = c->Wsf; a.out1f = inc; }
            else { a.srcf = c->Wsf; a.base = c->W; a.out0 = c->W; a.out0f = c->Wf; a.accf = inc; }
        } else if (stage == 1) {
            a.src = c->W; a.out0 = c->Ws; a.out1 = c->Ac;
        } else {
            a.src = c->Ws; a.out0 = c->W; a.acc = c->Ac;
        }
        const int pi = prof_begin(c, st, 0);
        CK(launch_stage1d(f32, c->g, a, hf, tn, c->ds, st));
        prof_end(c, st, pi);
        ++c->launches;
        return GKS_OK;
    }
    for (int pass = 0; pass < 2; ++pass) {
        SweepArgs a{};
        a.stage = stage;
        a.pass = pass;
        a.dirn = pass;  // x faces first, then y faces
        a.src = (stage == 1) ? c->W : c->Ws;
        a.srcf = (stage == 1) ? c->Wf : c->Wsf;
        a.basef = c->Wf;
        // float64 path: stage 2 starts from the accumulator; float32 path: from W
        // (its accumulator is the increment inc1)
        a.base = (stage == 1 || f32) ? c->W : c->Ac;
        a.out0 = (stage == 1) ? c->Ws : c->W;
        a.out0f = (stage == 1) ? c->Wsf : c->Wf;
        a.out1 = (stage == 1) ? c->Ac : nullptr;
        a.inc0 = c->inc0;
        a.inc1 = c->inc1;
        a.hmin = fmin(c->g.dx, c->g.dy);
        if (pass == 0) {
            a.nn = c->desc.nx; a.nt = c->desc.ny; a.sn = 1; a.st = c->g.pitch;
            a.ihn = 1.0 / c->g.dx; a.iht = 1.0 / c->g.dy;
        } else {
            a.nn = c->desc.ny; a.nt = c->desc.nx; a.sn = c->g.pitch; a.st = 1;
            a.ihn = 1.0 / c->g.dy; a.iht = 1.0 / c->g.dx;
        }
        a.with_sigma = (pass == 1) ? with_sigma : 0;
        const int pi = prof_begin(c, st, 0);
        cudaError_t e = f32 ? launch_sweep_f32(c->g, a, hf, tn, tt, c->ds, st)
                            : launch_sweep_f64(c->g, a, hf, tn, tt, c->ds, st);
        CK(e);
        prof_end(c, st, pi);
        ++c->launches;
    }
    return GKS_OK;
}

__global__ void k_prepare(DevState* ds, int mode, double dt, double t_end, long long max_steps)
{
    // mode 0: fixed dt, no t_end; 1: CFL dt towards t_end; 2: reset t, counters
    // and error word; 3: CFL dt, no t_end
    if (threadIdx.x || blockIdx.x) return;
    if (mode == 2) {
        ds->t = 0.0;
        ds->steps = 0;
        ds->fallbacks = 0;
        ds->err = 0;
    }
    ds->done = 0;
    ds->sigma = 0;
    ds->max_steps = max_steps;
    if (mode == 0) {
        ds->dt = dt;
        ds->fixed_dt = 1;
        ds->t_end = INFINITY;
    } else {
        ds->fixed_dt = 0;
        ds->t_end = (mode == 1) ? t_end : INFINITY;
    }
}

gks_status enqueue_sigma(gks_ctx* c, cudaStream_t st)
{
    const long long ncell = (long long)c->desc.nx * (c->desc.dim == 2 ? c->desc.ny : 1);
    int blocks = (int)((ncell + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    const int pi = prof_begin(c, st, 2);
    if (c->desc.precision == GKS_FP32_FLUX) k_sigma<float><<<blocks, 256, 0, st>>>(c->g, c->W, c->ds);
    else k_sigma<double><<<blocks, 256, 0, st>>>(c->g, c->W, c->ds);
    CK(cudaGetLastError());
    prof_end(c, st, pi);
    ++c->launches;
    return GKS_OK;
}

gks_status enqueue_commit(gks_ctx* c, int init, cudaStream_t st)
{
    const int pi = prof_begin(c, st, 2);
    k_commit<<<1, 32, 0, st>>>(c->ds, init);
    CK(cudaGetLastError());
    prof_end(c, st, pi);
    ++c->launches;
    return GKS_OK;
}

// one S2O4 step: ghosts(W), stage 1, ghosts(W*), stage 2 (+ CFL rate), commit
gks_status enqueue_step(gks_ctx* c, cudaStream_t st)
{
    gks_status s;
    if ((s = enqueue_ghosts(c, c->W, st))) return s;
    if ((s = enqueue_stage(c, 1, 0, st))) return s;
    if ((s = enqueue_ghosts(c, c->Ws, st))) return s;
    if ((s = enqueue_stage(c, 2, 1, st))) return s;
    return enqueue_commit(c, 0, st);
}

gks_status sync_state(gks_ctx* c)
{
    CK(cudaMemcpyAsync(c->hs, c->ds, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GKS_OK;
}

gks_status check_err(gks_ctx* c)
{
    if (c->hs->err & 2u)
        return fail(c, GKS_ENONPHYSICAL, "positivity fallback failed: an adjacent cell state is non-physical");
    if (c->hs->err & 1u)
        return fail(c, GKS_ENONPHYSICAL, "non-physical or non-finite state after an update (t = %.17g)",
                    c->hs->t);
    return GKS_OK;
}

}  // namespace

namespace gks {
namespace rt {

gks_status copy_interior(gks_ctx* c, double* arr, const double* W, int on_device, bool in)
{
    // A caller's array [nv][ny][nx] is moved in one contiguous copy (host
    // arrays through a device staging buffer) and scattered into / gathered
    // from the ghosted layout by a kernel: one large transfer runs at the
    // link's rate, where a pitched copy of short rows does not.
    // on_device: GKS_HOST_MEMORY (returns when the copy is done),
    // GKS_DEVICE_MEMORY, GKS_HOST_PINNED_ASYNC (enqueued on the stream only)
    if (on_device != GKS_HOST_MEMORY && on_device != GKS_DEVICE_MEMORY && on_device != GKS_HOST_PINNED_ASYNC)
        return GKS_EINVAL;
    const bool host = on_device != GKS_DEVICE_MEMORY;
    const long long n = (long long)c->nv * c->desc.nx * ((c->desc.dim == 2) ? c->desc.ny : 1);
    const double* src = W;
    double* dst = const_cast<double*>(W);
    if (host) {
        if (!c->stage) CK(cudaMalloc(&c->stage, sizeof(double) * (size_t)n));
        src = dst = c->stage;
        if (in) CK(cudaMemcpyAsync(c->stage, W, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    }
    const int blocks = (int)std::min<long long>((n + 255) / 256, 8192);
    if (in) k_unpack<<<blocks, 256, 0, c->stream>>>(c->g, src, arr, n);
    else k_pack<<<blocks, 256, 0, c->stream>>>(c->g, arr, dst, n);
    CK(cudaGetLastError());
    ++c->launches;
    if (host && !in)
        CK(cudaMemcpyAsync(const_cast<double*>(W), c->stage, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                           c->stream));
    if (on_device != GKS_HOST_PINNED_ASYNC) CK(cudaStreamSynchronize(c->stream));
    return GKS_OK;
}

}  // namespace rt
}  // namespace gks
using gks::rt::copy_interior;

namespace {

gks_status build_graph(gks_ctx* c)
{
    if (c->graph && c->graph_version == c->param_version) return GKS_OK;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const long long before = c->launches;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    gks_status s = GKS_OK;
    for (int k = 0; k < GRAPH_STEPS && s == GKS_OK; ++k) s = enqueue_step(c, c->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->capturing = false;
    c->graph_nodes = c->launches - before;
    c->launches = before;  // captured, not launched
    if (s != GKS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    CK(e);
    e = cudaGraphInstantiate(&c->graph, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    c->graph_version = c->param_version;
    return GKS_OK;
}

gks_status prepare_kernels(gks_ctx* c)
{
    cudaError_t e = cudaSuccess;
    if (c->desc.dim == 2 && c->desc.precision == GKS_FP32_FLUX && !prepared_f32) {
        e = prepare_sweep_f32();
        prepared_f32 = (e == cudaSuccess);
    }
    if (c->desc.dim == 2 && c->desc.precision == GKS_FP64 && !prepared_f64) {
        e = prepare_sweep_f64();
        prepared_f64 = (e == cudaSuccess);
    }
    CK(e);
    return GKS_OK;
}

}  // namespace

// ====================================================================== C ABI
namespace gks {
const char* scheme_problem(const gks_scheme* s, int check_cfl, gks_status* code)
{
    *code = GKS_EINVAL;
    if (check_cfl && !(s->cfl > 0.0)) return "scheme parameters out of range: cfl must be > 0";
    if (s->q < 1 || s->q > 32 || !(s->eps >= 0.0) || !(s->ct1 >= 0.0) || !(s->ct2 >= 0.0) || !(s->ct1_t >= 0.0) ||
        !(s->ct2_t >= 0.0) || s->tau_mode < 0 || s->tau_mode > 2 || !(s->c1 >= 0.0) || !(s->c2 >= 0.0))
        return "scheme parameters out of range";
    if (s->recon < GKS_RECON_TENO_D || s->recon > GKS_RECON_TENO5 ||
        (s->recon == GKS_RECON_WENO_AO && (!(s->d_hi > 0.0 && s->d_hi <= 1.0) || !(s->d_lo >= 0.0 && s->d_lo <= 1.0) ||
                                           !(s->eps_ao > 0.0))) ||
        (s->recon == GKS_RECON_WENO_Z && !(s->eps_ao > 0.0)))
        return "reconstruction parameters out of range";
    if (s->merge != GKS_MERGE_KINETIC && s->merge != GKS_MERGE_AVERAGE)
        return "merge must be GKS_MERGE_KINETIC or GKS_MERGE_AVERAGE";
    if (s->charvars != 0 && s->charvars != 1) return "charvars must be 0 or 1";
    if (s->charvars && s->recon != GKS_RECON_TENO_D) {
        *code = GKS_EUNSUPPORTED;
        return "characteristic variables are taken with TENO-D only";
    }
    if (!s->positivity_fallback) {
        *code = GKS_EUNSUPPORTED;
        return "the kernels always apply the positivity fallback";
    }
    *code = GKS_OK;
    return nullptr;
}
}  // namespace gks

extern "C" {

const char* gks_status_string(int s)
{
    switch (s) {
    case GKS_OK: return "ok";
    case GKS_EINVAL: return "invalid argument";
    case GKS_ENOMEM: return "out of memory";
    case GKS_ECUDA: return "CUDA error";
    case GKS_ENONPHYSICAL: return "non-physical state";
    case GKS_ETIMEOUT: return "device wait timed out";
    case GKS_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char* gks_last_error(const gks_ctx* c) { return c ? c->err.c_str() : "null context"; }

long long gks_kernel_launches(const gks_ctx* c) { return c ? c->launches : 0; }

gks_status gks_create(const gks_grid_desc* d, gks_ctx** out)
{
    if (!d || !out) return GKS_EINVAL;
    *out = nullptr;
    if (d->dim != 1 && d->dim != 2) return GKS_EINVAL;
    if (d->nx < 3 || (d->dim == 2 && d->ny < 3)) return GKS_EINVAL;
    if (!(d->x1 > d->x0) || (d->dim == 2 && !(d->y1 > d->y0))) return GKS_EINVAL;
    if (d->precision != GKS_FP64 && d->precision != GKS_FP32_FLUX) return GKS_EINVAL;
    for (int k = 0; k < 4; ++k) {
        if (d->bc[k] < GKS_BC_PERIODIC || d->bc[k] > GKS_BC_MOVING_SHOCK) return GKS_EINVAL;
        // the wall-after-x0 and moving-shock rules are rules of the y sides
        if ((d->bc[k] == GKS_BC_WALL_AFTER_X0 || d->bc[k] == GKS_BC_MOVING_SHOCK) && (k < 2 || d->dim != 2))
            return GKS_EINVAL;
    }
    if ((d->bc[0] == GKS_BC_PERIODIC) != (d->bc[1] == GKS_BC_PERIODIC)) return GKS_EINVAL;
    if (d->dim == 2 && (d->bc[2] == GKS_BC_PERIODIC) != (d->bc[3] == GKS_BC_PERIODIC)) return GKS_EINVAL;
    if ((long long)d->nx * (d->dim == 2 ? d->ny : 1) > (1ll << 31)) return GKS_EINVAL;

    gks_ctx* c = new (std::nothrow) gks_ctx();
    if (!c) return GKS_ENOMEM;
    c->desc = *d;
    if (d->dim == 1) c->desc.ny = 1;
    c->nv = d->dim + 2;
    c->gas = {1.4, 0.0, 1.0};
    c->sch.cfl = 0.5;
    c->sch.c1 = 0.01;
    c->sch.c2 = 1.0;
    c->sch.ct1 = c->sch.ct1_t = 1e-7;
    c->sch.ct2 = c->sch.ct2_t = 1e-5;
    c->sch.eps = 1e-40;
    c->sch.q = 7;
    c->sch.tau_mode = GKS_TAU_EULER;
    c->sch.positivity_fallback = 1;
    c->sch.recon = GKS_RECON_TENO_D;
    c->sch.d_hi = c->sch.d_lo = 0.85;
    c->sch.eps_ao = 1e-8;
    c->sch.merge = GKS_MERGE_KINETIC;
    c->sch.charvars = 0;

    GridDev& g = c->g;
    g.dim = d->dim;
    g.nx = d->nx;
    g.ny = c->desc.ny;
    g.pitch = ((d->nx + 2 * NG + 15) / 16) * 16;
    g.gy = (d->dim == 2) ? d->ny + 2 * NG : 1;
    g.plane = (long long)g.gy * g.pitch;
    g.dx = (d->x1 - d->x0) / d->nx;
    g.dy = (d->dim == 2) ? (d->y1 - d->y0) / d->ny : 1.0;
    for (int k = 0; k < 4; ++k) g.bc[k] = d->bc[k];
    g.gamma = c->gas.gamma;
    g.mu = c->gas.mu;
    g.ox = d->x0;
    g.oy = (d->dim == 2) ? d->y0 : 0.0;
    g.bs = BcStates{};

    c->arr_bytes = (size_t)c->nv * g.plane * sizeof(double);
    cudaError_t e1 = cudaMalloc(&c->W, c->arr_bytes);
    cudaError_t e2 = cudaMalloc(&c->Ws, c->arr_bytes);
    cudaError_t e3 = cudaMalloc(&c->Ac, c->arr_bytes);
    cudaError_t e4 = cudaMalloc(&c->ds, sizeof(DevState));
    cudaError_t e5 = cudaMallocHost(&c->hs, sizeof(DevState));
    cudaError_t e6 = cudaSuccess, e7 = cudaSuccess;
    if (d->dim == 2) {
        const size_t inc_bytes = (size_t)c->nv * g.plane * (d->precision == GKS_FP32_FLUX ? 4 : 8);
        e6 = cudaMalloc(&c->inc0, inc_bytes);
        e7 = cudaMalloc(&c->inc1, inc_bytes);
        if (d->precision == GKS_FP32_FLUX && e6 == cudaSuccess && e7 == cudaSuccess) {
            const size_t fb = (size_t)c->nv * g.plane * sizeof(float);
            e6 = cudaMalloc(&c->Wf, fb);
            if (e6 == cudaSuccess) e6 = cudaMalloc(&c->Wsf, fb);
        }
    } else if (d->precision == GKS_FP32_FLUX) {
        // 1-D float32 path: W* and the accumulator increment in float32, and a
        // float32 shadow of W (the stage-1 input)
        const size_t fb = (size_t)c->nv * g.plane * sizeof(float);
        e6 = cudaMalloc(&c->Wsf, fb);
        e7 = cudaMalloc(&c->inc1, fb);
        if (e6 == cudaSuccess) e6 = cudaMalloc(&c->Wf, fb);
    }
    if (e1 || e2 || e3 || e4 || e5 || e6 || e7) {
        gks_destroy(c);
        cudaGetLastError();
        return GKS_ENOMEM;
    }
    cudaMemset(c->W, 0, c->arr_bytes);
    cudaMemset(c->Ws, 0, c->arr_bytes);
    cudaMemset(c->Ac, 0, c->arr_bytes);
    memset(c->hs, 0, sizeof(DevState));
    c->hs->cfl = c->sch.cfl;
    c->hs->t_end = INFINITY;
    if (cudaMemcpy(c->ds, c->hs, sizeof(DevState), cudaMemcpyHostToDevice) != cudaSuccess ||
        prepare_kernels(c) != GKS_OK) {
        gks_destroy(c);
        return GKS_ECUDA;
    }
    *out = c;
    return GKS_OK;
}

void gks_destroy(gks_ctx* c)
{
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto& p : c->ev) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    cudaFree(c->W);
    cudaFree(c->Ws);
    cudaFree(c->Ac);
    cudaFree(c->inc0);
    cudaFree(c->inc1);
    cudaFree(c->Wf);
    cudaFree(c->Wsf);
    cudaFree(c->stage);
    cudaFree(c->ds);
    if (c->hs) cudaFreeHost(c->hs);
    delete c;
}

gks_status gks_set_gas(gks_ctx* c, const gks_gas* gas)
{
    if (!c || !gas) return GKS_EINVAL;
    if (!(gas->gamma > 1.0 && gas->gamma < 3.0) || !(gas->mu >= 0.0) || !(gas->Pr > 0.0))
        return fail(c, GKS_EINVAL, "gas parameters out of range");
    c->gas = *gas;
    c->cfl_dt_ready = false;
    c->g.gamma = gas->gamma;
    c->g.mu = gas->mu;
    ++c->param_version;
    return GKS_OK;
}

gks_status gks_set_boundary_states(gks_ctx* c, const gks_boundary_states* b)
{
    if (!c || !b) return GKS_EINVAL;
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(b->inflow[k]) || !std::isfinite(b->pre[k]))
            return fail(c, GKS_EINVAL, "boundary states must be finite");
    if (!(b->shock_theta > 0.0 && b->shock_theta < 3.14159265358979323846) || !std::isfinite(b->shock_x0) ||
        !std::isfinite(b->shock_speed))
        return fail(c, GKS_EINVAL, "shock angle must lie in (0, pi); shock data finite");
    BcStates& s = c->g.bs;
    for (int k = 0; k < 4; ++k) { s.in[k] = b->inflow[k]; s.pre[k] = b->pre[k]; }
    s.x0 = b->shock_x0;
    s.cot = std::cos(b->shock_theta) / std::sin(b->shock_theta);
    s.vx = b->shock_speed / std::sin(b->shock_theta);
    ++c->param_version;
    return GKS_OK;
}


gks_status gks_set_scheme(gks_ctx* c, const gks_scheme* s)
{
    if (!c || !s) return GKS_EINVAL;
    gks_status code = GKS_OK;
    if (const char* why = gks::scheme_problem(s, 1, &code)) return fail(c, code, "%s", why);
    c->sch = *s;
    ++c->param_version;
    c->cfl_dt_ready = false;
    // cfl lives in the device state
    c->hs->cfl = s->cfl;
    CK(cudaMemcpyAsync(&c->ds->cfl, &c->hs->cfl, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GKS_OK;
}

gks_status gks_set_stream(gks_ctx* c, void* stream)
{
    if (!c) return GKS_EINVAL;
    c->stream = (cudaStream_t)stream;
    return GKS_OK;
}

gks_status gks_set_state(gks_ctx* c, const double* W, int on_device)
{
    if (!c || !W) return GKS_EINVAL;
    c->cfl_dt_ready = false;
    gks_status s = copy_interior(c, c->W, W, on_device, true);
    if (s) return s;
    if (c->Wf) {
        const long long n = (long long)c->nv * c->g.plane;
        k_to_float<<<(int)((n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256), 256, 0, c->stream>>>(c->W, c->Wf, n);
        CK(cudaGetLastError());
        ++c->launches;
    }
    k_prepare<<<1, 32, 0, c->stream>>>(c->ds, 2, 0.0, INFINITY, 0);
    CK(cudaGetLastError());
    ++c->launches;
    if (on_device == GKS_HOST_PINNED_ASYNC) {
        // the host mirror of t and the counters is refreshed by the next
        // synchronising call
        c->hs->t = 0.0;
        c->hs->steps = 0;
        return GKS_OK;
    }
    return sync_state(c);
}

gks_status gks_get_state(gks_ctx* c, double* W, int on_device)
{
    if (!c || !W) return GKS_EINVAL;
    return copy_interior(c, c->W, W, on_device, false);
}

gks_status gks_get_buffer(gks_ctx* c, int which, double* W, int on_device)
{
    if (!c || !W || which < 0 || which > 2 || (on_device != GKS_HOST_MEMORY && on_device != GKS_DEVICE_MEMORY))
        return GKS_EINVAL;
    double* arr = which == 0 ? c->W : (which == 1 ? c->Ws : c->Ac);
    if (c->Wsf && which > 0) {
        // float32 path: W* lives in float32, the accumulator as an increment
        const long long n = (long long)c->nv * c->g.plane;
        const int blocks = (int)((n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256);
        if (which == 1) k_widen<<<blocks, 256, 0, c->stream>>>(c->Wsf, c->Ws, n);
        else k_accumulator<<<blocks, 256, 0, c->stream>>>(c->W, static_cast<const float*>(c->inc1), c->Ac, n);
        CK(cudaGetLastError());
        ++c->launches;
    }
    return copy_interior(c, arr, W, on_device, false);
}

gks_status gks_compute_dt(gks_ctx* c, double* dt)
{
    if (!c || !dt) return GKS_EINVAL;
    CK(cudaMemsetAsync(&c->ds->sigma, 0, sizeof(unsigned long long), c->stream));
    gks_status s = enqueue_sigma(c, c->stream);
    if (s) return s;
    if ((s = sync_state(c))) return s;
    if ((s = check_err(c))) return s;
    double sig;
    memcpy(&sig, &c->hs->sigma, sizeof sig);
    *dt = c->sch.cfl / sig;
    CK(cudaMemsetAsync(&c->ds->sigma, 0, sizeof(unsigned long long), c->stream));
    return GKS_OK;
}

gks_status gks_stage(gks_ctx* c, int stage, double dt)
{
    const NvtxRange range("gks_stage");
    if (!c || (stage != 1 && stage != 2) || !(dt > 0.0) || !std::isfinite(dt)) return GKS_EINVAL;
    c->cfl_dt_ready = false;
    k_prepare<<<1, 32, 0, c->stream>>>(c->ds, 0, dt, 0.0, 0);
    CK(cudaGetLastError());
    ++c->launches;
    gks_status s = enqueue_ghosts(c, stage == 1 ? c->W : c->Ws, c->stream);
    if (s) return s;
    return enqueue_stage(c, stage, 0, c->stream);
}

gks_status gks_step(gks_ctx* c, double dt)
{
    const NvtxRange range("gks_step");
    if (!c || !std::isfinite(dt)) return GKS_EINVAL;
    gks_status s;
    if (dt > 0.0) {
        c->cfl_dt_ready = false;
        k_prepare<<<1, 32, 0, c->stream>>>(c->ds, 0, dt, 0.0, 0);
        CK(cudaGetLastError());
        ++c->launches;
    } else if (!c->cfl_dt_ready) {
        k_prepare<<<1, 32, 0, c->stream>>>(c->ds, 3, 0.0, 0.0, 0);
        CK(cudaGetLastError());
        ++c->launches;
        if ((s = enqueue_sigma(c, c->stream))) return s;
        if ((s = enqueue_commit(c, 1, c->stream))) return s;
    }
    // else: the previous CFL step's commit already chose dt from this state
    s = enqueue_step(c, c->stream);
    c->cfl_dt_ready = (s == GKS_OK && !(dt > 0.0));
    return s;
}

gks_status gks_advance_to(gks_ctx* c, double t_end, long long max_steps, long long* steps_done, double* t_out)
{
    const NvtxRange range("gks_advance_to");
    if (!c || !std::isfinite(t_end)) return GKS_EINVAL;
    c->cfl_dt_ready = false;
    gks_status s;
    if ((s = sync_state(c))) return s;
    const long long steps0 = c->hs->steps;
    if (!(c->hs->t < t_end)) {
        if (steps_done) *steps_done = 0;
        if (t_out) *t_out = c->hs->t;
        return GKS_OK;
    }
    const long long limit = max_steps > 0 ? steps0 + max_steps : 0;
    k_prepare<<<1, 32, 0, c->stream>>>(c->ds, 1, 0.0, t_end, limit);
    CK(cudaGetLastError());
    ++c->launches;
    if ((s = enqueue_sigma(c, c->stream))) return s;
    if ((s = enqueue_commit(c, 1, c->stream))) return s;
    if ((s = build_graph(c))) return s;
    for (;;) {
        CK(cudaGraphLaunch(c->graph, c->stream));
        c->launches += c->graph_nodes;
        if ((s = sync_state(c))) return s;
        if ((s = check_err(c))) return s;
        if (c->hs->done) break;
    }
    if (steps_done) *steps_done = c->hs->steps - steps0;
    if (t_out) *t_out = c->hs->t;
    return GKS_OK;
}

gks_status gks_get_diagnostics(gks_ctx* c, gks_diag* out)
{
    if (!c || !out) return GKS_EINVAL;
    gks_status s = sync_state(c);
    if (s) return s;
    out->error_word = c->hs->err;
    out->fallbacks = (long long)c->hs->fallbacks;
    out->t = c->hs->t;
    out->steps = c->hs->steps;
    out->dt = c->hs->dt;
    return check_err(c);
}

gks_status gks_profile_enable(gks_ctx* c, int enable)
{
    if (!c) return GKS_EINVAL;
    c->prof = enable != 0;
    return GKS_OK;
}

gks_status gks_profile_read(gks_ctx* c, int kind, long long* launches, double* total_ms)
{
    if (!c || kind < 0 || kind > 2) return GKS_EINVAL;
    CK(prof_harvest(c));
    if (launches) *launches = c->prof_n[kind];
    if (total_ms) *total_ms = c->prof_ms[kind];
    c->prof_n[kind] = 0;
    c->prof_ms[kind] = 0.0;
    return GKS_OK;
}

}  // extern "C"
