// gks_ctx.h -- the context object behind gks_ctx* (include/gks.h) and the
// runtime helpers that other translation units of the library use on it.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/gks.h"
#include "gks_kernels.cuh"
#include "gks_launch.h"
#include "gks_nvtx.h"

struct gks_ctx {
    gks_grid_desc desc{};
    gks::GridDev g{};
    gks_gas gas{};
    gks_scheme sch{};
    int nv = 0;
    double *W = nullptr, *Ws = nullptr, *Ac = nullptr;
    void *inc0 = nullptr, *inc1 = nullptr;  // 2-D: x-sweep increments, working precision;
                                             // 1-D float32: inc1 = accumulator increment
    float* Wf = nullptr;                     // float32 shadow of W (float32 path)
    float* Wsf = nullptr;                    // W* in float32 (float32 path)
    double* stage = nullptr;                 // device staging of host arrays (allocated on first use)
    size_t arr_bytes = 0;
    gks::DevState* ds = nullptr;      // device
    gks::DevState* hs = nullptr;      // pinned host mirror
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    long long graph_nodes = 0;
    unsigned long long param_version = 1, graph_version = 0;
    long long launches = 0;
    // the device already holds the CFL time step of the current state (set by
    // a CFL step's commit, cleared by anything else that changes W or dt)
    bool cfl_dt_ready = false;
    std::string err;
    // per-kernel event timing (gks_profile_enable)
    bool prof = false, capturing = false;
    struct EvPair {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<EvPair> ev;
    size_t ev_used = 0;
    long long prof_n[3] = {0, 0, 0};
    double prof_ms[3] = {0, 0, 0};
};

namespace gks {
namespace rt {

// records a formatted message in the context and returns s
gks_status fail(gks_ctx* c, gks_status s, const char* fmt, ...);
// fill the ghost layers of W or W* (the float32 shadow on the 2-D float32 path)
gks_status enqueue_ghosts(gks_ctx* c, double* arr, cudaStream_t st);
// fill the ghost layers of a float64 array at the state's time (whatever the
// context's precision; diagnostics that read W itself)
gks_status fill_ghosts_f64(gks_ctx* c, double* arr, cudaStream_t st);
// copy the interior [nv][ny][nx] between a caller's buffer and a ghosted array
gks_status copy_interior(gks_ctx* c, double* arr, const double* W, int on_device, bool in);
HostFlux host_flux(const gks_ctx* c);
TenoParams teno_params(const gks_ctx* c, bool tangential);

}  // namespace rt
}  // namespace gks

#define CK(call)                                                                                             \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return gks::rt::fail(c, GKS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
