// gks_noalloc.cu -- gks_step1d_noalloc: one S2O4 step of a 1-D problem that
// allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host whose device memory is owned
// by another allocator (a framework's caching allocator, or a fixed memory
// budget handed out by a scheduler), or a latency-critical loop that cannot
// afford cudaMalloc's implicit device-wide synchronisation.  For them the
// working buffers of the step (ghosted copies of W^n and W*, the stage
// accumulator, the new state and the small device-side step state) live in
// one file-scope static __device__ array, sized for at most
// GKS_NOALLOC_MAX_NX cells (about 1.6 MB, held by every GPU that loads the
// library until the process exits).  The caller passes device pointers for
// input and output only.
//
// Host code must not use the array's name as a device address (in host code
// it names a host-side stand-in).  The device address is looked up with
// cudaGetSymbolAddress on the first call made in a CUDA context (the first
// call on each device, and again after that device's context was destroyed
// and re-created, e.g. by cudaDeviceReset), with that device current, and
// cached per device together with the context's unique id.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gks.h"
#include "gks_launch.h"

using namespace gks;

namespace {

constexpr int NX_MAX = GKS_NOALLOC_MAX_NX;
constexpr int PITCH = ((NX_MAX + 2 * NG + 15) / 16) * 16;   // one ghosted row, 128-byte multiple
constexpr long long ARRAY = 3ll * PITCH;                    // three conserved variables
constexpr long long STATE_DOUBLES = (sizeof(DevState) + sizeof(double) - 1) / sizeof(double);
// layout: [W^n | W* | accumulator | new state] x ARRAY doubles, then DevState
constexpr long long SCRATCH_DOUBLES = 4 * ARRAY + STATE_DOUBLES;

static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
struct ScratchAddr {
    unsigned long long ctx_id;  // unique id of the context the address belongs to (0: none)
    double* addr;
};
ScratchAddr g_addr[MAX_DEVICES] = {};
std::mutex g_mu;

// driver entry points for the current context's unique id (looked up through
// the runtime, so the library needs no link against the driver library)
typedef int (*PfnCtxGetCurrent)(void**);
typedef int (*PfnCtxGetId)(void*, unsigned long long*);

// unique id of the current context, 0 if there is none or it is unknown
unsigned long long current_context_id()
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PfnCtxGetId>(f);
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// device address of g_scratch in the current device's context
cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    if (id == 0 || g_addr[dev].ctx_id != id || !g_addr[dev].addr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);  // makes the device's primary context current if none is
        if (e != cudaSuccess) return e;
        g_addr[dev].addr = static_cast<double*>(p);
        g_addr[dev].ctx_id = current_context_id();  // 0 (unknown): looked up again next call
    }
    *out = g_addr[dev].addr;
    return cudaSuccess;
}

// ghost source along a line of n interior cells (same rules as the library's
// ghost fill): periodic, zero gradient, mirror (velocity negated)
__device__ int ghost_source(int bc, int n, int g, bool& flip)
{
    flip = false;
    if (g >= NG && g < NG + n) return g;
    const bool low = g < NG;
    if (bc == GKS_BC_PERIODIC) return NG + (((g - NG) % n) + n) % n;
    if (bc == GKS_BC_ZEROGRAD) return low ? NG : NG + n - 1;
    flip = true;  // symmetry, reflect, no-slip: 1-D velocity negated
    return low ? 2 * NG - 1 - g : 2 * (NG + n) - 1 - g;
}

// copy the caller's interior [3][nx] into the ghosted scratch row, fill the
// ghosts, and reset the step state (everything that must start at zero)
__global__ void k_load(const double* __restrict__ Win, double* __restrict__ W, int nx, int bc0, int bc1,
                       DevState* ds, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        memset(ds, 0, sizeof(DevState));
        ds->dt = dt;
        ds->fixed_dt = 1u;
        ds->t_end = INFINITY;
    }
    if (i >= nx + 2 * NG) return;
    bool flip;
    const int src = ghost_source(i < NG ? bc0 : bc1, nx, i, flip);
    for (int v = 0; v < 3; ++v) {
        const double val = Win[(long long)v * nx + (src - NG)];
        W[(long long)v * PITCH + i] = (flip && v == 1) ? -val : val;
    }
}

template <typename E>
__global__ void k_ghosts(E* __restrict__ W, int nx, int bc0, int bc1)
{
    const int k = threadIdx.x;
    if (k >= 2 * NG) return;
    const int i = k < NG ? k : nx + k;
    bool flip;
    const int src = ghost_source(k < NG ? bc0 : bc1, nx, i, flip);
    for (int v = 0; v < 3; ++v) {
        const E val = W[(long long)v * PITCH + src];
        W[(long long)v * PITCH + i] = (flip && v == 1) ? -val : val;
    }
}

__global__ void k_store(const double* __restrict__ W, double* __restrict__ Wout, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    for (int v = 0; v < 3; ++v) Wout[(long long)v * nx + i] = W[(long long)v * PITCH + NG + i];
}

}  // namespace

extern "C" gks_status gks_step1d_noalloc(const double* W_in, double* W_out, int nx, double dx, const int* bc,
                                         const gks_gas* gas, const gks_scheme* sch, int precision, double dt,
                                         void* stream, unsigned int* error_word)
{
    if (!W_in || !W_out || !bc || !gas || !sch || nx < 3 || !(dx > 0.0) || !(dt > 0.0) || !std::isfinite(dt))
        return GKS_EINVAL;
    if (nx > NX_MAX) return GKS_EUNSUPPORTED;  // beyond the static scratch (GKS_NOALLOC_MAX_NX)
    if (precision != GKS_FP64 && precision != GKS_FP32_FLUX) return GKS_EINVAL;
    for (int k = 0; k < 2; ++k)
        if (bc[k] < GKS_BC_PERIODIC || bc[k] > GKS_BC_REFLECT) return GKS_EINVAL;
    if ((bc[0] == GKS_BC_PERIODIC) != (bc[1] == GKS_BC_PERIODIC)) return GKS_EINVAL;
    if (!(gas->gamma > 1.0 && gas->gamma < 3.0) || !(gas->mu >= 0.0) || !(gas->Pr > 0.0)) return GKS_EINVAL;
    gks_status code = GKS_OK;
    if (gks::scheme_problem(sch, 0, &code)) return code;  // the CFL number is not used here
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the call ends by reading the error word back and synchronising the
    // stream, neither of which a capturing stream allows
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return GKS_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return GKS_EINVAL;

    double* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return GKS_ECUDA;
    double* W = base;
    double* Ws = base + ARRAY;
    double* Ac = base + 2 * ARRAY;
    double* Wn = base + 3 * ARRAY;
    DevState* ds = reinterpret_cast<DevState*>(base + 4 * ARRAY);

    GridDev g{};
    g.dim = 1;
    g.nx = nx;
    g.ny = 1;
    g.pitch = PITCH;
    g.gy = 1;
    g.plane = PITCH;
    g.dx = dx;
    g.dy = 1.0;
    g.bc[0] = bc[0];
    g.bc[1] = bc[1];
    g.bc[2] = g.bc[3] = GKS_BC_ZEROGRAD;
    g.gamma = gas->gamma;
    g.mu = gas->mu;

    HostFlux hf;
    hf.gamma = gas->gamma;
    hf.K = (3.0 - gas->gamma) / (gas->gamma - 1.0);  // 1-D internal degrees of freedom
    hf.ntot = hf.K + 1.0;
    hf.c1 = sch->c1;
    hf.c2 = sch->c2;
    hf.mu = gas->mu;
    hf.prfac = (sch->tau_mode == GKS_TAU_NS) ? 1.0 / gas->Pr - 1.0 : 0.0;
    hf.tau_mode = sch->tau_mode;
    hf.merge = sch->merge;
    TenoParams tn{sch->eps, sch->q, sch->ct1, sch->ct2, sch->charvars ? REC_TENO_CHAR : sch->recon, sch->d_hi,
                  sch->d_lo, sch->eps_ao};
    const int f32 = precision == GKS_FP32_FLUX;

    // the float32 path keeps W* and the accumulator increment in float32, in
    // the same scratch regions
    float* Wsf = reinterpret_cast<float*>(Ws);
    float* incf = reinterpret_cast<float*>(Ac);
    k_load<<<(nx + 2 * NG + 127) / 128, 128, 0, st>>>(W_in, W, nx, bc[0], bc[1], ds, dt);
    Stage1DArgs a1{};
    a1.idx = 1.0 / dx;
    a1.src = W;
    if (f32) { a1.out0f = Wsf; a1.out1f = incf; }
    else { a1.out0 = Ws; a1.out1 = Ac; }
    a1.stage = 1;
    if (launch_stage1d(f32, g, a1, hf, tn, ds, st) != cudaSuccess) return GKS_ECUDA;
    if (f32) k_ghosts<float><<<1, 32, 0, st>>>(Wsf, nx, bc[0], bc[1]);
    else k_ghosts<double><<<1, 32, 0, st>>>(Ws, nx, bc[0], bc[1]);
    Stage1DArgs a2{};
    a2.idx = 1.0 / dx;
    if (f32) { a2.srcf = Wsf; a2.base = W; a2.accf = incf; }
    else { a2.src = Ws; a2.acc = Ac; }
    a2.out0 = Wn;
    a2.stage = 2;
    a2.with_sigma = 1;  // checks the new state for rho, p > 0 and finiteness
    if (launch_stage1d(f32, g, a2, hf, tn, ds, st) != cudaSuccess) return GKS_ECUDA;
    k_store<<<(nx + 127) / 128, 128, 0, st>>>(Wn, W_out, nx);
    if (cudaGetLastError() != cudaSuccess) return GKS_ECUDA;

    // read the error word back into host stack memory (no allocation)
    unsigned int err = 0;
    if (cudaMemcpyAsync(&err, &ds->err, sizeof err, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GKS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GKS_ECUDA;
    if (error_word) *error_word = err;
    return err ? GKS_ENONPHYSICAL : GKS_OK;
}
