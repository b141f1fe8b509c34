// gks_launch.h -- host-side launchers of the stage kernels, one translation
// unit per precision so the heavy instantiations compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gks.h"
#include "gks_kernels.cuh"

namespace gks {

// tile of the 2-D sweep: TN cells along the face normal (TN + 1 faces) x TT
// rows, one thread per (face, row) pair; float32 blocks hold 64 registers per
// thread (1024 / threads blocks per SM)
constexpr int SWEEP_TN = 31;
constexpr int SWEEP_TT32 = 16;
constexpr int SWEEP_TT64 = 8;
// cells per block of the 1-D stage (TN + 2 = 128 threads: one per
// reconstructed cell, face and updated cell)
constexpr int STAGE1D_TN = 126;

struct HostFlux {
    double gamma, K, ntot, c1, c2, mu, prfac;
    int tau_mode;
    int merge = 0;
};

cudaError_t launch_sweep_f32(const GridDev& g, const SweepArgs& a, const HostFlux& hf, const TenoParams& tn,
                             const TenoParams& tt, DevState* ds, cudaStream_t st);
cudaError_t launch_sweep_f64(const GridDev& g, const SweepArgs& a, const HostFlux& hf, const TenoParams& tn,
                             const TenoParams& tt, DevState* ds, cudaStream_t st);
// raise the dynamic shared-memory limit of every 2-D sweep instantiation
// (current device); call once before the first launch
cudaError_t prepare_sweep_f32();
cudaError_t prepare_sweep_f64();
cudaError_t launch_stage1d(int fp32, const GridDev& g, const Stage1DArgs& a, const HostFlux& hf,
                           const TenoParams& tn, DevState* ds, cudaStream_t st);

// Range checks of a gks_scheme shared by every entry point that takes one
// (gks_set_scheme, gks_batch_set_scheme, gks_step1d_noalloc).  Returns
// nullptr when the scheme is valid, else the reason, with *code set to the
// status to return.  The CFL number is checked only where it is used
// (check_cfl != 0).
const char* scheme_problem(const gks_scheme* s, int check_cfl, gks_status* code);

template <typename T>
inline FluxParams<T> make_flux_params(const HostFlux& h)
{
    FluxParams<T> p;
    p.gm1 = (T)(h.gamma - 1.0);
    p.K = (T)h.K;
    p.ntot = (T)h.ntot;
    p.inv_ntot = (T)(1.0 / h.ntot);
    p.dt = (T)0;
    p.c1 = (T)h.c1;
    p.c2 = (T)h.c2;
    p.mu = (T)h.mu;
    p.prfac = (T)h.prfac;
    p.tau_mode = h.tau_mode;
    p.merge = h.merge;
    return p;
}

}  // namespace gks
