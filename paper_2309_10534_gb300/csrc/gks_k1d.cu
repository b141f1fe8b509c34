// gks_k1d.cu -- instantiations and launcher of the fused 1-D stage kernel.
#include "gks_launch.h"

namespace gks {

namespace {
template <typename T, bool NONEQ, bool PRFIX>
cudaError_t launch_one(const GridDev& g, const Stage1DArgs& a, const HostFlux& hf, const TenoParams& tn,
                       DevState* ds, cudaStream_t st)
{
    constexpr int TN = STAGE1D_TN;
    dim3 grid((g.nx + TN - 1) / TN);
    k1d_stage<T, NONEQ, PRFIX, TN><<<grid, TN + 1, 0, st>>>(g, a, make_flux_params<T>(hf), teno_t<T>(tn), ds);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const GridDev& g, const Stage1DArgs& a, const HostFlux& hf, const TenoParams& tn,
                     DevState* ds, cudaStream_t st)
{
    if (hf.tau_mode == 0) return launch_one<T, false, false>(g, a, hf, tn, ds, st);
    if (hf.prfac != 0.0 && hf.tau_mode == 2) return launch_one<T, true, true>(g, a, hf, tn, ds, st);
    return launch_one<T, true, false>(g, a, hf, tn, ds, st);
}
}  // namespace

cudaError_t launch_stage1d(int fp32, const GridDev& g, const Stage1DArgs& a, const HostFlux& hf,
                           const TenoParams& tn, DevState* ds, cudaStream_t st)
{
    return fp32 ? dispatch<float>(g, a, hf, tn, ds, st) : dispatch<double>(g, a, hf, tn, ds, st);
}

}  // namespace gks
