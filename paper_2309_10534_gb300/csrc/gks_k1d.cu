// gks_k1d.cu -- instantiations and launcher of the fused 1-D stage kernel.
#include "gks_launch.h"

namespace gks {

namespace {
template <typename T, bool NONEQ, bool PRFIX, int REC>
cudaError_t launch_one(const GridDev& g, const Stage1DArgs& a, const HostFlux& hf, const TenoParams& tn,
                       DevState* ds, cudaStream_t st)
{
    constexpr int TN = STAGE1D_TN;
    dim3 grid((g.nx + TN - 1) / TN);
    k1d_stage<T, NONEQ, PRFIX, TN, REC><<<grid, TN + 2, 0, st>>>(g, a, make_flux_params<T>(hf), teno_t<T>(tn), ds);
    return cudaGetLastError();
}

template <typename T, int REC>
cudaError_t dispatch(const GridDev& g, const Stage1DArgs& a, const HostFlux& hf, const TenoParams& tn,
                     DevState* ds, cudaStream_t st)
{
    if (hf.tau_mode == 0) return launch_one<T, false, false, REC>(g, a, hf, tn, ds, st);
    if (hf.prfac != 0.0 && hf.tau_mode == 2) return launch_one<T, true, true, REC>(g, a, hf, tn, ds, st);
    return launch_one<T, true, false, REC>(g, a, hf, tn, ds, st);
}
}  // namespace

cudaError_t launch_stage1d(int fp32, const GridDev& g, const Stage1DArgs& a, const HostFlux& hf,
                           const TenoParams& tn, DevState* ds, cudaStream_t st)
{
    if (tn.recon == 1)
        return fp32 ? dispatch<float, 1>(g, a, hf, tn, ds, st) : dispatch<double, 1>(g, a, hf, tn, ds, st);
    if (tn.recon == 2)
        return fp32 ? dispatch<float, 2>(g, a, hf, tn, ds, st) : dispatch<double, 2>(g, a, hf, tn, ds, st);
    if (tn.recon == 3)
        return fp32 ? dispatch<float, 3>(g, a, hf, tn, ds, st) : dispatch<double, 3>(g, a, hf, tn, ds, st);
    if (tn.recon == REC_TENO_CHAR)
        return fp32 ? dispatch<float, REC_TENO_CHAR>(g, a, hf, tn, ds, st)
                    : dispatch<double, REC_TENO_CHAR>(g, a, hf, tn, ds, st);
    return fp32 ? dispatch<float, 0>(g, a, hf, tn, ds, st) : dispatch<double, 0>(g, a, hf, tn, ds, st);
}

}  // namespace gks
