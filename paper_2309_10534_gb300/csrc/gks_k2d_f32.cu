// gks_k2d_f32.cu -- instantiations and launcher of the 2-D sweep in float.
#include "gks_launch.h"

namespace gks {

namespace {
template <bool NONEQ, bool PRFIX, int REC>
cudaError_t launch_one(const GridDev& g, const SweepArgs& a, const FluxParams<float>& fp, const TenoParams& tn,
                       const TenoParams& tt, DevState* ds, cudaStream_t st)
{
    constexpr int TN = SWEEP_TN, TT = SWEEP_TT32;
    auto kern = k2d_sweep<float, NONEQ, PRFIX, TN, TT, REC>;
    const size_t smem = sizeof(SweepSmem<float, TN, TT, rec_conventional(REC)>);
    dim3 grid((a.nn + TN - 1) / TN, (a.nt + TT - 1) / TT);
    kern<<<grid, TT * (TN + 1), smem, st>>>(g, a, fp, teno_t<float>(tn), teno_t<float>(tt), ds);
    return cudaGetLastError();
}
template <bool NONEQ, bool PRFIX, int REC>
cudaError_t set_smem()
{
    return cudaFuncSetAttribute(k2d_sweep<float, NONEQ, PRFIX, SWEEP_TN, SWEEP_TT32, REC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(SweepSmem<float, SWEEP_TN, SWEEP_TT32, rec_conventional(REC)>));
}
template <int REC>
cudaError_t set_smem_all()
{
    cudaError_t e = set_smem<false, false, REC>();
    if (e == cudaSuccess) e = set_smem<true, false, REC>();
    if (e == cudaSuccess) e = set_smem<true, true, REC>();
    return e;
}
template <int REC>
cudaError_t launch_rec(const GridDev& g, const SweepArgs& a, const HostFlux& hf, const TenoParams& tn,
                       const TenoParams& tt, DevState* ds, cudaStream_t st)
{
    const FluxParams<float> fp = make_flux_params<float>(hf);
    if (hf.tau_mode == 0) return launch_one<false, false, REC>(g, a, fp, tn, tt, ds, st);
    if (hf.prfac != 0.0 && hf.tau_mode == 2) return launch_one<true, true, REC>(g, a, fp, tn, tt, ds, st);
    return launch_one<true, false, REC>(g, a, fp, tn, tt, ds, st);
}
}  // namespace

cudaError_t prepare_sweep_f32()
{
    cudaError_t e = set_smem_all<0>();
    if (e == cudaSuccess) e = set_smem_all<1>();
    if (e == cudaSuccess) e = set_smem_all<2>();
    if (e == cudaSuccess) e = set_smem_all<3>();
    if (e == cudaSuccess) e = set_smem_all<REC_TENO_CHAR>();
    return e;
}

cudaError_t launch_sweep_f32(const GridDev& g, const SweepArgs& a, const HostFlux& hf, const TenoParams& tn,
                             const TenoParams& tt, DevState* ds, cudaStream_t st)
{
    switch (tn.recon) {
    case 1: return launch_rec<1>(g, a, hf, tn, tt, ds, st);
    case 2: return launch_rec<2>(g, a, hf, tn, tt, ds, st);
    case 3: return launch_rec<3>(g, a, hf, tn, tt, ds, st);
    case REC_TENO_CHAR: return launch_rec<REC_TENO_CHAR>(g, a, hf, tn, tt, ds, st);
    default: return launch_rec<0>(g, a, hf, tn, tt, ds, st);
    }
}

}  // namespace gks
