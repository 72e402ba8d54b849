// FP64 instantiations of the fused step.
#include "kernels_fused_inst.cuh"
#include "kernels_tm2d.cuh"
#include "kernels_ax3d.cuh"

namespace axp {
cudaError_t fused_dispatch_f64(int mode, int set, const fused::Params<double> &P, int nchunks, cudaStream_t s,
                               int *occ)
{
    return fused::dispatch<double, false>(mode, set, P, nchunks, s, occ);
}

cudaError_t tm2d_dispatch_f64(const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ, int tx)
{
    return tm2d::launch<double, false>(P, nchunks, s, occ, tx);
}

cudaError_t tm2d_list_dispatch_f64(const fused::Params<double> &P, const int4 *items, int nblocks, int per_block,
                                   cudaStream_t s, int *occ, int tx)
{
    return tm2d::launch_list<double, false>(P, items, nblocks, per_block, s, occ, tx);
}

cudaError_t ax3d_dispatch_f64(const fused::Params<double> &P, int nchunks, cudaStream_t s, int *occ)
{
    return ax3d::launch<double, false>(P, nchunks, s, occ);
}
}  // namespace axp
