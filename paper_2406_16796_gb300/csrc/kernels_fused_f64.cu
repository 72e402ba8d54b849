// FP64 instantiations of the fused step.
#include "kernels_fused_inst.cuh"

namespace axp {
cudaError_t fused_dispatch_f64(int mode, int set, const fused::Params<double> &P, int nchunks, cudaStream_t s,
                               int *occ)
{
    return fused::dispatch<double, false>(mode, set, P, nchunks, s, occ);
}
}  // namespace axp
