// FP32-split instantiations of the fused step (increment storage of phi).
#include "kernels_fused_inst.cuh"

namespace axp {
cudaError_t fused_dispatch_f32(int mode, int set, const fused::Params<float> &P, int nchunks, cudaStream_t s,
                               int *occ)
{
    return fused::dispatch<float, true>(mode, set, P, nchunks, s, occ);
}
}  // namespace axp
