// FP32-split instantiations of the fused step (increment storage of phi).
#include "kernels_fused_inst.cuh"
#include "kernels_tm2d.cuh"
#include "kernels_ax3d.cuh"
#include "kernels_tm2d_x2.cuh"

namespace axp {
cudaError_t fused_dispatch_f32(int mode, int set, const fused::Params<float> &P, int nchunks, cudaStream_t s,
                               int *occ)
{
    return fused::dispatch<float, true>(mode, set, P, nchunks, s, occ);
}

cudaError_t tm2d_dispatch_f32(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ, int tx)
{
    return tm2d::launch<float, true>(P, nchunks, s, occ, tx);
}

cudaError_t tm2d_x2_dispatch_f32(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ, int cols)
{
    return tm2d_x2::launch(P, nchunks, s, occ, cols);
}

// FP32-split axion box: the two-cell form on an even-width grid
cudaError_t ax3d_dispatch_f32(const fused::Params<float> &P, int nchunks, cudaStream_t s, int *occ)
{
#ifndef AXP_AX3D_ONE_CELL
    if (P.n[0] % 2 == 0) return ax3d::launch_x2(P, nchunks, s, occ);
#endif
    return ax3d::launch<float, true>(P, nchunks, s, occ);
}
}  // namespace axp
