// kernels_fused_inst.cuh -- per-precision dispatch over the fused-kernel instantiations.
#pragma once

#include "kernels_fused.cuh"

namespace axp {
namespace fused {

// Order-0 component sets with a fused instantiation: none, TM (E0z; B0x, B0y),
// TE (E0x, E0y; B0z) and all.  Bits: E0 xyz in 0-2, B0 xyz in 3-5.
constexpr uint32_t kSets[4] = {0u, (4u) | (3u << 3), (3u) | (4u << 3), 63u};

template <typename T, bool INCR>
cudaError_t dispatch(int mode, int set, const Params<T> &P, int nchunks, cudaStream_t s, int *occ)
{
#define AXP_CASE(M, S, E, B) \
    if (mode == M && set == S) return launch<T, INCR, M, E, B>(P, nchunks, s, occ);
    AXP_CASE(1, 0, 0, 0) AXP_CASE(1, 1, 4, 3) AXP_CASE(1, 2, 3, 4) AXP_CASE(1, 3, 7, 7)
    AXP_CASE(2, 0, 0, 0) AXP_CASE(2, 1, 4, 3) AXP_CASE(2, 2, 3, 4) AXP_CASE(2, 3, 7, 7)
    AXP_CASE(3, 0, 0, 0) AXP_CASE(3, 1, 4, 3) AXP_CASE(3, 2, 3, 4) AXP_CASE(3, 3, 7, 7)
#undef AXP_CASE
    return cudaErrorInvalidValue;
}

}  // namespace fused
}  // namespace axp
