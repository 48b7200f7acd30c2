// Explicit instantiation of the float moment kernel for tiles of any degree, chunk plan 2
// (kKmaxF32Small accumulators per lane: more column chunks, fewer registers, 3 CTAs per SM).
// A separate translation unit so that the build compiles both budgets in parallel.
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<float, -1, kKmaxF32Small>(const MomJob*, const MomTile*, int, int*, const SysGeom*,
                                                        double*, int, cudaStream_t);
}  // namespace tcm
