// Explicit instantiation of the float moment kernel for tiles of any degree (the mixed path's
// persistent launch per batch), chunk plan 1 (kKmaxF32 accumulators per lane).  Its code holds
// every degree's recurrence, so this translation unit is one of the two longest of the build.
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<float, -1, kKmaxF32>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
