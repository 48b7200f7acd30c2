// Explicit instantiation of the float moment kernel for tiles of any degree (the mixed path's
// single persistent launch per batch).  Its code holds every degree's recurrence, so this
// translation unit is the longest of the build.
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<float, -1>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
