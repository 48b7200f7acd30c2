// Explicit instantiations of the moment kernels: float, Lmax 14..19.
// (Split across translation units so that they compile in parallel.)
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<float, 14>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 15>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 16>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 17>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 18>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 19>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
