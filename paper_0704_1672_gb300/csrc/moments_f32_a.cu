// Explicit instantiations of the moment kernels: float, Lmax 0..13.
// (Split across translation units so that they compile in parallel.)
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<float, 0>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 1>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 2>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 3>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 4>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 5>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 6>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 7>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 8>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 9>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 10>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 11>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 12>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<float, 13>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
