// Explicit instantiations of the moment kernels: double, Lmax 0..13.
// (Split across translation units so that they compile in parallel.)
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<double, 0>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 1>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 2>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 3>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 4>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 5>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 6>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 7>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 8>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 9>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 10>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 11>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 12>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 13>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
