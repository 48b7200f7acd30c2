// Explicit instantiations of the moment kernels: double, Lmax 0..13.
// (Split across translation units so that they compile in parallel.)
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<double, 0, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 1, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 2, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 3, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 4, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 5, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 6, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 7, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 8, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 9, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 10, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 11, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 12, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 13, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
