// Explicit instantiations of the moment kernels: double, Lmax 20..22.
// (Split across translation units so that they compile in parallel.)
#include "moments_kernel.cuh"

namespace tcm {
template int launch_moments_t<double, 20, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 21, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
template int launch_moments_t<double, 22, kKmaxF64>(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);
}  // namespace tcm
