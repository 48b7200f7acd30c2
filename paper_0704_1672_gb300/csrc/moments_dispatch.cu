// Runtime dispatch from (precision, Lmax) to the explicitly instantiated moment kernels.
#include <cuda_runtime.h>

#include <array>
#include <utility>

#include "tcm_internal.h"

namespace tcm {

// Defined (and explicitly instantiated) in moments_kernel.cuh / moments_*.cu.
template <typename T, int L>
int launch_moments_t(const MomJob* jobs, const MomTile* tiles, int n_tiles, int* counter, const SysGeom* geoms,
                     double* partials, int grid, cudaStream_t s);

namespace {

using LaunchFn = int (*)(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);

template <typename T, int... Ls>
constexpr auto make_table(std::integer_sequence<int, Ls...>) {
  return std::array<LaunchFn, sizeof...(Ls)>{{&launch_moments_t<T, Ls>...}};
}

const auto kF32 = make_table<float>(std::make_integer_sequence<int, kLmaxMax + 1>{});
const auto kF64 = make_table<double>(std::make_integer_sequence<int, kLmaxMax + 1>{});

constexpr int stride_of(int precision) { return precision == TCM_FP64 ? 34 : 36; }
constexpr int size_of(int precision) { return precision == TCM_FP64 ? 8 : 4; }

}  // namespace

int moments_kmax(int precision) { return precision == TCM_FP64 ? kKmaxF64 : kKmaxF32; }

int moments_nchunks(int precision, int L) { return plan_nch(L, moments_kmax(precision)); }

int moments_smem_bytes(int precision, int L) {
  const int kmax = moments_kmax(precision);
  const int nch = plan_nch(L, kmax);
  int mx = 0;
  for (int c = 0; c < nch; ++c) {
    const int n = chunk_off(L, plan_m0(L, kmax, nch, c), plan_m0(L, kmax, nch, c + 1));
    mx = n > mx ? n : mx;
  }
  return (kThreads / 32) * mx * stride_of(precision) * size_of(precision);
}

int launch_moments(int precision, int L, const MomJob* jobs, const MomTile* tiles, int n_tiles, int* counter,
                   const SysGeom* geoms, double* partials, int grid, cudaStream_t s) {
  if (L < 0 || L > kLmaxMax || n_tiles <= 0) return n_tiles == 0 ? 0 : -1;
  const LaunchFn f = precision == TCM_FP64 ? kF64[L] : kF32[L];
  return f(jobs, tiles, n_tiles, counter, geoms, partials, grid, s);
}

}  // namespace tcm
