// Runtime dispatch from (precision, Lmax) to the explicitly instantiated moment kernels.
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <utility>
#include <vector>

#include "tcm_internal.h"

namespace tcm {

// Defined (and explicitly instantiated) in moments_kernel.cuh / moments_*.cu.
template <typename T, int L, int KM>
int launch_moments_t(const MomJob* jobs, const MomTile* tiles, int n_tiles, int* counter, const SysGeom* geoms,
                     double* partials, int grid, cudaStream_t s);

namespace {

using LaunchFn = int (*)(const MomJob*, const MomTile*, int, int*, const SysGeom*, double*, int, cudaStream_t);

template <typename T, int... Ls>
constexpr auto make_table(std::integer_sequence<int, Ls...>) {
  return std::array<LaunchFn, sizeof...(Ls)>{{&launch_moments_t<T, Ls, kKmaxF64>...}};
}

const auto kF64 = make_table<double>(std::make_integer_sequence<int, kLmaxMax + 1>{});

}  // namespace

namespace {
// The chunk plans, tabulated once (plan_nch and plan_m0 are loops meant for compile time; the
// host planning of a batch asks for them per job and per group).
struct ChunkTables {
  int nch[kNumPlans][kLmaxMax + 1];
  int m0[kNumPlans][kLmaxMax + 1][kLmaxMax + 2];
  double cost[kNumPlans][kLmaxMax + 1][kLmaxMax + 1];
  ChunkTables() {
    for (int pi = 0; pi < kNumPlans; ++pi) {
      const int kmax = plan_kmax(pi);
      for (int L = 0; L <= kLmaxMax; ++L) {
        nch[pi][L] = plan_nch(L, kmax);
        for (int c = 0; c <= nch[pi][L]; ++c) m0[pi][L][c] = plan_m0(L, kmax, nch[pi][L], c);
        // relative cost of one atom of a chunk: its accumulators, the seed power u^m0 and the
        // per-atom set-up
        for (int c = 0; c < nch[pi][L]; ++c)
          cost[pi][L][c] = 1.25 * chunk_off(L, m0[pi][L][c], m0[pi][L][c + 1]) + 4.0 * m0[pi][L][c] + 30.0;
      }
    }
  }
};
const ChunkTables& chunk_tables() {
  static const ChunkTables t;
  return t;
}
}  // namespace

int moments_nchunks(int plan, int L) { return chunk_tables().nch[plan][L]; }

int moments_chunk_m0(int plan, int L, int chunk) { return chunk_tables().m0[plan][L][chunk]; }

const double* moments_chunk_costs(int plan, int L) { return chunk_tables().cost[plan][L]; }

void finalize_tables(std::vector<int>& imap_off, std::vector<int>& imap, std::vector<double>& fmap) {
  const int N = kLmaxMax + 1;
  std::vector<double> ftab;
  std::vector<long double> fact(2 * N + 2);
  fact[0] = 1.0L;
  for (size_t k = 1; k < fact.size(); ++k) fact[k] = fact[k - 1] * (long double)k;
  ftab.assign(N * N, 0.0);
  for (int m = 0; m < N; ++m) {
    // s_lm: normalisation of the kernels' G_lm (tcm_internal.h): s_mm = (2m-1)!!,
    // s_m+1,m = (2m+1) s_mm, s_l+1,m = (l+m) s_l-1,m / (l-m+1)
    long double s_prev = 0.0L, s = 1.0L;
    for (int k = 1; k < 2 * m; k += 2) s *= (long double)k;
    for (int l = m; l < N; ++l) {
      if (l == m + 1) {
        s_prev = s;
        s = (long double)(2 * m + 1) * s;
      } else if (l > m + 1) {
        const long double sn = (long double)(l - 1 + m) * s_prev / (long double)(l - m);
        s_prev = s;
        s = sn;
      }
      // (-1)^m of the Condon-Shortley phase times sigma_{l-m} of the kernels' H variables
      const long double sgn = ((m & 1) ? -1.0L : 1.0L) * (((l - m) & 2) ? -1.0L : 1.0L);
      ftab[l * N + m] = (double)(sgn * std::sqrt(fact[l - m] / fact[l + m]) * s);
    }
  }
  imap_off.assign(kNumPlans * (N + 1), 0);
  imap.clear();
  for (int pi = 0; pi < kNumPlans; ++pi) {
    const int kmax = plan_kmax(pi);
    for (int L = 0; L < N; ++L) {
      const int nch = plan_nch(L, kmax);
      const size_t base = imap.size();
      imap_off[pi * (N + 1) + L] = (int)base;
      imap.resize(base + (size_t)nch * kmax, -1);
      for (int ch = 0; ch < nch; ++ch) {
        const int m0 = plan_m0(L, kmax, nch, ch), m1 = plan_m0(L, kmax, nch, ch + 1);
        for (int m = m0; m < m1; ++m)
          for (int l = m; l <= L; ++l) {
            if (m == 0) {
              imap[base + ch * kmax + acc_slot(L, m0, m1, l, 0, 0)] = l * l;
            } else {
              imap[base + ch * kmax + acc_slot(L, m0, m1, l, m, 0)] = l * l + 2 * m - 1;
              imap[base + ch * kmax + acc_slot(L, m0, m1, l, m, 1)] = l * l + 2 * m;
            }
          }
      }
    }
    imap_off[pi * (N + 1) + N] = (int)imap.size();
  }
  fmap.assign(imap.size(), 0.0);
  for (size_t q = 0; q < imap.size(); ++q) {
    const int p = imap[q];
    if (p < 0) continue;
    int l = 0;
    while ((l + 1) * (l + 1) <= p) ++l;
    fmap[q] = ftab[l * N + ((p - l * l + 1) >> 1)];
  }
}

int launch_moments(int plan, int L, const MomJob* jobs, const MomTile* tiles, int n_tiles, int* counter,
                   const SysGeom* geoms, double* partials, int grid, cudaStream_t s) {
  if (n_tiles <= 0) return n_tiles == 0 ? 0 : -1;
  switch (plan) {  // the float kernels take tiles of any degree
    case 1: return launch_moments_t<float, -1, kKmaxF32>(jobs, tiles, n_tiles, counter, geoms, partials, grid, s);
    case 2: return launch_moments_t<float, -1, kKmaxF32Small>(jobs, tiles, n_tiles, counter, geoms, partials, grid, s);
    case 0: return L < 0 || L > kLmaxMax ? -1 : kF64[L](jobs, tiles, n_tiles, counter, geoms, partials, grid, s);
    default: return -1;
  }
}

namespace {
__global__ void __launch_bounds__(256) k_expand_tiles(const MomGroup* __restrict__ groups, int n_groups,
                                                      const MomJob* __restrict__ jobs, MomTile* __restrict__ tiles,
                                                      const SysJob* __restrict__ sjobs, int n_sjobs,
                                                      SysTile* __restrict__ t1, SysTile* __restrict__ t2) {
  const int g = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g < n_groups) {
    const MomGroup gr = groups[g];
    const MomJob& j = jobs[gr.job];
    const int row = j.tile_base + gr.chunk * j.tiles_per_chunk;
    for (int t = lane; t < gr.n; t += 32) tiles[gr.first + t] = MomTile{gr.job, gr.chunk, t, row + t};
  } else if (g - n_groups < n_sjobs) {
    const int ji = g - n_groups;
    const SysJob sj = sjobs[ji];
    for (int t = lane; t < sj.n_tiles; t += 32) {
      if (sj.first1 >= 0) t1[sj.first1 + t] = SysTile{ji, t};
      if (sj.first2 >= 0) t2[sj.first2 + t] = SysTile{ji, t};
    }
  }
}
}  // namespace

int launch_expand_tiles(const MomGroup* groups, int n_groups, const MomJob* jobs, MomTile* tiles, const SysJob* sjobs,
                        int n_sjobs, SysTile* t1, SysTile* t2, cudaStream_t s) {
  const int n = n_groups + n_sjobs;
  if (n <= 0) return 0;
  k_expand_tiles<<<(n + 7) / 8, 256, 0, s>>>(groups, n_groups, jobs, tiles, sjobs, n_sjobs, t1, t2);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tcm
