// The pass over each system's atoms before the moment pass (step a1 and the mixed path's
// low-degree sums), for any mix of system sizes, in two launches:
//
//   pass 1 (systems without a given centre): the centroid (Section II: the centres may be any
//           point; the centroid of the positions by default);
//   pass 2: the radius a = max |x - c| (exact in double) and, for the mixed path, the
//           low-degree sums S = sum q, P_k = sum q d_k, T_kl = sum q d_k d_l (d = x - c) from
//           which k_finalize forms Q_lm, l <= 2, of every moment job of the system
//           (Eq. (multipole) in Cartesian form).
//
// Each system is cut into warp tiles whose size depends on its own atom count only (so a
// system's results do not depend on the batch it is in); one warp per tile, all systems' tiles
// in one launch, so small and large systems alike spread over the GPU.  Per-atom arithmetic is
// float for float records: error-free two-sums for the centroid, float-float (two-sum and
// fma-based two-product) for the low-degree sums, and a float filter for the radius that sends
// only the atoms within a relative 4e-6 of a lane's running maximum to an exact double
// recomputation.  Tile partials are doubles; the last tile of a system to finish (a ticket)
// reduces them in tile order, so every result is deterministic.
#include <cuda_runtime.h>

#include "tcm_internal.h"

namespace tcm {

namespace {

struct FF {  // unevaluated sum h + l of two floats
  float h, l;
};

// s + e += x: Knuth's two-sum of s and x.h; its rounding error, x.l and the running error go to e.
__device__ __forceinline__ void ff_acc(float& s, float& e, FF x) {
  const float t = s + x.h;
  const float bb = t - s;
  e += ((s - (t - bb)) + (x.h - bb)) + x.l;
  s = t;
}

// Product of two FF values to about 2^-46 relative: the exact product of the high parts (fma
// error term) plus the two cross terms.
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return FF{p, e};
}

// x - (hi + lo) as an FF pair: exact two-sum of x and -hi, then -lo into the error term.
__device__ __forceinline__ FF ff_sub_split(float x, float hi, float lo) {
  const float s = x - hi;
  const float bb = s - x;
  const float e = (x - (s - bb)) + (-hi - bb);
  return FF{s, e - lo};
}

__device__ __forceinline__ void ff_warp_sum(float& s, float& e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
    ff_acc(s, e, FF{s2, e2});
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Lane l adds rows l, l + 32, ... of n, then the lanes' sums are added in a fixed tree: the same
// result for the same rows in every run.  Rows are read through L2 (written by other CTAs).
__device__ __forceinline__ double ordered_sum(const double* p, int n, int stride, int lane) {
  double t = 0.0;
  for (int r = lane; r < n; r += 32) t += __ldcg(p + (long long)r * stride);
  return warp_sum_d(t);
}

constexpr int kSysWarps = kSysThreads / 32;

// Last tile of a job to finish (after its partial rows are written and fenced): lane 0 takes the
// ticket; the result is broadcast to the warp.  The last one resets the ticket for the next use.
__device__ __forceinline__ bool last_tile(int* ticket, int n_tiles, int lane) {
  __threadfence();  // every lane's partial-row writes, before the ticket
  __syncwarp();
  int last = 0;
  if (lane == 0) {
    last = atomicAdd(ticket, 1) == n_tiles - 1;
    if (last) *ticket = 0;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) __threadfence();
  return last;
}

__global__ void __launch_bounds__(kSysThreads) k_sys_centroid(const SysJob* __restrict__ jobs,
                                                              const SysTile* __restrict__ tiles, int n_tiles,
                                                              double* __restrict__ part, int* __restrict__ tickets,
                                                              SysGeom* __restrict__ geoms) {
  const int w = blockIdx.x * kSysWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n_tiles) return;
  const SysTile tl = tiles[w];
  const SysJob j = jobs[tl.job];
  const long long i0 = (long long)tl.t * j.atoms_per_tile;
  const long long i1 = min(j.n, i0 + (long long)j.atoms_per_tile);
  double sum[3];
  if (j.dtype == TCM_F32) {
    float s[3] = {0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f};
    for (long long i = i0 + lane; i < i1; i += 32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(j.xyzq) + i);
      ff_acc(s[0], e[0], FF{v.x, 0.f});
      ff_acc(s[1], e[1], FF{v.y, 0.f});
      ff_acc(s[2], e[2], FF{v.z, 0.f});
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ff_warp_sum(s[k], e[k]);
      sum[k] = (double)s[k] + (double)e[k];
    }
  } else {
    double s[3] = {0.0, 0.0, 0.0};
    for (long long i = i0 + lane; i < i1; i += 32) {
      const double2 a = __ldg(reinterpret_cast<const double2*>(j.xyzq) + 2 * i);
      const double2 b = __ldg(reinterpret_cast<const double2*>(j.xyzq) + 2 * i + 1);
      s[0] += a.x;
      s[1] += a.y;
      s[2] += b.x;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sum[k] = warp_sum_d(s[k]);
  }
  double* row = part + (long long)(j.tile_base + tl.t) * kSysPart;
  if (lane < 3) row[lane] = lane == 0 ? sum[0] : (lane == 1 ? sum[1] : sum[2]);
  if (!last_tile(&tickets[2 * tl.job], j.n_tiles, lane)) return;
  const double* p0 = part + (long long)j.tile_base * kSysPart;
  const double inv = j.n > 0 ? 1.0 / (double)j.n : 0.0;
  const double cx = ordered_sum(p0, j.n_tiles, kSysPart, lane) * inv;
  const double cy = ordered_sum(p0 + 1, j.n_tiles, kSysPart, lane) * inv;
  const double cz = ordered_sum(p0 + 2, j.n_tiles, kSysPart, lane) * inv;
  if (lane == 0) {
    geoms[j.geom].c[0] = cx;
    geoms[j.geom].c[1] = cy;
    geoms[j.geom].c[2] = cz;
  }
}

__global__ void __launch_bounds__(kSysThreads) k_sys_radius_low(const SysJob* __restrict__ jobs,
                                                                const SysTile* __restrict__ tiles, int n_tiles,
                                                                double* __restrict__ part, int* __restrict__ tickets,
                                                                SysGeom* __restrict__ geoms) {
  const int w = blockIdx.x * kSysWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n_tiles) return;
  const SysTile tl = tiles[w];
  const SysJob j = jobs[tl.job];
  pdl_wait();  // the centroids of pass 1 are complete
  const SysGeom g = geoms[j.geom];
  const long long i0 = (long long)tl.t * j.atoms_per_tile;
  const long long i1 = min(j.n, i0 + (long long)j.atoms_per_tile);
  double rmax = 0.0;  // exact max |x - c|^2 of this lane's atoms
  float s[kLowSums], e[kLowSums];
#pragma unroll
  for (int k = 0; k < kLowSums; ++k) s[k] = e[k] = 0.f;
  if (j.dtype == TCM_F32) {
    float chi[3], clo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      chi[k] = (float)g.c[k];
      clo[k] = (float)(g.c[k] - (double)chi[k]);
    }
    float thr = 0.f;  // lane's running float maximum, lowered by a relative 4e-6
    for (long long i = i0 + lane; i < i1; i += 32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(j.xyzq) + i);
      FF d[3];
      d[0] = ff_sub_split(v.x, chi[0], clo[0]);
      d[1] = ff_sub_split(v.y, chi[1], clo[1]);
      d[2] = ff_sub_split(v.z, chi[2], clo[2]);
      // |x - c|^2 in float (within about 4e-7 of the exact value): only atoms near the lane's
      // running maximum are recomputed exactly
      const float r2f = __fmaf_rn(d[0].h, d[0].h, __fmaf_rn(d[1].h, d[1].h, d[2].h * d[2].h));
      if (r2f >= thr) {
        const double dx = (double)v.x - g.c[0], dy = (double)v.y - g.c[1], dz = (double)v.z - g.c[2];
        rmax = fmax(rmax, dx * dx + dy * dy + dz * dz);
        thr = fmaxf(thr, r2f * (1.0f - 4e-6f));
      }
      if (j.need_low) {
        const FF q{v.w, 0.f};
        ff_acc(s[0], e[0], q);
        const FF qd0 = ff_mul(q, d[0]), qd1 = ff_mul(q, d[1]), qd2 = ff_mul(q, d[2]);
        ff_acc(s[1], e[1], qd0);
        ff_acc(s[2], e[2], qd1);
        ff_acc(s[3], e[3], qd2);
        ff_acc(s[4], e[4], ff_mul(qd0, d[0]));
        ff_acc(s[5], e[5], ff_mul(qd0, d[1]));
        ff_acc(s[6], e[6], ff_mul(qd0, d[2]));
        ff_acc(s[7], e[7], ff_mul(qd1, d[1]));
        ff_acc(s[8], e[8], ff_mul(qd1, d[2]));
        ff_acc(s[9], e[9], ff_mul(qd2, d[2]));
      }
    }
  } else {
    for (long long i = i0 + lane; i < i1; i += 32) {
      const double2 a = __ldg(reinterpret_cast<const double2*>(j.xyzq) + 2 * i);
      const double2 b = __ldg(reinterpret_cast<const double2*>(j.xyzq) + 2 * i + 1);
      const double dd[4] = {a.x - g.c[0], a.y - g.c[1], b.x - g.c[2], b.y};
      rmax = fmax(rmax, dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
      if (j.need_low) {
        FF t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float h = (float)dd[k];
          t[k] = FF{h, (float)(dd[k] - (double)h)};
        }
        const FF q = t[3];
        ff_acc(s[0], e[0], q);
        const FF qd0 = ff_mul(q, t[0]), qd1 = ff_mul(q, t[1]), qd2 = ff_mul(q, t[2]);
        ff_acc(s[1], e[1], qd0);
        ff_acc(s[2], e[2], qd1);
        ff_acc(s[3], e[3], qd2);
        ff_acc(s[4], e[4], ff_mul(qd0, t[0]));
        ff_acc(s[5], e[5], ff_mul(qd0, t[1]));
        ff_acc(s[6], e[6], ff_mul(qd0, t[2]));
        ff_acc(s[7], e[7], ff_mul(qd1, t[1]));
        ff_acc(s[8], e[8], ff_mul(qd1, t[2]));
        ff_acc(s[9], e[9], ff_mul(qd2, t[2]));
      }
    }
  }
  rmax = warp_max_d(rmax);
  double* row = part + (long long)(j.tile_base + tl.t) * kSysPart;
  if (j.need_low) {
#pragma unroll
    for (int k = 0; k < kLowSums; ++k) ff_warp_sum(s[k], e[k]);
    if (lane < kLowSums) {
      float sv = 0.f, ev = 0.f;
#pragma unroll
      for (int k = 0; k < kLowSums; ++k)
        if (lane == k) {
          sv = s[k];
          ev = e[k];
        }
      row[kSysPartLow + lane] = (double)sv + (double)ev;
    }
  }
  if (lane == 0) row[kSysPartR2] = rmax;
  if (!j.need_radius || !last_tile(&tickets[2 * tl.job + 1], j.n_tiles, lane)) return;
  double m = 0.0;
  const double* p0 = part + (long long)j.tile_base * kSysPart + kSysPartR2;
  for (int r = lane; r < j.n_tiles; r += 32) m = fmax(m, __ldcg(p0 + (long long)r * kSysPart));
  m = warp_max_d(m);
  if (lane == 0) geoms[j.geom].a = sqrt(m);
}

}  // namespace

int sys_tile_atoms(long long n) {
  // about 64 tiles for a system, between 256 and 2,048 atoms (8 to 64 per lane)
  long long t = 256;
  while (t < 2048 && t * 64 < n) t *= 2;
  return (int)t;
}

int launch_sys(const SysJob* jobs, const SysTile* t1, int n1, const SysTile* t2, int n2, double* part, int* tickets,
               SysGeom* geoms, cudaStream_t s) {
  if (n1 > 0) {
    k_sys_centroid<<<(n1 + kSysWarps - 1) / kSysWarps, kSysThreads, 0, s>>>(jobs, t1, n1, part, tickets, geoms);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
  }
  if (n2 > 0 && launch_pdl(k_sys_radius_low, dim3((n2 + kSysWarps - 1) / kSysWarps), dim3(kSysThreads), 0, s, jobs,
                           t2, n2, part, tickets, geoms) != cudaSuccess)
    return -1;
  return 0;
}

int sys_launches(int n1, int n2) { return (n1 > 0 ? 1 : 0) + (n2 > 0 ? 1 : 0); }

}  // namespace tcm
