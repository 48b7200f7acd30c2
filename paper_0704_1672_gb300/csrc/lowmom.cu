// Low-degree sums of the mixed-precision path (Eq. (multipole) for l <= 2, in Cartesian form).
//
// The float moment kernels give every term q rho^l G_lm a relative rounding error of a few
// 2^-24: the centred, rotated and scaled coordinates are rounded to float, and each lane sums
// its atoms in float.  The lowest degrees carry most of a separated pair's energy, and for
// net-zero systems the (l1, l2) blocks of Eq. (Formula) cancel, so those few 2^-24 reach the
// energy magnified by sum |U_l1l2| / |E|.  This kernel recomputes degrees 0..2 from the
// Cartesian sums about the system's centre (no rotation, no scaling),
//   S = sum q,  P_k = sum q d_k,  T_kl = sum q d_k d_l,     d = x - c,
// in float-float arithmetic (error-free two-sum and fma-based two-product), about 150 float
// instructions per atom.  Degree l <= 2 of Q_lm is a linear function of (S, P, T) after the
// rotation P' = R P, T' = R T R^T, which k_finalize applies per moment job in double; one pass
// per system serves all of its orientations.
//
// Float input: x is exact in float and c = c_hi + c_lo, so d = (x - c_hi) - c_lo is formed
// exactly as a float-float pair by a two-sum.  Double input: d is formed in double (one
// subtraction per coordinate) and split into float hi and lo parts, as is the charge.
#include <cuda_runtime.h>

#include "tcm_internal.h"

namespace tcm {

namespace {

struct FF {  // unevaluated sum h + l of two floats
  float h, l;
};

// s + e += x (an FF value): Knuth's two-sum of s and x.h; the rounding error, x.l and the
// running error term go to e.
__device__ __forceinline__ void ff_acc(float& s, float& e, FF x) {
  const float t = s + x.h;
  const float bb = t - s;
  e += ((s - (t - bb)) + (x.h - bb)) + x.l;
  s = t;
}

// Product of two FF values to about 2^-46 relative: the exact product of the high parts
// (fma error term) plus the two cross terms.
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return FF{p, e};
}

// Exact difference x - (hi + lo) as an FF pair (two-sum of x and -hi, then -lo into the error).
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

__global__ void __launch_bounds__(kLowThreads) k_lowmom(const LowJob* __restrict__ jobs, const LowTile* __restrict__ tiles,
                                                        int n_tiles, const SysGeom* __restrict__ geoms,
                                                        double* __restrict__ lowpart) {
  const int w = blockIdx.x * (kLowThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n_tiles) return;
  const LowTile tl = tiles[w];
  const LowJob j = jobs[tl.job];
  pdl_wait();  // the centres of the launch before are complete
  const SysGeom g = geoms[j.geom];
  float chi[3], clo[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    chi[k] = (float)g.c[k];
    clo[k] = (float)(g.c[k] - (double)chi[k]);
  }
  float s[kLowSums], e[kLowSums];
#pragma unroll
  for (int k = 0; k < kLowSums; ++k) s[k] = e[k] = 0.f;
  const long long i0 = (long long)tl.t * kLowTileAtoms;
  const long long i1 = min(j.n, i0 + (long long)kLowTileAtoms);
  for (long long i = i0 + lane; i < i1; i += 32) {
    FF d[3], q;
    if (j.dtype == TCM_F32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(j.xyzq) + i);
      d[0] = ff_sub_split(v.x, chi[0], clo[0]);
      d[1] = ff_sub_split(v.y, chi[1], clo[1]);
      d[2] = ff_sub_split(v.z, chi[2], clo[2]);
      q = FF{v.w, 0.f};
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(j.xyzq) + 2 * i);
      const double2 b = __ldg(reinterpret_cast<const double2*>(j.xyzq) + 2 * i + 1);
      const double dd[4] = {a.x - g.c[0], a.y - g.c[1], b.x - g.c[2], b.y};
      FF t[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float h = (float)dd[k];
        t[k] = FF{h, (float)(dd[k] - (double)h)};
      }
      d[0] = t[0];
      d[1] = t[1];
      d[2] = t[2];
      q = t[3];
    }
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
    lowpart[(long long)(j.tile_base + tl.t) * kLowSums + lane] = (double)sv + (double)ev;
  }
}

}  // namespace

int launch_lowmom(const LowJob* ljobs, const LowTile* ltiles, int n_ltiles, const SysGeom* geoms, double* lowpart,
                  cudaStream_t s) {
  if (n_ltiles <= 0) return 0;
  const int grid = (n_ltiles + kLowThreads / 32 - 1) / (kLowThreads / 32);
  return launch_pdl(k_lowmom, dim3(grid), dim3(kLowThreads), 0, s, ljobs, ltiles, n_ltiles, geoms, lowpart) ==
                 cudaSuccess
             ? 0
             : -1;
}

}  // namespace tcm
