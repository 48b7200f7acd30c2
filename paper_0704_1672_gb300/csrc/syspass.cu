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
// in one launch, so small and large systems alike spread over the GPU.  A lane issues the loads
// of several atoms before their arithmetic.  Per-atom arithmetic is
// float for float records: error-free two-sums for the centroid, float-float (two-sum and
// fma-based two-product) for the low-degree sums, and a float filter for the radius: a second
// scan of the tile (from cache) recomputes in double only the atoms within a relative 4e-6 of
// the tile's float maximum.  Tile partials are doubles; the last tile of a system to finish (a ticket)
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

// |x - c|^2 in float from the exact difference d (each coordinate rounded once): within about
// 3 x 2^-24 of the exact value.  The first scan of the radius filter takes this from the
// differences it forms for the low-degree sums anyway.
__device__ __forceinline__ float r2_float(const FF* d) {
  const float x = d[0].h + d[0].l, y = d[1].h + d[1].l, z = d[2].h + d[2].l;
  return __fmaf_rn(x, x, __fmaf_rn(y, y, z * z));
}

// |x - c|^2 in plain float, d_k = (x_k - c_hi,k) - c_lo,k: each difference within 2^-23 of its
// value, the square within about 7 x 2^-24 (4.2e-7).  The second scan of the radius filter uses
// this cheaper form; with the first scan's 1.8e-7 the two stay far inside the filter's 4e-6
// margin, so the atom of the exact maximum is always among the candidates.
__device__ __forceinline__ float r2_plain(const float4& v, const float* chi, const float* clo) {
  const float x = (v.x - chi[0]) - clo[0], y = (v.y - chi[1]) - clo[1], z = (v.z - chi[2]) - clo[2];
  return __fmaf_rn(x, x, __fmaf_rn(y, y, z * z));
}

// Product of a float q (exact) and an FF value: the exact product of the high parts plus q times
// the low part.
__device__ __forceinline__ FF ff_mul_f(float q, FF b) {
  const float p = q * b.h;
  float e = __fmaf_rn(q, b.h, -p);
  e = __fmaf_rn(q, b.l, e);
  return FF{p, e};
}

__device__ __forceinline__ void ff_warp_sum(float& s, float& e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
    ff_acc(s, e, FF{s2, e2});
  }
}

// Reduce-scatter of N float-float sums over the 32 lanes of a warp: at each level (lane offset
// O = 16, 8, ..., 1) a lane keeps the first ceil(n/2) of its n sums if its O bit is clear, the
// rest (padded with zeros) if it is set, and adds in its partner's values of the sums it keeps,
// so each level moves half the values of the previous one (one butterfly per sum would move all
// of them at every level).  A fixed pattern: the same inputs give the same sums in every run.
// For N = 10, lane l ends with the whole of sum 5 b4 + 3 b3 + 2 b2 + b1 in (s[0], e[0]), where
// b_i is bit i of l, if bit l of kRs10Lanes is set (ten lanes; the others hold zeros).
constexpr unsigned kRs10Lanes = 0x05150515u;
template <int N, int O>
__device__ __forceinline__ void ff_reduce_scatter(float* s, float* e, int lane) {
  if constexpr (O > 0) {
    constexpr int K = (N + 1) / 2;
    const bool hi = (lane & O) != 0;
    float ns[K], ne[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float gs = K + j < N ? s[K + j] : 0.f, ge = K + j < N ? e[K + j] : 0.f;
      const float send_s = hi ? s[j] : gs, send_e = hi ? e[j] : ge;
      float a = hi ? gs : s[j], b = hi ? ge : e[j];
      const float rs = __shfl_xor_sync(0xffffffffu, send_s, O), re = __shfl_xor_sync(0xffffffffu, send_e, O);
      ff_acc(a, b, FF{rs, re});
      ns[j] = a;
      ne[j] = b;
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      s[j] = ns[j];
      e[j] = ne[j];
    }
    ff_reduce_scatter<K, O / 2>(s, e, lane);
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp maximum of non-negative doubles through their bit patterns (they order like the integers),
// so that the comparisons stay off the FP64 pipe.
__device__ __forceinline__ double warp_max_d(double v) {
  long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
  return __longlong_as_double(b);
}

// Float-float sums of N consecutive (hi, lo) pairs over n tile rows (stride in floats, p and the
// stride 16-byte aligned): lane l adds rows l, l + 32, ... (all N pairs of a row loaded
// together), then the lanes' pairs are added in a fixed tree, so the same rows give the same
// results in every run.  Float instructions only.  Rows are read through L2 (written by other
// CTAs).  With kR2, also the maximum of the double at float offset r2_off of each row.
template <int N, bool kR2>
__device__ __forceinline__ void ordered_ff_sums(const float* p, int n, int stride, int lane, double* out,
                                                int r2_off = 0, double* r2max = nullptr) {
  float s[N], e[N];
#pragma unroll
  for (int k = 0; k < N; ++k) s[k] = e[k] = 0.f;
  long long b2 = 0;
  for (int r = lane; r < n; r += 32) {
    const float* row = p + (long long)r * stride;
    float4 v[N / 2];
    float2 v1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) v[k] = __ldcg(reinterpret_cast<const float4*>(row) + k);
    if (N % 2) v1 = __ldcg(reinterpret_cast<const float2*>(row) + N - 1);
    if (kR2) b2 = max(b2, __ldcg(reinterpret_cast<const long long*>(row + r2_off)));
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      ff_acc(s[2 * k], e[2 * k], FF{v[k].x, v[k].y});
      ff_acc(s[2 * k + 1], e[2 * k + 1], FF{v[k].z, v[k].w});
    }
    if (N % 2) ff_acc(s[N - 1], e[N - 1], FF{v1.x, v1.y});
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    ff_warp_sum(s[k], e[k]);
    out[k] = (double)s[k] + (double)e[k];
  }
  if (kR2) {  // non-negative doubles order like their bit patterns
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b2 = max(b2, __shfl_xor_sync(0xffffffffu, b2, o));
    *r2max = __longlong_as_double(b2);
  }
}

// Tile rows hold their sums as (hi, lo) float pairs: no per-tile double arithmetic, which on GB300
// runs at 1/64 of the float rate.  Float offsets within a row:
constexpr int kRowFloats = 2 * kSysPart;
constexpr int kRowCen = 0;                 // centroid sums, 3 pairs
constexpr int kRowLow = 2 * kSysPartLow;   // low-degree sums, kLowSums pairs

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

// Atoms per lane whose loads are issued together before any of their arithmetic (the per-atom
// work is short, so a lane must keep several loads in flight to cover the memory latency).
constexpr int kSysBatch = 4;

template <typename Q>
__device__ __forceinline__ FF q_times(Q q, FF d);
template <>
__device__ __forceinline__ FF q_times<FF>(FF q, FF d) { return ff_mul(q, d); }
template <>
__device__ __forceinline__ FF q_times<float>(float q, FF d) { return ff_mul_f(q, d); }
__device__ __forceinline__ FF as_ff(FF q) { return q; }
__device__ __forceinline__ FF as_ff(float q) { return FF{q, 0.f}; }

// q is a float (float records: the charge is exact) or an FF pair (double records).
template <typename Q>
__device__ __forceinline__ void low_accumulate(float* s, float* e, Q q, const FF* d) {
  ff_acc(s[0], e[0], as_ff(q));
  const FF qd0 = q_times(q, d[0]), qd1 = q_times(q, d[1]), qd2 = q_times(q, d[2]);
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
  FF pair[3];
  if (j.dtype == TCM_F32) {
    const float4* X = reinterpret_cast<const float4*>(j.xyzq);
    float s[3] = {0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f};
    for (long long i = i0 + lane; i < i1; i += 32 * kSysBatch) {
      float4 v[kSysBatch];
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u)  // padding atoms add exact zeros
        v[u] = i + 32 * u < i1 ? __ldg(X + i + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u) {
        ff_acc(s[0], e[0], FF{v[u].x, 0.f});
        ff_acc(s[1], e[1], FF{v[u].y, 0.f});
        ff_acc(s[2], e[2], FF{v[u].z, 0.f});
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ff_warp_sum(s[k], e[k]);
      pair[k] = FF{s[k], e[k]};
    }
  } else {
    const double2* X = reinterpret_cast<const double2*>(j.xyzq);
    double s[3] = {0.0, 0.0, 0.0};
    for (long long i = i0 + lane; i < i1; i += 32 * kSysBatch) {
      double2 a[kSysBatch], b[kSysBatch];
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u) {
        const bool ok = i + 32 * u < i1;
        a[u] = ok ? __ldg(X + 2 * (i + 32 * u)) : make_double2(0.0, 0.0);
        b[u] = ok ? __ldg(X + 2 * (i + 32 * u) + 1) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u) {
        s[0] += a[u].x;
        s[1] += a[u].y;
        s[2] += b[u].x;
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // double records: the tile's double sum as a float pair
      const double t = warp_sum_d(s[k]);
      const float h = (float)t;
      pair[k] = FF{h, (float)(t - (double)h)};
    }
  }
  float* row = reinterpret_cast<float*>(part + (long long)(j.tile_base + tl.t) * kSysPart);
  if (lane < 6) row[kRowCen + lane] = (lane & 1) ? pair[lane >> 1].l : pair[lane >> 1].h;
  if (!last_tile(&tickets[2 * tl.job], j.n_tiles, lane)) return;
  const float* p0 = reinterpret_cast<const float*>(part + (long long)j.tile_base * kSysPart);
  const double inv = j.n > 0 ? 1.0 / (double)j.n : 0.0;
  double cs[3];
  ordered_ff_sums<3, false>(p0 + kRowCen, j.n_tiles, kRowFloats, lane, cs);
  if (lane < 3) {  // the centre and its split into float parts
    const double c = (lane == 0 ? cs[0] : (lane == 1 ? cs[1] : cs[2])) * inv;
    const float hi = (float)c;
    geoms[j.geom].c[lane] = c;
    geoms[j.geom].chi[lane] = hi;
    geoms[j.geom].clo[lane] = (float)(c - (double)hi);
  }
}

__global__ void __launch_bounds__(kSysThreads, 3) k_sys_radius_low(const SysJob* __restrict__ jobs,
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
  double rmax = 0.0;  // exact max |x - c|^2 of the tile's atoms
  float s[kLowSums], e[kLowSums];
#pragma unroll
  for (int k = 0; k < kLowSums; ++k) s[k] = e[k] = 0.f;
  if (j.dtype == TCM_F32) {
    const float4* X = reinterpret_cast<const float4*>(j.xyzq);
    const float* chi = g.chi;
    const float* clo = g.clo;
    float mf = 0.f;  // lane's largest |x - c|^2 in float (within about 4e-7 of the exact value)
    for (long long i = i0 + lane; i < i1; i += 32 * kSysBatch) {
      float4 v[kSysBatch];
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u)
        v[u] = i + 32 * u < i1 ? __ldg(X + i + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u) {
        const FF d[3] = {ff_sub_split(v[u].x, chi[0], clo[0]), ff_sub_split(v[u].y, chi[1], clo[1]),
                         ff_sub_split(v[u].z, chi[2], clo[2])};
        if (i + 32 * u < i1) mf = fmaxf(mf, r2_float(d));
        if (j.need_low) low_accumulate(s, e, v[u].w, d);  // padding atoms carry q = 0
      }
    }
    // the exact radius: only atoms within a relative 4e-6 of the tile's float maximum can hold
    // the exact maximum; a second scan of the tile (from cache) recomputes just those in double
    if (j.need_radius) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
      const float thr = mf * (1.0f - 4e-6f);
      for (long long i0w = i0; i0w < i1; i0w += 32) {  // warp-uniform trip count
        const long long i = i0w + lane;
        bool cand = false;
        if (i < i1) cand = r2_plain(__ldg(X + i), chi, clo) >= thr;
        // the candidates one at a time, in a loop whose trip count is the warp's candidate count:
        // a predicated double block would occupy GB300's 1/64-rate FP64 pipe for every atom
        unsigned m = __ballot_sync(0xffffffffu, cand);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const float4 w = __ldcg(X + i0w + src);
          const double ex = (double)w.x - g.c[0], ey = (double)w.y - g.c[1], ez = (double)w.z - g.c[2];
          rmax = fmax(rmax, ex * ex + ey * ey + ez * ez);  // the same value in every lane
        }
      }
    }
  } else {
    const double2* X = reinterpret_cast<const double2*>(j.xyzq);
    for (long long i = i0 + lane; i < i1; i += 32 * kSysBatch) {
      double2 a[kSysBatch], b[kSysBatch];
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u) {
        const bool ok = i + 32 * u < i1;
        a[u] = ok ? __ldg(X + 2 * (i + 32 * u)) : make_double2(g.c[0], g.c[1]);
        b[u] = ok ? __ldg(X + 2 * (i + 32 * u) + 1) : make_double2(g.c[2], 0.0);  // padding: d = 0, q = 0
      }
#pragma unroll
      for (int u = 0; u < kSysBatch; ++u) {
        const double dd[4] = {a[u].x - g.c[0], a[u].y - g.c[1], b[u].x - g.c[2], b[u].y};
        rmax = fmax(rmax, dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        if (j.need_low) {
          FF t[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float h = (float)dd[k];
            t[k] = FF{h, (float)(dd[k] - (double)h)};
          }
          low_accumulate(s, e, t[3], t);
        }
      }
    }
  }
  rmax = warp_max_d(rmax);
  double* row = part + (long long)(j.tile_base + tl.t) * kSysPart;
  if (j.need_low) {
    static_assert(kLowSums == 10, "the lane map of the reduce-scatter is for ten sums");
    ff_reduce_scatter<kLowSums, 16>(s, e, lane);
    if ((kRs10Lanes >> lane) & 1u) {  // the lane holding sum k writes its (hi, lo) pair
      const int k = 5 * ((lane >> 4) & 1) + 3 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
      reinterpret_cast<float2*>(reinterpret_cast<float*>(row) + kRowLow)[k] = make_float2(s[0], e[0]);
    }
  }
  if (lane == 0) row[kSysPartR2] = rmax;
  if (!last_tile(&tickets[2 * tl.job + 1], j.n_tiles, lane)) return;
  // the last tile of the system: its radius and its low-degree sums over all tiles (tile order),
  // written once to the system's sum row, which every moment job of the system reads
  const double* p0 = part + (long long)j.tile_base * kSysPart;
  if (j.need_low) {  // one pass over the tile rows: the ten sums and the radius together
    double* sr = part + (long long)j.sum_row * kSysPart;
    double low[kLowSums], m = 0.0;
    ordered_ff_sums<kLowSums, true>(reinterpret_cast<const float*>(p0) + kRowLow, j.n_tiles, kRowFloats, lane, low,
                                    2 * (kSysPartR2 - kSysPartLow), &m);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < kLowSums; ++k) sr[kSysPartLow + k] = low[k];
      if (j.need_radius) geoms[j.geom].a = sqrt(m);
    }
  } else if (j.need_radius) {
    double m = 0.0;
    for (int r = lane; r < j.n_tiles; r += 32) m = fmax(m, __ldcg(p0 + (long long)r * kSysPart + kSysPartR2));
    m = warp_max_d(m);
    if (lane == 0) geoms[j.geom].a = sqrt(m);
  }
}

}  // namespace

int sys_tile_atoms(long long n) {
  // 256-atom tiles (8 per lane) up to 32,768 atoms, 512 up to 65,536, 1,024 above: enough warps
  // for the GPU even for a single system, few enough partial rows for the largest (128-atom
  // tiles were tried: their per-tile reductions cost more on a batch of many systems than the
  // extra warps gained on a pair of 20,000-atom systems)
  long long t = 256;
  while (t < 1024 && t * 128 < n) t *= 2;
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
