// Internal definitions shared by the CUDA translation units of libtcm.so.
//
// Moment kernel formulation (Eq. (multipole)).  For one charge q at r = |r| rhat
// the regular solid harmonic is q r^l C_lm(rhat) with C_lm = sqrt(4pi/(2l+1)) Y_lm.
// The kernels never evaluate a trigonometric function: with u = (x + iy)/r and
// c = z/r they run, per column m, the three-term recurrence
//     G_mm     = u^m
//     G_m+1,m  = c G_mm
//     G_l+1,m  = k_lm c G_lm - G_l-1,m           (l >= m+1)
// whose normalisation is chosen so that the G_l-1 coefficient is exactly one, and
// accumulate q (r/a)^l G_lm (in the sign-alternated form H of moments_kernel.cuh).
// The deferred factor F_lm a^l (times the sign of H) turns the sums into Q_lm.
//
// Accumulators live in registers, so the (Lmax+1)^2 components are split into
// column chunks [m0, m1) of at most kmax accumulators; a chunk is a separate tile
// of work that re-reads the atoms.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/tcm.h"

namespace tcm {

constexpr int kLmaxMax = TCM_LMAX_MAX;
constexpr int kThreads = 128;  // threads per moment CTA (4 warps)

// Accumulator budget per thread for the float and double moment kernels, and the CTAs
// per SM the moment kernels are compiled for (register limit 65536 / (128 x CTAs)).
#ifndef TCM_KMAX_F32
#define TCM_KMAX_F32 160
#endif
#ifndef TCM_KMAX_F64
#define TCM_KMAX_F64 80
#endif
#ifndef TCM_MOMENT_CTAS_PER_SM
#define TCM_MOMENT_CTAS_PER_SM 2
#endif
constexpr int kKmaxF32 = TCM_KMAX_F32;
constexpr int kKmaxF64 = TCM_KMAX_F64;

// Chunk plans ("plans" below): the split of the (L+1)^2 accumulators of degree L into column
// chunks of at most kmax.  Plan 0 is the double kernels' (kmax = kKmaxF64); the float kernel is
// built for two budgets, plan 1 (kKmaxF32 accumulators per lane, 2 CTAs per SM) and plan 2
// (kKmaxF32Small, fewer accumulators and registers, 3 CTAs per SM), chosen per degree
// (tcm_ctx_set_chunking_l, the autotuner).  Partial rows keep the largest budget's stride in
// every plan.
constexpr int kKmaxF32Small = 96;
constexpr int kNumPlans = 3;
__host__ __device__ constexpr int plan_kmax(int plan) {
  return plan == 0 ? kKmaxF64 : (plan == 1 ? kKmaxF32 : kKmaxF32Small);
}
__host__ __device__ constexpr int plan_row(int plan) { return plan == 0 ? kKmaxF64 : kKmaxF32; }
// CTAs per SM a float moment kernel of budget kmax is compiled for (its register limit).
__host__ __device__ constexpr int moment_ctas(int kmax) { return kmax <= kKmaxF32Small ? 3 : TCM_MOMENT_CTAS_PER_SM; }

// ---------------------------------------------------------------------------------
// Column-chunk plan (host and device, compile time).
__host__ __device__ constexpr int col_acc(int L, int m) { return m == 0 ? (L + 1) : 2 * (L - m + 1); }

// First column of chunk c when the columns 0..L are split greedily into nch chunks of at
// most kmax accumulators: a chunk closes once it reaches the balanced target, provided
// the remaining columns still fit into the remaining chunks.
__host__ __device__ constexpr int plan_m0(int L, int kmax, int nch, int c) {
  int total = (L + 1) * (L + 1);
  int target = (total + nch - 1) / nch;
  int m = 0;
  int placed = 0;
  for (int cc = 0; cc < nch; ++cc) {
    if (cc == c) return m;
    int acc = 0;
    while (m <= L && acc + col_acc(L, m) <= kmax) {
      const int rest = total - placed - acc;
      if (acc >= target && rest <= kmax * (nch - cc - 1)) break;
      acc += col_acc(L, m);
      ++m;
    }
    placed += acc;
  }
  return m;
}
__host__ __device__ constexpr int plan_nch(int L, int kmax) {
  int n = 1;
  while (plan_m0(L, kmax, n, n) != L + 1) ++n;
  return n;
}
// Accumulator offset of column m inside the chunk that starts at m0.
__host__ __device__ constexpr int chunk_off(int L, int m0, int m) {
  int o = 0;
  for (int k = m0; k < m; ++k) o += col_acc(L, k);
  return o;
}

// Accumulator layout of a chunk [m0, m1) at degree L.  Column 0 (real) takes slots 0..L.
// The complex columns from c0 = max(m0, 1) are grouped in pairs (c0, c0+1), (c0+2, c0+3), ...
// (a last column left over stays single).  A pair (a, b = a+1) keeps Re and Im of its two
// columns side by side, so one packed instruction advances both columns:
//   slots o, o+1                       Re, Im of column a at l = a
//   slots o+2+4(l-b) + {0, 1, 2, 3}    Re_a, Re_b, Im_a, Im_b at l >= b
// and a single column m keeps (Re, Im) at o + 2(l-m) + {0, 1}; o = chunk_off(L, m0, first column).
__host__ __device__ constexpr int acc_first_complex(int m0) { return m0 == 0 ? 1 : m0; }
__host__ __device__ constexpr bool acc_pair_a(int m0, int m1, int m) {
  return m >= acc_first_complex(m0) && ((m - acc_first_complex(m0)) % 2 == 0) && m + 1 < m1;
}
__host__ __device__ constexpr bool acc_pair_b(int m0, int m1, int m) {
  return m > acc_first_complex(m0) && acc_pair_a(m0, m1, m - 1);
}
// Slot of component (l, m), part 0 = Re, 1 = Im (part ignored in column 0).
__host__ __device__ constexpr int acc_slot(int L, int m0, int m1, int l, int m, int part) {
  if (m == 0) return l;
  if (acc_pair_a(m0, m1, m)) {
    const int o = chunk_off(L, m0, m);
    if (l == m) return o + part;
    return o + 2 + 4 * (l - m - 1) + 2 * part;
  }
  if (acc_pair_b(m0, m1, m)) {
    const int o = chunk_off(L, m0, m - 1);
    return o + 2 + 4 * (l - m) + 2 * part + 1;
  }
  return chunk_off(L, m0, m) + 2 * (l - m) + part;
}

// Recurrence coefficient k_lm (l >= m+1), from the ratio r_l = s_l / s_l-1 of the
// normalisations s_lm with F_lm = P_l^m e^{i m phi} = s_lm G_lm:
//   s_mm = (2m-1)!!, s_m+1,m = (2m+1) s_mm, s_l+1 = (l+m) s_l-1 / (l-m+1).
__host__ __device__ constexpr double kcoef(int l, int m) {
  double r = 2.0 * m + 1.0;  // r_{m+1}
  for (int j = m + 1; j < l; ++j) r = (double)(j + m) / ((double)(j - m + 1) * r);
  return (2.0 * l + 1.0) * r / (double)(l + m);
}

// Scaling radius used by the moment kernels: the smallest power of two >= a, so that
// 1/a' is exact in float and the final factor a'^l exact in double.
__host__ __device__ inline double scale_radius(double a) {
  if (!(a > 0.0)) return 1.0;
  int e = 0;
  frexp(a, &e);  // a = f 2^e, 0.5 <= f < 1
  return ldexp(1.0, e);
}

// ---------------------------------------------------------------------------------
// Device descriptors.

struct SysGeom {   // centre and radius of one system (device)
  double c[3];
  double a;
  float chi[3], clo[3];  // the centre split into float parts c = chi + clo (set with c)
  float pad_[2];
};

struct MomJob {    // one moment set: a system at one Lmax under one rotation
  const void* xyzq;
  long long n;
  int dtype;
  int L;
  int geom;        // index into the SysGeom array
  int tiles_per_chunk;
  int atoms_per_tile;
  int tile_base;   // id of the job's first tile; tile id = base + chunk * tpc + t
  double rot[9];   // row-major, identity when unrotated
  double* out;     // packed moments, (L+1)^2 doubles
  int low_base;    // mixed precision: the row of the system-pass partials holding the system's
  int low_tiles;   // low-degree sums (SysJob.sum_row) when low_tiles != 0; 0 = the degrees l <= 2
                   // keep the float kernel's values
  int plan;        // chunk plan of its moment tiles (0: double kernels; 1, 2: float budgets)
  int pad_;
};

struct MomTile {   // one tile of moment work
  int job;
  int chunk;
  int t;           // tile index inside the chunk
  int id;          // global tile id (row of the partials buffer)
};

struct MomGroup {  // the tiles of one (job, chunk), written to the tile list on the device
  int job;
  int chunk;
  int n;           // tiles (the job's tiles_per_chunk)
  int first;       // position of its first tile in the tile list
};

// The pass over a system's atoms before the moment pass (syspass.cu): pass 1 its centroid
// (need_center), pass 2 its radius (need_radius) and, for the mixed path, its low-degree sums
// (need_low).  A system's warp tiles depend on its atom count only (sys_tile_atoms).
struct SysJob {
  const void* xyzq;
  long long n;
  int dtype;
  int geom;          // index into the SysGeom array
  int need_center, need_radius, need_low;
  int tile_base;     // row of its first tile in the partials (kSysPart doubles per row)
  int n_tiles;
  int atoms_per_tile;
  int sum_row;       // row of its low-degree sums over all tiles (written by its last tile)
  int first1;        // position of its first tile in the pass-1 tile list (-1: no pass 1)
  int first2;        // position of its first tile in the pass-2 tile list (-1: no pass 2)
};

struct SysTile {
  int job;
  int t;
};

// Low-degree sums of one system in float-float arithmetic (mixed precision): about the
// system's centre c, with d = x - c and no rotation or scaling,
//   S = sum q,  P_k = sum q d_k,  T_kl = sum q d_k d_l  (k <= l),
// the kLowSums values from which k_finalize forms Q_lm, l <= 2, of every job of the system
// under that job's rotation.  The degrees that carry most of a well-separated pair's energy
// are then accurate to about 2^-44 of their terms instead of the float recurrence's 2^-24.
constexpr int kLowSums = 10;            // S, P_x, P_y, P_z, T_xx, T_xy, T_xz, T_yy, T_yz, T_zz
constexpr int kLowLmax = 2;             // degrees replaced by the low-degree sums

constexpr int kSysThreads = 256;
constexpr int kSysPartR2 = 3;    // partial row: the centroid sums [0, 3), the tile's max |x - c|^2,
constexpr int kSysPartLow = 4;   // and the low-degree sums [4, 4 + kLowSums)
constexpr int kSysPart = kSysPartLow + kLowSums;

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// is set up while its predecessor drains; pdl_wait() blocks until the predecessor grid has
// completed and its memory is visible (a no-op for an ordinary launch).  Only the finalisation
// issues griddepcontrol.launch_dependents (pdl_trigger), so that the contraction's CTAs set up
// their tables while the last finalisation CTAs run; dependent CTAs made resident before the
// moment kernel's tail had drained slowed the replayed step down (0.372 ms against 0.325 ms).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization (programmatic dependent launch): the kernel
// may be scheduled while the previous kernel on the stream drains, and must call
// griddepcontrol.wait before it reads that kernel's results.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// ---------------------------------------------------------------------------------
// Launchers (defined in the .cu files).

// Moment kernels: one persistent launch over `n_tiles` tiles.  plan 0 (double kernels): every
// tile has degree L; plans 1 and 2 (float kernels): tiles of any degree whose jobs have that
// plan (each tile runs the code of its job's degree); the tiles are taken in array order.
// counter[0] and counter[32] must be zero on entry; the launch leaves them zero.
int launch_moments(int plan, int L, const MomJob* jobs, const MomTile* tiles, int n_tiles,
                   int* counter, const SysGeom* geoms, double* partials, int grid, cudaStream_t s);
// The tile lists of a call, written on the device: the moment pass's from its groups,
// tiles[g.first + t] = (g.job, g.chunk, t, row), t < g.n, row = jobs[g.job].tile_base +
// g.chunk * tiles_per_chunk + t; and the system pass's, t1[sj.first1 + t] = t2[sj.first2 + t] =
// (job, t), t < sj.n_tiles.  One warp per group or system job.
int launch_expand_tiles(const MomGroup* groups, int n_groups, const MomJob* jobs, MomTile* tiles, const SysJob* sjobs,
                        int n_sjobs, SysTile* t1, SysTile* t2, cudaStream_t s);
int moments_nchunks(int plan, int L);
int moments_chunk_m0(int plan, int L, int chunk);  // first column of a chunk (chunk = nch: L + 1)
const double* moments_chunk_costs(int plan, int L);  // relative cost per atom of each chunk
// Host: the inverse component maps of every plan and their factors F_lm (imap_off has
// kNumPlans (kLmaxMax + 2) entries, plan by plan, each block ending with its total).
void finalize_tables(std::vector<int>& imap_off, std::vector<int>& imap, std::vector<double>& fmap);

// Step a1 and the low-degree sums: pass 1 over the n1 tiles of the systems that need a centroid,
// then pass 2 over the n2 tiles of those that need a radius or low-degree sums (programmatic
// serialization).  part: kSysPart doubles per tile row; tickets: two ints per job, zero on entry
// and left zero.
int launch_sys(const SysJob* jobs, const SysTile* t1, int n1, const SysTile* t2, int n2, double* part, int* tickets,
               SysGeom* geoms, cudaStream_t s);
int sys_launches(int n1, int n2);
int sys_tile_atoms(long long n);
// Step a3: one CTA per job.  imap + imap_off[plan (kLmaxMax + 2) + L] lists, per (chunk, slot) of
// degree L under the job's plan, the packed component it holds (-1 for none), nch x
// plan_kmax(plan) entries; fmap beside it holds that component's F_lm with the sign of the
// kernels' H variables.  Partial rows are plan_row(plan) doubles apart.
// Jobs with low_tiles != 0 take their degrees l <= min(kLowLmax, L) from the low-degree sums of
// their system (row low_base of the system-pass partials syspart) rotated by the job's rotation.
int launch_finalize(const MomJob* jobs, int n_jobs, const double* partials, const SysGeom* geoms,
                    const int* imap, const double* fmap, const int* imap_off, const double* syspart,
                    cudaStream_t s);



}  // namespace tcm
