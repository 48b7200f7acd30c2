// Kernels around the moment pass:
//   a3  cross-tile reduction of the moment partials in double, fixed order, plus the
//       deferred normalisation F_lm a^l                                  (Eq. (multipole))
//   a4  irregular solid harmonics of the separation vector R0            (Eq. (Formula))
//   a5  two-center contraction in double                                 (Eq. (Formula))
//   a6  exact pairwise Coulomb sum in double                             (Eq. (Coulomb))
#include <cuda_runtime.h>

#include "contract.h"

namespace tcm {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// Fixed-order block sum (deterministic); result valid in thread 0.  blockDim <= 1024.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}
__device__ __forceinline__ void load_xyz(const void* p, int dtype, long long i, double& x, double& y, double& z,
                                         double& q) {
  if (dtype == TCM_F32) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
    x = v.x;
    y = v.y;
    z = v.z;
    q = v.w;
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p) + 2 * i);
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 2 * i + 1);
    x = a.x;
    y = a.y;
    z = b.x;
    q = b.y;
  }
}

// Degrees l <= kLowLmax of one job from its system's low-degree sums (system pass 2, reduced over
// the system's tiles by its last tile): the Cartesian sums are rotated by the job's rotation R
// (P' = R P, T' = R T R^T, p = R d) and turned into the packed Q_lm, l <= 2, with
//   Q_00 = S,  Q_10 = P'_z,  Q_11 = -(P'_x + i P'_y)/sqrt(2),
//   Q_20 = T'_zz - (T'_xx + T'_yy)/2,  Q_21 = -sqrt(3/2) (T'_xz + i T'_yz),
//   Q_22 = sqrt(3/8) (T'_xx - T'_yy + 2 i T'_xy),
// the regular solid harmonics r^l sqrt(4 pi/(2l+1)) Y_lm of Eq. (multipole) written out in x, y, z.
constexpr int kLowComps = (kLowLmax + 1) * (kLowLmax + 1);
__device__ void low_degrees(const MomJob& job, const double* __restrict__ syspart, double* s_low) {
  if (threadIdx.x < kLowSums) s_low[threadIdx.x] = __ldcg(syspart + (long long)job.low_base * kSysPart + kSysPartLow + threadIdx.x);
  __syncthreads();
  const int k = threadIdx.x;  // packed output slot, one thread each
  if (k >= (job.L + 1) * (job.L + 1) || k >= kLowComps) return;
  const double* R = job.rot;
  const double P[3] = {s_low[1], s_low[2], s_low[3]};
  const double T[3][3] = {{s_low[4], s_low[5], s_low[6]}, {s_low[5], s_low[7], s_low[8]}, {s_low[6], s_low[8], s_low[9]}};
  auto pr = [&](int a) { return R[3 * a] * P[0] + R[3 * a + 1] * P[1] + R[3 * a + 2] * P[2]; };  // (R P)_a
  auto tr = [&](int a, int b) {  // (R T R^T)_ab
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s += R[3 * a + i] * (T[i][0] * R[3 * b] + T[i][1] * R[3 * b + 1] + T[i][2] * R[3 * b + 2]);
    return s;
  };
  const double r2 = 0.70710678118654752440, s32 = 1.22474487139158904910, s38 = 0.61237243569579452455;
  double v;
  switch (k) {
    case 0: v = s_low[0]; break;
    case 1: v = pr(2); break;
    case 2: v = -r2 * pr(0); break;
    case 3: v = -r2 * pr(1); break;
    case 4: v = tr(2, 2) - 0.5 * (tr(0, 0) + tr(1, 1)); break;
    case 5: v = -s32 * tr(0, 2); break;
    case 6: v = -s32 * tr(1, 2); break;
    case 7: v = s38 * (tr(0, 0) - tr(1, 1)); break;
    default: v = s32 * tr(0, 1); break;
  }
  job.out[k] = v;
}

// a3: one CTA per moment job.  Threads walk the (chunk, slot) entries of the job's partial
// rows in memory order (coalesced), sum each over the job's tiles in tile order (double) and
// write F_lm a'^l times the sum to the packed component the slot holds.  The map entry, its
// factor F_lm and the partial rows do not depend on each other, so their loads overlap; a' is a
// power of two, so a'^l is formed exactly from its exponent.
constexpr int kFinalizeThreads = 512;
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const MomJob* __restrict__ jobs,
                                                               const double* __restrict__ partials,
                                                               const SysGeom* __restrict__ geoms,
                                                               const int* __restrict__ imap,
                                                               const double* __restrict__ fmap,
                                                               const int* __restrict__ imap_off,
                                                               const double* __restrict__ syspart) {
  __shared__ double s_low[kLowSums];
  pdl_trigger();  // the contraction may be scheduled; it waits for this grid before reading
  pdl_wait();     // the moment kernels' partial rows are complete
  const MomJob& job = jobs[blockIdx.x];
  const int L = job.L;
  const int tpc = job.tiles_per_chunk;
  const int kmax = plan_kmax(job.plan), row = plan_row(job.plan);
  const int* off = imap_off + job.plan * (kLmaxMax + 2);
  const int o = off[L];
  const int nq = off[L + 1] - o;  // nch x kmax
  const double a = geoms[job.geom].a;
  int e = 0;  // a' = scale_radius(a) = 2^e
  if (a > 0.0) frexp(a, &e);
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int p = imap[o + q];
    const double f = fmap[o + q];
    const int ch = q / kmax, slot = q - ch * kmax;
    const double* base = partials + (long long)(job.tile_base + ch * tpc) * row + slot;
    double s = 0.0;
#pragma unroll 8
    for (int t = 0; t < tpc; ++t) s += __ldcg(base + (long long)t * row);  // loads issued ahead of the adds
    if (p < 0) continue;
    int l = (int)sqrtf((float)p);
    while (l * l > p) --l;
    while ((l + 1) * (l + 1) <= p) ++l;
    const int ex = e * l;  // a'^l = 2^ex, built from its exponent bits when it is a normal double
    const double al = (ex >= -1022 && ex <= 1023) ? __longlong_as_double((long long)(ex + 1023) << 52) : ldexp(1.0, ex);
    if (job.low_tiles > 0 && p < kLowComps) continue;  // written from the low-degree sums below
    job.out[p] = f * al * s;
  }
  if (job.low_tiles > 0) low_degrees(job, syspart, s_low);
}

// a4 + a5: one CTA per energy, in the frame where R0hat is the z axis.
//
// With the stretched 3j symbol (L = l1 + l2) Eq. (Formula) reads
//   U = sum (-1)^l2 Qhat^A_l1m1 Qhat^B_l2m2 J_{l1+l2, m1+m2},
//   Qhat_lm = Q_lm / sqrt((l+m)!(l-m)!),  J_LM = sqrt((L+M)!(L-M)!) sqrt(4pi/(2L+1)) Y*_LM(R0hat) / R^{L+1}.
// U does not change when A, B and R0 rotate together.  In the frame W = R_y(-beta) R_z(-alpha)
// that takes R0hat = (sin b cos a, sin b sin a, cos b) to z, J_LM = delta_M0 L! / R^{L+1}, so
//   U = sum_{l1,l2} (-1)^l2 (l1+l2)! / R^{l1+l2+1}
//         [Qhat'^A_l1,0 Qhat'^B_l2,0 + 2 sum_{m>=1} (-1)^m Re(Qhat'^A_l1m conj(Qhat'^B_l2m))]
// (real charges: Q_l,-m = (-1)^m conj(Q_lm)).  Moments enter in the rotated frame: those of B
// either come from the moment kernels with W folded into the atom transform (mode kBInFrame),
// or, like those of A, are rotated here (kBLab by W; kBRotate by W rotB from a moment cache):
//   Q'_lm = sum_m' d^l_{m'm}(beta) P_lm',  P_lm' = e^{-i m' alpha} Q_lm'.
// The Wigner matrix d^l(beta) is never formed.  A rotation about y is a rotation about z
// between two rotations by pi/2 about x, which for the constant matrices D^l = d^l(pi/2) gives
//   d^l_{m'm}(beta) = i^(m-m') sum_k D^l_{km'} D^l_{km} e^{i k beta},
// so Q' follows from two products with D^l around a diagonal phase:
//   p_k = sum_m' D^l_{km'} v_m',  v_m' = (-i)^m' P_lm';   Q'_lm = i^m sum_k D^l_{km} e^{i k beta} p_k.
// For real charges v_-m' = (-1)^m' conj(v_m') and p_-k = (-1)^k conj(p_k); with
// D^l_{k,-m'} = (-1)^(l+k) D^l_{km'} and D^l_{km} = (-1)^(k-m) D^l_{mk} the terms of m' and -m'
// (and of k and -k) combine into one real product, which leaves, for k, m >= 0,
//   Re p_k = sum_{m' = l+k (mod 2)} D^l_{km'} Re v~_m',   Im p_k = sum_{other m'} D^l_{km'} Im v~_m',
//   S_m = (-1)^l [sum_{k = l+m (mod 2)} D^l_{mk} Re p~_k - i sum_{other k} D^l_{mk} Im p~_k],  Q'_lm = i^m S_m,
// with v~_m' = v_m' and p~_k = e^{i k beta} p_k, both doubled for indices >= 1: (l+1)^2 real
// multiply-adds per product and degree, no table of d^l(beta) per energy.
constexpr int kContractThreads = 512;  // most threads of a contraction CTA

// Layout of ztab (doubles): k! and 2 k! for k < 2 kZN, 1/sqrt((l+m)!(l-m)!) at [l][m], and the rows of
// D^l = d^l(pi/2): D^l_{km}, 0 <= k, m <= l, at kZ_DPI2 + dpi2_off(l) + k dpi2_stride(l) + m.  The
// row stride is odd (rows of even length get one zero), so that the lanes of a warp reading
// one entry of consecutive rows hit distinct shared-memory banks; shared memory holds the
// same layout.
constexpr int kZN = kLmaxMax + 1;
constexpr int kZ_FACT = 0;
constexpr int kZ_FACT2 = kZ_FACT + 2 * kZN;
constexpr int kZ_ISF = kZ_FACT2 + 2 * kZN;
constexpr int kZ_DPI2 = kZ_ISF + kZN * kZN;
__host__ __device__ constexpr int dpi2_stride(int l) { return (l + 1) | 1; }
__host__ __device__ constexpr int dpi2_off(int l) {  // sum over l' < l of (l'+1) dpi2_stride(l')
  return l * (l + 1) * (2 * l + 1) / 6 + (l / 2) * (l / 2 + 1);
}
constexpr int kZ_TOTAL = kZ_DPI2 + dpi2_off(kZN);

__device__ __forceinline__ double flip(double x, int odd) {  // (-1)^odd x without an FP64 op
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(odd & 1) << 63));
}

// i^n z for any integer n, by exchanging and negating the parts (no FP64 operation).
__device__ __forceinline__ double2 mul_ipow(double2 z, int n) {
  const int r = n & 3;
  const double2 s = (r & 1) ? make_double2(z.y, z.x) : z;
  return make_double2(flip(s.x, r == 1 || r == 2), flip(s.y, r >= 2));
}

__device__ __forceinline__ int tri_l(int k) {  // l with l(l+1)/2 <= k < (l+1)(l+2)/2
  int l = (int)((sqrtf(8.0f * k + 1.0f) - 1.0f) * 0.5f);
  while (l * (l + 1) / 2 > k) --l;
  while ((l + 1) * (l + 2) / 2 <= k) ++l;
  return l;
}

// Row product with a parity split: (sum over j = par (mod 2) of row[j] Re x_j, sum over the other
// j of row[j] Im x_j), j = 0..l.  One multiply-add per entry.
__device__ __forceinline__ double2 row_split(const double* row, const double2* x, int l, int par) {
  const double* xs = reinterpret_cast<const double*>(x);
  double a = 0.0, b = 0.0;  // even j, odd j
  int j = 0;
  for (; j + 1 <= l; j += 2) {
    a = fma(row[j], xs[2 * j + par], a);
    b = fma(row[j + 1], xs[2 * j + 3 - par], b);
  }
  if (j == l) a = fma(row[j], xs[2 * j + par], a);
  return par ? make_double2(b, a) : make_double2(a, b);
}

// Copies the rows of D^l for l <= L into shared memory (a constant table: no dependence on the
// kernels before, so it is read ahead of griddepcontrol.wait).
__device__ void load_dpi2(double* Ds, const double* __restrict__ ztab, int L) {
  const double* src = ztab + kZ_DPI2;
  const int n = dpi2_off(L + 1);
  for (int i = threadIdx.x; i < n; i += blockDim.x) Ds[i] = __ldg(src + i);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// x^n by binary powering (n >= 0).
__device__ __forceinline__ double rpow(double x, int n) {
  double r = 1.0;
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}

// z^lane in every lane of the calling warp (lane <= 31): an inclusive product scan of
// (1, z, z, ...), five steps of one complex multiplication each.
__device__ __forceinline__ double2 warp_pow_scan(double2 z, int lane) {
  double2 r = lane == 0 ? make_double2(1.0, 0.0) : z;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const double2 u = make_double2(__shfl_up_sync(0xffffffffu, r.x, s), __shfl_up_sync(0xffffffffu, r.y, s));
    if (lane >= s) r = cmul(r, u);
  }
  return r;
}
// x^(lane + 1) in every lane of the calling warp.
__device__ __forceinline__ double warp_rpow_scan(double x, int lane) {
  double r = x;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, r, s);
    if (lane >= s) r *= u;
  }
  return r;
}

// The phase factors of one rotation R_z(-gamma) R_y(-beta) R_z(-alpha), one warp per table,
// entry m = lane <= L:
//   in:   (-i)^m e^{-i m alpha}, doubled for m >= 1       (from e^{i alpha})
//   beta: e^{i k beta}, doubled for k >= 1                (from cos beta, sin beta)
//   out:  i^m e^{-i m gamma}                              (from e^{i gamma})
__device__ __forceinline__ void in_phases(double2* t, double2 e, int L, int lane) {
  const double2 z = mul_ipow(warp_pow_scan(make_double2(e.x, -e.y), lane), -lane);
  if (lane <= L) t[lane] = lane > 0 ? make_double2(2.0 * z.x, 2.0 * z.y) : z;
}
__device__ __forceinline__ void beta_phases(double2* t, double cb, double sb, int L, int lane) {
  const double2 z = warp_pow_scan(make_double2(cb, sb), lane);
  if (lane <= L) t[lane] = lane > 0 ? make_double2(2.0 * z.x, 2.0 * z.y) : z;
}
__device__ __forceinline__ void out_phases(double2* t, double2 e, int L, int lane) {
  const double2 z = mul_ipow(warp_pow_scan(make_double2(e.x, -e.y), lane), lane);
  if (lane <= L) t[lane] = z;
}

// First product of a rotation, item k = (l, kk) of the triangle: p~_kk from v~ (the moments
// times the input phases) of degree l.
__device__ __forceinline__ double2 rot_first(const double* Ds, const double2* v, const double2* eb, int k) {
  const int l = tri_l(k);
  const int kk = k - l * (l + 1) / 2;
  const double2 p = row_split(Ds + dpi2_off(l) + kk * dpi2_stride(l), v + l * (l + 1) / 2, l, (l + kk) & 1);
  return cmul(eb[kk], p);
}
// Second product, item k = (l, m): S_m, times the output phase (i^m when there is no gamma) and,
// with hat, 1/sqrt((l+m)!(l-m)!).
__device__ __forceinline__ double2 rot_second(const double* Ds, const double2* p, const double2* phout,
                                              const double* ztab, bool hat, int k) {
  const int l = tri_l(k);
  const int m = k - l * (l + 1) / 2;
  const double2 a = row_split(Ds + dpi2_off(l) + m * dpi2_stride(l), p + l * (l + 1) / 2, l, (l + m) & 1);
  const double2 S = make_double2(flip(a.x, l), flip(a.y, l + 1));
  double2 q = phout ? cmul(phout[m], S) : mul_ipow(S, m);
  if (hat) {
    const double f = ztab[kZ_ISF + l * kZN + m];
    q = make_double2(q.x * f, q.y * f);
  }
  return q;
}

// Eq. (Formula) for one (pair, orientation) per CTA, in the frame where R0hat = z.  With kGrad
// it also writes, per item, the force on B (-grad_R0 E) and the torques on A and on B about
// their centres, from the same frame moments:
//   in the frame, with c = (-1)^l2 L!/R^(L+1), c' = (-1)^l2 (L+1)!/R^(L+2), L = l1 + l2,
//   T0 = sum_m Qa_m Qb_-m,  S+ = sum_{m1+m2=1} Qa_m1 Qb_m2,  P = sum_{m1+m2=1} (l2+m2) Qa_m1 Qb_m2,
//   Z = sum_{m>=1} (-1)^m 2m Im(Qa_m conj Qb_m)  (Qhat normalisation throughout):
//   grad E = -sum c' (Re S+, Im S+, T0)       (only J_L,0 and J_L,+-1 have a first-order
//                                                derivative on the z axis);
//   tau_B = sum c (Im P, -Re P, -Z),  tau_A = sum c (Im P', -Re P', Z),  P' = (L+1) S+ - P
//   (infinitesimal rotations act on Qhat_lm through L_z and the ladder operators with the
//   integer weights (l+m+1), (l-m+1)).  The vectors go back to the lab frame with W^T.
// Launch bounds: the energy kernel stays within 64 registers (4 CTAs of 256 threads per SM for
// large batches); the gradient kernel, with nine sums per thread, may take more (at the default
// it was held to 64 and spilled).
template <bool kGrad>
__global__ void __launch_bounds__(kContractThreads, kGrad ? 1 : 2) k_contract(const PairDesc* __restrict__ items,
                                                               const MomJob* __restrict__ jobs,
                                                               const SysGeom* __restrict__ geoms,
                                                               const double* __restrict__ ztab,
                                                               const double* __restrict__ rots,
                                                               double* __restrict__ E, int32_t* __restrict__ status,
                                                               double* __restrict__ G) {
  extern __shared__ double2 sm2[];
  constexpr int kVWarps = kContractThreads / 32;
  __shared__ double she[kContractThreads];           // the virtual lanes' energy sums
  __shared__ double shv[(kGrad ? 8 : 1) * kVWarps];  // the virtual warps' gradient sums
  __shared__ int g_conv;
  const PairDesc d = items[blockIdx.x];  // descriptors and tables precede the kernels before
  const int L = d.L;
  const int nq = (L + 1) * (L + 2) / 2;
  const int n1 = L + 1;
  double2* qa = sm2;            // A: lab frame, v~, then Qhat' in the frame
  double2* qb = qa + nq;        // B: the same (or its frame moments, mode kBInFrame)
  double2* ta = qb + nq;        // p~ of A
  double2* tb = ta + nq;        // p~ of B
  double2* ph = tb + nq;        // input phases of W (alpha of R0)
  double2* eb = ph + n1;        // beta phases of W
  double2* pha = eb + n1;       // mode kBRotate: input, beta and output phases of W rotB
  double2* ebB = pha + n1;
  double2* phg = ebB + n1;
  double* rp = reinterpret_cast<double*>(phg + n1);  // R^-(k+1), k <= 2L + 1
  double* c2t = rp + 2 * L + 2;                       // 2 n! R^-(n+1), n <= 2L
  double* hb0 = c2t + 2 * L + 1;                      // Qhat'^B_l0 / 2
  double* Ds = hb0 + L + 1;                           // rows of D^l, l <= L
  // Before griddepcontrol.wait: everything that depends only on the descriptors and tables the
  // host uploaded ahead of the kernels (the d^l(pi/2) rows, the phase and power tables of the
  // frame, the moment sets' addresses), so it overlaps the tail of the kernel before.
  load_dpi2(Ds, ztab, L);
  const int bmode = d.b_mode;
  const double* pa = jobs[d.jobA].out;
  const double* pb = jobs[d.jobB].out;
  {  // the phase tables and R^-(k+1) (k <= 2L + 1 <= 49), one warp per table (warp-uniform tasks)
    const int lane = threadIdx.x & 31;
    const int ntask = bmode == kBRotate ? 7 : 4;
    for (int tt = threadIdx.x >> 5; tt < ntask; tt += blockDim.x >> 5) {
      const EulerZYZ* e = reinterpret_cast<const EulerZYZ*>(rots) + d.rot;
      switch (tt) {
        case 0: in_phases(ph, make_double2(d.fr[4], d.fr[5]), L, lane); break;
        case 1: beta_phases(eb, d.fr[2], d.fr[3], L, lane); break;
        case 2: {
          const double r = warp_rpow_scan(d.fr[0], lane);
          if (lane < 2 * L + 2) rp[lane] = r;
          break;
        }
        case 3:
          if (2 * L + 2 > 32) {
            const double r = warp_rpow_scan(d.fr[0], lane) * rpow(d.fr[0], 32);
            if (32 + lane < 2 * L + 2) rp[32 + lane] = r;
          }
          break;
        case 4: in_phases(pha, make_double2(e->ea[0], e->ea[1]), L, lane); break;
        case 5: beta_phases(ebB, e->cb, e->sb, L, lane); break;
        default: out_phases(phg, make_double2(e->eg[0], e->eg[1]), L, lane); break;
      }
    }
  }
  __syncthreads();
  for (int n = threadIdx.x; n <= 2 * L; n += blockDim.x) c2t[n] = ztab[kZ_FACT2 + n] * rp[n];
  pdl_wait();  // the moments (and centres and radii) of the launches before are complete
  // the radii come from the kernels before
  if (threadIdx.x == 0) g_conv = d.fr[1] > geoms[d.geomA].a + geoms[d.geomB].a;  // Eq. (mainCond)
  // v~ = input phases times the moments of the sides rotated here; mode kBInFrame scales B to Qhat
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const int l = tri_l(k);
    const int m = k - l * (l + 1) / 2;
    const double2 a = m == 0 ? make_double2(pa[l * l], 0.0) : make_double2(pa[l * l + 2 * m - 1], pa[l * l + 2 * m]);
    const double2 b = m == 0 ? make_double2(pb[l * l], 0.0) : make_double2(pb[l * l + 2 * m - 1], pb[l * l + 2 * m]);
    qa[k] = cmul(ph[m], a);
    if (bmode == kBLab) {
      qb[k] = cmul(ph[m], b);
    } else if (bmode == kBRotate) {
      qb[k] = cmul(pha[m], b);
    } else {
      const double f = ztab[kZ_ISF + l * kZN + m];
      qb[k] = make_double2(b.x * f, b.y * f);
      if (m == 0) hb0[l] = 0.5 * qb[k].x;
    }
  }
  __syncthreads();
  if (!g_conv) {  // the expansion does not converge: NaN and a status instead of an energy
    if (threadIdx.x == 0) {
      E[blockIdx.x] = __longlong_as_double(0x7ff8000000000000LL);
      if (status) status[blockIdx.x] = TCM_ENOTCONV;
    }
    if (kGrad && threadIdx.x < 9) G[9LL * blockIdx.x + threadIdx.x] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  const int nrot = bmode == kBInFrame ? 1 : 2;
  for (int it = threadIdx.x; it < nrot * nq; it += blockDim.x) {
    const int side = it >= nq;
    const int k = it - side * nq;
    if (side) tb[k] = rot_first(Ds, qb, bmode == kBRotate ? ebB : eb, k);
    else ta[k] = rot_first(Ds, qa, eb, k);
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nrot * nq; it += blockDim.x) {
    const int side = it >= nq;
    const int k = it - side * nq;
    if (side) {
      const double2 q = rot_second(Ds, tb, bmode == kBRotate ? phg : nullptr, ztab, true, k);
      qb[k] = q;
      const int l = tri_l(k);
      if (k == l * (l + 1) / 2) hb0[l] = 0.5 * q.x;
    } else {
      qa[k] = rot_second(Ds, ta, nullptr, ztab, true, k);
    }
  }
  __syncthreads();
  const double2* ra = qa;  // Qhat' of A and B in the frame
  const double2* rb = qb;
  // z-axis contraction: one thread per (l1, l2).  The pairs are taken in shells of equal
  // s = min(l1, l2), s = L first: the (L - s)^2 pairs before shell s are those of the larger
  // shells, and shell s lists (s, s), (s, s+1), (s+1, s), (s, s+2), ...  Neighbouring lanes then
  // run the m loops (s terms) to nearly the same length.
  //
  // The energy's summation order does not depend on the CTA size (which the launch picks from
  // the batch): pair p belongs to virtual lane p mod kContractThreads, each virtual lane adds its
  // pairs in increasing p, lane c of one warp adds virtual lanes c, c + 32, ... in order, and a
  // fixed shuffle tree adds the 32 lanes.  A CTA of nt threads runs virtual lanes t, t + nt, ...
  // one after the other, so an item's energy is the same in any batch.  (The sequential sums keep
  // the FP64 instructions of the reduction to about a tenth of a shuffle tree per warp.)  The
  // gradient sums take a shuffle tree per virtual warp of 32 lanes, then one over those.
  const int n_pairs = (L + 1) * (L + 1);
  for (int v = threadIdx.x; v < kContractThreads; v += blockDim.x) {  // block-uniform trip count
    double acc = 0.0;
    double gx = 0.0, gy = 0.0, gz = 0.0, tbx = 0.0, tby = 0.0, tbz = 0.0, tax = 0.0, tay = 0.0;
    for (int p = v; p < n_pairs; p += kContractThreads) {
      int u = (int)sqrtf((float)p);  // u = L - s = floor(sqrt(p))
      while (u * u > p) --u;
      while ((u + 1) * (u + 1) <= p) ++u;
      const int sh_s = L - u, j = p - u * u;
      const int l1 = (j & 1) ? sh_s : sh_s + (j >> 1);
      const int l2 = (j & 1) ? sh_s + ((j + 1) >> 1) : sh_s;
      const double2* a = ra + l1 * (l1 + 1) / 2;
      const double2* b = rb + l2 * (l2 + 1) / 2;
      const int mm = l1 < l2 ? l1 : l2;
      // even and odd m: with the m = 0 term at half weight, s / 2 = a_0 b_0 / 2 + sum_{m>=1} (-1)^m
      // Re(a_m conj b_m) = se - so, and the factor 2 sits in the table c2t
      double se = a[0].x * hb0[l2], so = 0.0;
      int m = 1;
      for (; m + 1 <= mm; m += 2) {
        so = fma(a[m].x, b[m].x, so);
        so = fma(a[m].y, b[m].y, so);
        se = fma(a[m + 1].x, b[m + 1].x, se);
        se = fma(a[m + 1].y, b[m + 1].y, se);
      }
      if (m <= mm) {
        so = fma(a[m].x, b[m].x, so);
        so = fma(a[m].y, b[m].y, so);
      }
      const double h = se - so;
      acc = fma(flip(c2t[l1 + l2], l2), h, acc);
      if (kGrad) {
        const double s = h + h;
        const double c = flip(ztab[kZ_FACT + l1 + l2] * rp[l1 + l2], l2);
        // S+ and P: pairs (m1, m2) = (m, 1 - m), m >= 1, and (-m, m + 1), m >= 0
        double spr = 0.0, spi = 0.0, pr = 0.0, pi = 0.0, z = 0.0;
        const int m1a = l1 < l2 + 1 ? l1 : l2 + 1;
        for (int m = 1; m <= m1a; ++m) {  // (-1)^(m-1) a_m conj(b_(m-1)), weight l2 + 1 - m
          const double2 x = a[m], y = b[m - 1];
          const double re = flip(fma(x.x, y.x, x.y * y.y), m - 1);
          const double im = flip(fma(x.y, y.x, -(x.x * y.y)), m - 1);
          const double w = (double)(l2 + 1 - m);
          spr += re;
          spi += im;
          pr = fma(w, re, pr);
          pi = fma(w, im, pi);
        }
        const int m1b = l1 < l2 - 1 ? l1 : l2 - 1;
        for (int m = 0; m <= m1b; ++m) {  // (-1)^m conj(a_m) b_(m+1), weight l2 + 1 + m
          const double2 x = a[m], y = b[m + 1];
          const double re = flip(fma(x.x, y.x, x.y * y.y), m);
          const double im = flip(fma(x.x, y.y, -(x.y * y.x)), m);
          const double w = (double)(l2 + 1 + m);
          spr += re;
          spi += im;
          pr = fma(w, re, pr);
          pi = fma(w, im, pi);
        }
        for (int m = 1; m <= mm; ++m) z += flip((double)(2 * m) * fma(a[m].y, b[m].x, -(a[m].x * b[m].y)), m);
        const double c1 = flip(ztab[kZ_FACT + l1 + l2 + 1] * rp[l1 + l2 + 1], l2);
        const double L1 = (double)(l1 + l2 + 1);
        gx = fma(-c1, spr, gx);
        gy = fma(-c1, spi, gy);
        gz = fma(-c1, s, gz);
        tbx = fma(c, pi, tbx);
        tby = fma(-c, pr, tby);
        tbz = fma(-c, z, tbz);
        tax = fma(c, fma(L1, spi, -pi), tax);
        tay = fma(-c, fma(L1, spr, -pr), tay);
      }
    }
    she[v] = acc;
    if (kGrad) {
      double w[8] = {gx, gy, gz, tbx, tby, tbz, tax, tay};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        w[k] = warp_sum(w[k]);
        if ((threadIdx.x & 31) == 0) shv[k * kVWarps + (v >> 5)] = w[k];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double e_sum = she[lane];
#pragma unroll
  for (int c = 1; c < kVWarps; ++c) e_sum += she[c * 32 + lane];
  e_sum = warp_sum(e_sum);  // valid in lane 0
  if (!kGrad) {
    if (lane == 0) {
      E[blockIdx.x] = e_sum;
      if (status) status[blockIdx.x] = TCM_OK;
    }
  } else {
    double w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = warp_sum(lane < kVWarps ? shv[k * kVWarps + lane] : 0.0);
    if (lane == 0) {
      const double v[9] = {e_sum, w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]};
      E[blockIdx.x] = v[0];
      if (status) status[blockIdx.x] = TCM_OK;
      const double cb = d.fr[2], sb = d.fr[3], ca = d.fr[4], sa = d.fr[5];
      const double W[9] = {cb * ca, cb * sa, -sb, -sa, ca, 0.0, sb * ca, sb * sa, cb};  // R_y(-b) R_z(-a)
      // frame -> lab: v_lab = W^T v_frame; force = -grad; tau_A,z = -tau_B,z
      const double f[3] = {-v[1], -v[2], -v[3]};
      const double ta[3] = {v[7], v[8], -v[6]};
      const double tb[3] = {v[4], v[5], v[6]};
      double* o = G + 9LL * blockIdx.x;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o[i] = W[i] * f[0] + W[3 + i] * f[1] + W[6 + i] * f[2];
        o[3 + i] = W[i] * ta[0] + W[3 + i] * ta[1] + W[6 + i] * ta[2];
        o[6 + i] = W[i] * tb[0] + W[3 + i] * tb[1] + W[6 + i] * tb[2];
      }
    }
  }
}

// Moments of a system rotated by M about its centre, from its lab-frame moments: the Wigner
// rotation R_z(-gamma) R_y(-beta) R_z(-alpha) = M applied degree by degree (one CTA per set),
// by the two products with d^l(pi/2) above.
__global__ void __launch_bounds__(kContractThreads) k_rotate_moments(const RotDesc* __restrict__ sets,
                                                                     const double* __restrict__ ztab) {
  extern __shared__ double2 sm2[];
  __shared__ EulerZYZ g_e;
  const RotDesc d = sets[blockIdx.x];
  const int L = d.L;
  const int nq = (L + 1) * (L + 2) / 2;
  const int n1 = L + 1;
  double2* q = sm2;
  double2* t = q + nq;
  double2* pha = t + nq;
  double2* ebB = pha + n1;
  double2* phg = ebB + n1;
  double* Ds = reinterpret_cast<double*>(phg + n1);
  load_dpi2(Ds, ztab, L);
  if (threadIdx.x == 0) g_e = euler_zyz(sets[blockIdx.x].M);
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const int l = tri_l(k);
    const int m = k - l * (l + 1) / 2;
    q[k] = m == 0 ? make_double2(d.in[l * l], 0.0) : make_double2(d.in[l * l + 2 * m - 1], d.in[l * l + 2 * m]);
  }
  __syncthreads();
  for (int tt = threadIdx.x >> 5; tt < 3; tt += blockDim.x >> 5) {
    const int lane = threadIdx.x & 31;
    if (tt == 0) in_phases(pha, make_double2(g_e.ea[0], g_e.ea[1]), L, lane);
    else if (tt == 1) beta_phases(ebB, g_e.cb, g_e.sb, L, lane);
    else out_phases(phg, make_double2(g_e.eg[0], g_e.eg[1]), L, lane);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const int l = tri_l(k);
    q[k] = cmul(pha[k - l * (l + 1) / 2], q[k]);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nq; k += blockDim.x) t[k] = rot_first(Ds, q, ebB, k);
  __syncthreads();
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const int l = tri_l(k);
    const int m = k - l * (l + 1) / 2;
    const double2 r = rot_second(Ds, t, phg, ztab, false, k);
    if (m == 0) {
      d.out[l * l] = r.x;
    } else {
      d.out[l * l + 2 * m - 1] = r.x;
      d.out[l * l + 2 * m] = r.y;
    }
  }
}

// a6: exact pairwise sum.  One thread per atom of A; B staged through shared memory
// already rotated and translated: b' = R0 + rot (x_b - c_B).  Double precision.
constexpr int kDirectThreads = 256;

struct alignas(32) Atom4 {  // a staged atom of B: position after rotation and separation, charge
  double x, y, z, w;
};

__global__ void __launch_bounds__(kDirectThreads) k_direct(const void* __restrict__ a, long long na, int dta,
                                                           const void* __restrict__ b, long long nb, int dtb,
                                                           const SysGeom* __restrict__ geo, const double* __restrict__ xf,
                                                           double* __restrict__ part) {
  __shared__ Atom4 sb[kDirectThreads];
  __shared__ double sh[32];
  const double* cA = geo[0].c;
  const double* cB = geo[1].c;
  const double* rot = xf + 12LL * blockIdx.y;  // this item's rotation of B and separation
  const double* R0 = rot + 9;
  part += (long long)blockIdx.y * gridDim.x;
  const long long i = (long long)blockIdx.x * kDirectThreads + threadIdx.x;
  double ax = 0.0, ay = 0.0, az = 0.0, qa = 0.0;
  if (i < na) {
    load_xyz(a, dta, i, ax, ay, az, qa);
    ax -= cA[0];
    ay -= cA[1];
    az -= cA[2];
  }
  double acc = 0.0;
  for (long long j0 = 0; j0 < nb; j0 += kDirectThreads) {
    const long long j = j0 + threadIdx.x;
    Atom4 v{1e300, 1e300, 1e300, 0.0};
    if (j < nb) {
      double x, y, z, q;
      load_xyz(b, dtb, j, x, y, z, q);
      x -= cB[0];
      y -= cB[1];
      z -= cB[2];
      v.x = R0[0] + rot[0] * x + rot[1] * y + rot[2] * z;
      v.y = R0[1] + rot[3] * x + rot[4] * y + rot[5] * z;
      v.z = R0[2] + rot[6] * x + rot[7] * y + rot[8] * z;
      v.w = q;
    }
    __syncthreads();
    sb[threadIdx.x] = v;
    __syncthreads();
    if (i < na) {
      const int cnt = (int)min((long long)kDirectThreads, nb - j0);
      for (int k = 0; k < cnt; ++k) {
        const Atom4 w = sb[k];
        const double dx = w.x - ax, dy = w.y - ay, dz = w.z - az;
        acc += w.w * rsqrt(dx * dx + dy * dy + dz * dz);
      }
    }
  }
  acc = block_sum(acc * qa, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// One CTA per item: each thread sums a contiguous stripe of the item's block partials, then a
// fixed-order block sum.
__global__ void k_direct_final(const double* __restrict__ part, int nblk, double* __restrict__ E) {
  __shared__ double sh[32];
  part += (long long)blockIdx.x * nblk;
  double s = 0.0;
  const int per = (nblk + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  for (int k = b0; k < min(nblk, b0 + per); ++k) s += part[k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) E[blockIdx.x] = s;
}

}  // namespace

// Threads per contraction CTA: the largest per-degree loops have (L+1)^2 iterations, so small
// degrees take smaller CTAs (more of them resident per SM); at least 64, at most 256.
// Threads of a contraction CTA: about one per (l1, l2) pair, up to 256; a batch of fewer than a
// thousand energies at high degree (a few CTAs per SM) takes 512, so that the rotation products
// and the pair loop run in one round and more warps hide the phases' latency.
int contract_threads(int L, long long n_items) {
  const int n = (L + 1) * (L + 1);
  if (n <= 64) return 64;
  if (n <= 128) return 128;
  return (n > 256 && n_items < 1024) ? kContractThreads : 256;
}

int contract_smem_bytes(int L) {
  const int nq = (L + 1) * (L + 2) / 2;
  return (4 * nq + 5 * (L + 1)) * (int)sizeof(double2) + (5 * L + 4 + dpi2_off(L + 1)) * (int)sizeof(double);
}

int rotate_smem_bytes(int L) {
  const int nq = (L + 1) * (L + 2) / 2;
  return (2 * nq + 3 * (L + 1)) * (int)sizeof(double2) + dpi2_off(L + 1) * (int)sizeof(double);
}

// The dynamic shared-memory limit of a kernel: above 48 KB of dynamic plus static shared memory
// a launch needs the raised limit.  These kernels hold at most 8 KB of static shared memory, so
// the limit is set whenever the dynamic part passes 40 KB (on every such launch: the attribute
// is per device, and a call costs far less than the kernels it precedes).
template <typename F>
int raise_smem_limit(F kernel, int dyn) {
  if (dyn <= 40 * 1024) return 0;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess ? 0 : -1;
}

int launch_rotate_moments(const RotDesc* sets, int n_sets, int Lmax_sets, const double* ztab, cudaStream_t s) {
  if (n_sets <= 0) return 0;
  const int smem = rotate_smem_bytes(Lmax_sets);
  if (raise_smem_limit(k_rotate_moments, smem) != 0) return -1;
  k_rotate_moments<<<n_sets, contract_threads(Lmax_sets, n_sets), smem, s>>>(sets, ztab);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_finalize(const MomJob* jobs, int n_jobs, const double* partials, const SysGeom* geoms, const int* imap,
                    const double* fmap, const int* imap_off, const double* syspart, cudaStream_t s) {
  if (n_jobs <= 0) return 0;
  return launch_pdl(k_finalize, dim3(n_jobs), dim3(kFinalizeThreads), 0, s, jobs, partials, geoms, imap, fmap,
                    imap_off, syspart) == cudaSuccess
             ? 0
             : -1;
}

int launch_contract(const PairDesc* items, int n_items, int Lmax_items, const MomJob* jobs, const SysGeom* geoms,
                    const double* ztab, const double* rots, double* E, int32_t* status, double* G, cudaStream_t s) {
  if (n_items <= 0) return 0;
  const int smem = contract_smem_bytes(Lmax_items);
  const int nt = contract_threads(Lmax_items, n_items);
  if (G) {
    if (raise_smem_limit(k_contract<true>, smem) != 0) return -1;
    if (launch_pdl(k_contract<true>, dim3(n_items), dim3(nt), smem, s, items, jobs, geoms, ztab, rots, E, status, G) !=
        cudaSuccess)
      return -1;
  } else {
    if (raise_smem_limit(k_contract<false>, smem) != 0) return -1;
    if (launch_pdl(k_contract<false>, dim3(n_items), dim3(nt), smem, s, items, jobs, geoms, ztab, rots, E, status,
                   (double*)nullptr) != cudaSuccess)
      return -1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int contract_table_size() { return kZ_TOTAL; }

// d^l_{km}(pi/2) for 0 <= k, m <= l: at beta = pi/2 both half-angle factors are 2^(-1/2), so
//   d^l_{km}(pi/2) = 2^-l sqrt((l+k)!(l-k)! / ((l+m)!(l-m)!)) sum_s (-1)^(k-m+s) C(l+m, s) C(l-m, l-k-s),
// an exact integer sum (at most C(2l, l-k) in magnitude) times one square root.
static double dpi2_entry(int l, int k, int m, const long long (*C)[2 * kZN + 1], const long double* fact) {
  long long S = 0;
  for (int s = (m > k ? m - k : 0); s <= l + m && s <= l - k; ++s) {
    const long long t = C[l + m][s] * C[l - m][l - k - s];
    S += ((k - m + s) & 1) ? -t : t;
  }
  const long double r = sqrtl(fact[l + k] * fact[l - k] / (fact[l + m] * fact[l - m]));
  return (double)ldexpl((long double)S * r, -l);
}

void contract_tables(double* t) {
  for (int k = 0; k < kZ_TOTAL; ++k) t[k] = 0.0;
  long double fact[2 * kZN + 2];
  fact[0] = 1.0L;
  for (int k = 1; k < 2 * kZN + 2; ++k) fact[k] = fact[k - 1] * (long double)k;
  for (int k = 0; k < 2 * kZN; ++k) {
    t[kZ_FACT + k] = (double)fact[k];
    t[kZ_FACT2 + k] = (double)(2.0L * fact[k]);
  }
  for (int l = 0; l < kZN; ++l)
    for (int m = 0; m <= l; ++m) t[kZ_ISF + l * kZN + m] = (double)(1.0L / sqrtl(fact[l + m] * fact[l - m]));
  static long long C[2 * kZN + 1][2 * kZN + 1];  // binomials up to C(2 kLmaxMax, .), exact
  for (int n = 0; n <= 2 * kZN; ++n) {
    C[n][0] = 1;
    for (int k = 1; k <= 2 * kZN; ++k) C[n][k] = n == 0 ? 0 : C[n - 1][k - 1] + C[n - 1][k];
  }
  for (int l = 0; l < kZN; ++l)
    for (int k = 0; k <= l; ++k)
      for (int m = 0; m <= l; ++m) t[kZ_DPI2 + dpi2_off(l) + k * dpi2_stride(l) + m] = dpi2_entry(l, k, m, C, fact);
}

int direct_blocks(long long na) { return (int)((na + kDirectThreads - 1) / kDirectThreads); }

int launch_direct(const void* a, long long na, int dta, const void* b, long long nb, int dtb, const SysGeom* geo,
                  const double* xf, int n_items, double* part, int nblk, double* E, cudaStream_t s) {
  for (int i0 = 0; i0 < n_items; i0 += 65535) {  // grid.y limit
    const int n = min(65535, n_items - i0);
    if (nblk > 0) k_direct<<<dim3(nblk, n), kDirectThreads, 0, s>>>(a, na, dta, b, nb, dtb, geo, xf + 12LL * i0,
                                                                    part + (long long)i0 * nblk);
    k_direct_final<<<n, 128, 0, s>>>(part + (long long)i0 * nblk, nblk, E + i0);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tcm
