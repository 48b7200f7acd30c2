// Moment kernels, Eq. (multipole): persistent warps pull warp tiles (job, column chunk,
// atom range); every lane keeps the chunk's accumulators in registers while it walks
// its atoms, then the warp reduces them into one double-precision partial row per tile.  Included by the per-Lmax translation units, which instantiate
// launch_moments_t<T, L> explicitly.
//
// Per atom (after the per-tile transform M = rot / a', a' = scale_radius(a) a power of
// two, and the split centre c = c_hi + c_lo):
//   d   = (x - c_hi) - c_lo                       exact-ish centring in float
//   p   = M d                                     rotation and radius scaling fused
//   rinv = rsqrt(|p|^2) (+ one Newton step in float), u = (p_x + i p_y) rinv,
//   c = p_z rinv, rho = |p|
//   column recurrences of tcm_internal.h, accumulating q rho^l G_lm.
// No trigonometric function and no division is evaluated per atom.
#pragma once

#include <cuda_runtime.h>

#include "tcm_internal.h"

namespace tcm {

template <typename T>
struct MomTraits;
template <>
struct MomTraits<float> {
  static constexpr int kmax = kKmaxF32;  // the largest budget (plan 1)
  static constexpr int row = kKmaxF32;   // partial-row stride of every float plan
  static constexpr int stride = 36;  // row stride (floats) of the transpose buffer: 16-B rows, no LDS.128 conflicts
};
template <>
struct MomTraits<double> {
  static constexpr int kmax = kKmaxF64;
  static constexpr int row = kKmaxF64;
  static constexpr int stride = 34;  // doubles
};

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rsqrtT(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrtT(double x) { return rsqrt(x); }

template <typename T, int L, int KM = MomTraits<T>::kmax>
struct Plan {
  static constexpr int kmax = KM;
  static constexpr int nch = plan_nch(L, kmax);
  __host__ __device__ static constexpr int m0(int c) { return plan_m0(L, kmax, nch, c); }
  __host__ __device__ static constexpr int nacc(int c) { return chunk_off(L, m0(c), m0(c + 1)); }
  __host__ __device__ static constexpr int max_nacc() {
    int mx = 0;
    for (int c = 0; c < nch; ++c) mx = nacc(c) > mx ? nacc(c) : mx;
    return mx;
  }
  __host__ __device__ static constexpr int smem_bytes() {
    return (kThreads / 32) * max_nacc() * MomTraits<T>::stride * (int)sizeof(T);
  }
};

// Pairs: float2 in the float kernels, where the (Re, Im) halves of a complex step go
// through one packed f32x2 instruction; double2 with scalar arithmetic in the double ones.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
template <typename T>
using P2 = typename Pair<T>::type;

__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
template <typename T>
__device__ __forceinline__ P2<T> pair(T a, T b) {
  P2<T> r;
  r.x = a;
  r.y = b;
  return r;
}

// Register state of one column chunk [M0, M1).  The kernels carry H_j = sigma_j G_{m+j}
// (sigma = +, +, -, -, +, +, ... along each column), for which the recurrence reads
//   H_{j+1} = (-1)^j k_{m+j,m} c H_j + H_{j-1}
// without a subtraction.  Complex columns go in pairs (acc_slot in tcm_internal.h): one packed
// multiply (k_a c, k_b c), two packed FMAs for the recurrences of both columns and two packed
// FMAs for their accumulation, 5 packed instructions per two complex steps.  The sign
// sigma_{l-m} is part of the finalisation factor.
template <typename T, int L, int M0, int M1>
struct Regs {
  static constexpr int NC = M1 - M0;
  static constexpr int NACC = chunk_off(L, M0, M1);
  static constexpr int N0 = M0 == 0 ? L + 1 : 0;  // real accumulators of column 0
  static constexpr int NP = (NACC - N0) / 2;      // complex accumulators
  T acc0[N0 > 0 ? N0 : 1];
  P2<T> accp[NP > 0 ? NP : 1];
  T g0, p0;             // column 0: H_j, H_j-1
  P2<T> g[NC], p[NC];   // columns m >= 1
  T dr, di;             // running diagonal power u^m
  T q00, q00e;          // float kernels: Q_00 = sum q as an error-free (sum, error) pair
};

// Q_00 is the total charge: for a neutral system it is a tiny difference of large partial
// sums, and a charged partner multiplies its error by its own charge.  The float kernels
// therefore accumulate it with Knuth's two-sum (the rounding error of every addition goes
// to q00e) and reduce it across the warp in double.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  const float t = s + x;
  const float bb = t - s;
  e += (s - (t - bb)) + (x - bb);
  s = t;
}

// The signed recurrence coefficient of step jj (>= 2) along column m at degree l.
template <typename T, int l, int m>
__device__ __forceinline__ constexpr T kstep() {
  return (T)((((l - m) - 1) & 1) ? -kcoef(l - 1, m) : kcoef(l - 1, m));
}

// Recurrence coefficients as pair operands in constant memory, so that the packed multiply
// (t_a, t_b) = (k_a, k_b) (c, c) reads them straight from the constant bank instead of
// building each pair in registers:
//   two[l][m]  = (k of column m, k of column m + 1) at degree l (1 for column m+1's first
//                step, jj = 1, which is G = c G), for a column pair (m, m+1) with l >= m + 2;
//   one[l][m]  = (k, k) of a single column m at degree l >= m + 2.
template <typename T>
struct KPairs {
  P2<T> two[kLmaxMax + 1][kLmaxMax + 1];
  P2<T> one[kLmaxMax + 1][kLmaxMax + 1];
  constexpr KPairs() : two(), one() {
    for (int l = 0; l <= kLmaxMax; ++l)
      for (int m = 0; m <= kLmaxMax; ++m) {
        if (l < m + 2) continue;
        const T ka = (T)((((l - m) - 1) & 1) ? -kcoef(l - 1, m) : kcoef(l - 1, m));
        const T kb = l == m + 2 ? (T)1 : (T)((((l - m - 1) - 1) & 1) ? -kcoef(l - 1, m + 1) : kcoef(l - 1, m + 1));
        two[l][m].x = ka;
        two[l][m].y = kb;
        one[l][m].x = ka;
        one[l][m].y = ka;
      }
  }
};
static_assert(KPairs<float>().two[5][1].x != 0.0f && KPairs<float>().two[3][1].y == 1.0f,
              "the coefficient table must be a constant expression");
static __constant__ KPairs<float> c_kpairs_f = KPairs<float>();
static __constant__ KPairs<double> c_kpairs_d = KPairs<double>();
template <typename T>
__device__ __forceinline__ const KPairs<T>& kpairs();
template <>
__device__ __forceinline__ const KPairs<float>& kpairs<float>() { return c_kpairs_f; }
template <>
__device__ __forceinline__ const KPairs<double>& kpairs<double>() { return c_kpairs_d; }

// Advance the running diagonal power (dr, di) = u^m to the next column.
template <typename T, int L, int M0, int M1>
__device__ __forceinline__ void next_power(Regs<T, L, M0, M1>& s, T ux, T uy) {
  const T nr = s.dr * ux - s.di * uy;
  const T ni = s.dr * uy + s.di * ux;
  s.dr = nr;
  s.di = ni;
}

// Column 0 (real) at degree l.
template <typename T, int L, int M0, int M1, int l>
__device__ __forceinline__ void col0_step(Regs<T, L, M0, M1>& s, P2<T> cc, P2<T> qq) {
  if constexpr (l == 0) {
    s.g0 = (T)1;
  } else if constexpr (l == 1) {
    s.p0 = s.g0;
    s.g0 = cc.x;
  } else {
    const T t = kstep<T, l, 0>() * cc.x;
    const T n = fmaT(t, s.g0, s.p0);
    s.p0 = s.g0;
    s.g0 = n;
  }
  if constexpr (l == 0 && sizeof(T) == 4)
    two_sum_acc(s.q00, s.q00e, qq.x);  // G_00 = 1
  else
    s.acc0[l] = fmaT(qq.x, s.g0, s.acc0[l]);
}

// A single complex column m at degree l: (Re, Im) in one pair register.
template <typename T, int L, int M0, int M1, int l, int m>
__device__ __forceinline__ void single_step(Regs<T, L, M0, M1>& s, T ux, T uy, P2<T> cc, P2<T> qq) {
  if constexpr (m <= l) {
    constexpr int j = m - M0;
    if constexpr (l == m) {
      if constexpr (m > M0) next_power(s, ux, uy);
      s.g[j] = pair<T>(s.dr, s.di);
    } else if constexpr (l == m + 1) {
      s.p[j] = s.g[j];
      s.g[j] = mul2(cc, s.g[j]);
    } else {
      const P2<T> tt = mul2(cc, kpairs<T>().one[l][m]);
      const P2<T> n = fma2(tt, s.g[j], s.p[j]);
      s.p[j] = s.g[j];
      s.g[j] = n;
    }
    constexpr int a = (acc_slot(L, M0, M1, l, m, 0) - Regs<T, L, M0, M1>::N0) / 2;
    s.accp[a] = fma2(qq, s.g[j], s.accp[a]);
  }
}

// A pair of complex columns (ma, mb = ma + 1) at degree l.  Registers: g[ja] = (Re_a, Re_b),
// g[jb] = (Im_a, Im_b), and the same for the previous level in p.  From l = mb + 1 on one packed
// multiply (k_a c, k_b c) and two packed FMAs advance both columns; column b's first step
// (jj = 1, G = c G) is the general step with k = 1 and a zero previous value.
template <typename T, int L, int M0, int M1, int l, int ma>
__device__ __forceinline__ void pair_step(Regs<T, L, M0, M1>& s, T ux, T uy, P2<T> cc, P2<T> qq) {
  if constexpr (ma <= l) {
    constexpr int ja = ma - M0, jb = ja + 1, mb = ma + 1;
    using R = Regs<T, L, M0, M1>;
    if constexpr (l == ma) {  // seed column a
      if constexpr (ma > M0) next_power(s, ux, uy);
      s.g[ja].x = s.dr;
      s.g[jb].x = s.di;
      constexpr int a = (acc_slot(L, M0, M1, l, ma, 0) - R::N0) / 2;
      s.accp[a].x = fmaT(qq.x, s.dr, s.accp[a].x);
      s.accp[a].y = fmaT(qq.x, s.di, s.accp[a].y);
    } else {
      if constexpr (l == mb) {  // column a: G = c G; column b: seed
        s.p[ja].x = s.g[ja].x;
        s.p[jb].x = s.g[jb].x;
        s.g[ja].x = cc.x * s.g[ja].x;
        s.g[jb].x = cc.x * s.g[jb].x;
        next_power(s, ux, uy);
        s.g[ja].y = s.dr;
        s.g[jb].y = s.di;
        s.p[ja].y = (T)0;
        s.p[jb].y = (T)0;
      } else {
        const P2<T> tt = mul2(cc, kpairs<T>().two[l][ma]);
        const P2<T> nr = fma2(tt, s.g[ja], s.p[ja]);
        const P2<T> ni = fma2(tt, s.g[jb], s.p[jb]);
        s.p[ja] = s.g[ja];
        s.p[jb] = s.g[jb];
        s.g[ja] = nr;
        s.g[jb] = ni;
      }
      constexpr int ar = (acc_slot(L, M0, M1, l, ma, 0) - R::N0) / 2;  // (Re_a, Re_b)
      constexpr int ai = (acc_slot(L, M0, M1, l, ma, 1) - R::N0) / 2;  // (Im_a, Im_b)
      s.accp[ar] = fma2(qq, s.g[ja], s.accp[ar]);
      s.accp[ai] = fma2(qq, s.g[jb], s.accp[ai]);
    }
  }
}

template <typename T, int L, int M0, int M1, int l, int m>
__device__ __forceinline__ void level_cols(Regs<T, L, M0, M1>& s, T ux, T uy, P2<T> cc, P2<T> qq) {
  if constexpr (m < M1) {
    if constexpr (m == 0) {
      col0_step<T, L, M0, M1, l>(s, cc, qq);
      level_cols<T, L, M0, M1, l, 1>(s, ux, uy, cc, qq);
    } else if constexpr (acc_pair_a(M0, M1, m)) {
      pair_step<T, L, M0, M1, l, m>(s, ux, uy, cc, qq);
      level_cols<T, L, M0, M1, l, m + 2>(s, ux, uy, cc, qq);
    } else {
      single_step<T, L, M0, M1, l, m>(s, ux, uy, cc, qq);
      level_cols<T, L, M0, M1, l, m + 1>(s, ux, uy, cc, qq);
    }
  }
}

template <typename T, int L, int M0, int M1, int l>
__device__ __forceinline__ void levels(Regs<T, L, M0, M1>& s, T ux, T uy, P2<T> cc, P2<T> rr, P2<T> qq) {
  level_cols<T, L, M0, M1, l, M0>(s, ux, uy, cc, qq);
  if constexpr (l < L) levels<T, L, M0, M1, l + 1>(s, ux, uy, cc, rr, mul2(qq, rr));
}

// Per-tile transform of the coordinates: centring and rot / a.
template <typename T>
struct Xform {
  T chi[3], clo[3];  // centre split into high and low parts (float path); clo = 0 in double
  T M[9];
};

template <typename T>
__device__ __forceinline__ Xform<T> make_xform(const MomJob& job, const SysGeom& g) {
  Xform<T> x;
  const double ia = 1.0 / scale_radius(g.a);  // exact: a power of two
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // float: the centre's split from the geometry record
    x.chi[k] = sizeof(T) == 4 ? (T)g.chi[k] : (T)g.c[k];
    x.clo[k] = sizeof(T) == 4 ? (T)g.clo[k] : (T)0;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) x.M[k] = (T)(job.rot[k] * ia);
  return x;
}

// Centred coordinates of one atom record.  The input type is a template parameter so that
// the atom loop never carries the other type's instructions (a runtime test inside the
// loop is if-converted, and the idle double path still occupies the FP64 pipe).
template <typename T>
__device__ __forceinline__ void centre(const float4& v, const Xform<T>& xf, const double*, T& d0, T& d1, T& d2, T& q) {
  d0 = ((T)v.x - xf.chi[0]) - xf.clo[0];
  d1 = ((T)v.y - xf.chi[1]) - xf.clo[1];
  d2 = ((T)v.z - xf.chi[2]) - xf.clo[2];
  q = (T)v.w;
}
struct Rec64 {
  double2 a, b;
};
template <typename T>
__device__ __forceinline__ void centre(const Rec64& v, const Xform<T>&, const double* cd, T& d0, T& d1, T& d2, T& q) {
  d0 = (T)(v.a.x - cd[0]);
  d1 = (T)(v.a.y - cd[1]);
  d2 = (T)(v.b.x - cd[2]);
  q = (T)v.b.y;
}
__device__ __forceinline__ float4 load_rec(const float4* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ Rec64 load_rec(const Rec64* p, long long i) {
  const double2* q = reinterpret_cast<const double2*>(p + i);
  return Rec64{__ldg(q), __ldg(q + 1)};
}

// (u_x, u_y, c, rho) of the centred atom in the scaled, rotated frame.
template <typename T>
__device__ __forceinline__ void setup(T d0, T d1, T d2, const Xform<T>& xf, T& ux, T& uy, T& cz, T& rho) {
  const T px = fmaT(xf.M[0], d0, fmaT(xf.M[1], d1, xf.M[2] * d2));
  const T py = fmaT(xf.M[3], d0, fmaT(xf.M[4], d1, xf.M[5] * d2));
  const T pz = fmaT(xf.M[6], d0, fmaT(xf.M[7], d1, xf.M[8] * d2));
  const T r2 = fmaT(px, px, fmaT(py, py, pz * pz));
  T rinv = r2 > (T)0 ? rsqrtT(r2) : (T)0;
  if constexpr (sizeof(T) == 4) {  // one Newton step: the hardware rsqrt is a few ulp off
    const T h = r2 * rinv;
    rinv = fmaT(fmaT(-h, rinv, (T)1), (T)0.5 * rinv, rinv);
  }
  ux = px * rinv;
  uy = py * rinv;
  cz = pz * rinv;
  rho = r2 * rinv;
}

// Sum of a 32-entry row of the transpose buffer in a fixed tree order, compensated: every
// addition is an error-free two-sum whose rounding error is carried along, so the float row
// sum keeps about 48 bits (a plain float tree would add about 2 x 2^-24 of the row's
// magnitude).  Float instructions only: on GB300 the FP64 pipe runs at 1/64 of the FP32 rate,
// and a double tree (with its conversions) held the warps at the end of every tile.
__device__ __forceinline__ void two_sum_ff(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ double row_sum32(const float* p) {
  const float4* v = reinterpret_cast<const float4*>(p);
  float s[8], e[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 w = v[k];
    float a, ea, b, eb;
    two_sum_ff(w.x, w.y, a, ea);
    two_sum_ff(w.z, w.w, b, eb);
    two_sum_ff(a, b, s[k], e[k]);
    e[k] += ea + eb;
  }
#pragma unroll
  for (int h = 4; h >= 1; h >>= 1)
#pragma unroll
    for (int k = 0; k < h; ++k) {
      float t, et;
      two_sum_ff(s[k], s[k + h], t, et);
      e[k] = (e[k] + e[k + h]) + et;
      s[k] = t;
    }
  return (double)s[0] + (double)e[0];
}

__device__ __forceinline__ double row_sum32(const double* p) {
  const double2* v = reinterpret_cast<const double2*>(p);
  double s[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double2 w0 = v[2 * k], w1 = v[2 * k + 1];
    s[k] = (w0.x + w0.y) + (w1.x + w1.y);
  }
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// Warp reduction of the per-lane accumulators into one double row `out[0..NACC)` (the
// column-0 reals first, then the complex pairs, in slot order).  The warp transposes its
// 32 x NACC block through its own shared-memory region and every lane tree-sums whole rows
// (fixed order, compensated) and stores them in double.  No CTA barrier is involved.
template <typename T, int L, int M0, int M1>
__device__ __forceinline__ void warp_reduce_store(const Regs<T, L, M0, M1>& s, T* wb, double* out) {
  using R = Regs<T, L, M0, M1>;
  constexpr int NACC = R::NACC;
  constexpr int S = MomTraits<T>::stride;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < R::N0; ++k) wb[k * S + lane] = s.acc0[k];
#pragma unroll
  for (int k = 0; k < R::NP; ++k) {
    wb[(R::N0 + 2 * k) * S + lane] = s.accp[k].x;
    wb[(R::N0 + 2 * k + 1) * S + lane] = s.accp[k].y;
  }
  __syncwarp();
#pragma unroll
  for (int rr = 0; rr < (NACC + 31) / 32; ++rr) {
    const int r = lane + 32 * rr;
    if (r < NACC) out[r] = row_sum32(wb + r * S);
  }
  if constexpr (M0 == 0 && sizeof(T) == 4) {  // slot 0 is Q_00: exact lane pairs summed in double
    double v = (double)s.q00 + (double)s.q00e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[0] = v;
  }
  __syncwarp();
}

// u^E by repeated squaring (E a compile-time constant >= 1).
template <typename T, int E>
__device__ __forceinline__ void upow(T ux, T uy, T& pr, T& pi) {
  if constexpr (E == 1) {
    pr = ux;
    pi = uy;
  } else if constexpr (E % 2 == 0) {
    T hr, hi;
    upow<T, E / 2>(ux, uy, hr, hi);
    pr = fmaT(hr, hr, -(hi * hi));
    pi = (T)2 * hr * hi;
  } else {
    T hr, hi;
    upow<T, E - 1>(ux, uy, hr, hi);
    pr = fmaT(hr, ux, -(hi * uy));
    pi = fmaT(hr, uy, hi * ux);
  }
}

// Walks this lane's atoms of the warp tile [i0, i1), the next record prefetched while the
// current one is processed.
template <typename T, int L, int M0, int M1, typename Rec>
__device__ __forceinline__ void atom_loop(Regs<T, L, M0, M1>& s, const Rec* __restrict__ xyzq, long long i0,
                                          long long i1, const Xform<T>& xf, const double* cd) {
  long long i = i0 + (threadIdx.x & 31);
  if (i >= i1) return;
  Rec nxt = load_rec(xyzq, i);
  for (; i < i1; i += 32) {
    const Rec cur = nxt;
    if (i + 32 < i1) nxt = load_rec(xyzq, i + 32);
    T d0, d1, d2, q, ux, uy, cz, rho;
    centre<T>(cur, xf, cd, d0, d1, d2, q);
    if constexpr (M0 == 0 && sizeof(T) == 4 && sizeof(Rec) == 32)
      s.q00e += (T)(cur.b.y - (double)q);  // double input: keep the charge's rounding remainder in Q_00
    setup<T>(d0, d1, d2, xf, ux, uy, cz, rho);
    const P2<T> cc = pair<T>(cz, cz), rr = pair<T>(rho, rho), qq = pair<T>(q, q);
    if constexpr (M0 == 0) {
      s.dr = (T)1;
      s.di = (T)0;
    } else {
      upow<T, M0>(ux, uy, s.dr, s.di);  // the chunk's first column starts at u^M0
    }
    levels<T, L, M0, M1, 0>(s, ux, uy, cc, rr, qq);
  }
}

template <typename T, int L, int M0, int M1>
__device__ __forceinline__ void run_chunk(const MomTile& tile, const MomJob* __restrict__ jobs,
                                          const SysGeom* __restrict__ geoms, double* __restrict__ partials, T* wb,
                                          Xform<T>* xf_w) {
  using R = Regs<T, L, M0, M1>;
  const MomJob& job = jobs[tile.job];
  const SysGeom g = geoms[job.geom];
  if ((threadIdx.x & 31) == 0) *xf_w = make_xform<T>(job, g);  // double math once per tile
  __syncwarp();
  const Xform<T> xf = *xf_w;
  const long long n = job.n;
  const long long i0 = (long long)tile.t * job.atoms_per_tile;
  const long long i1 = min(n, i0 + (long long)job.atoms_per_tile);
  const void* xyzq = job.xyzq;
  const int dtype = job.dtype;
  R s;
  s.q00 = s.q00e = (T)0;
#pragma unroll
  for (int k = 0; k < R::N0; ++k) s.acc0[k] = (T)0;
#pragma unroll
  for (int k = 0; k < R::NP; ++k) s.accp[k] = pair<T>((T)0, (T)0);
  if (dtype == TCM_F32)
    atom_loop<T, L, M0, M1>(s, reinterpret_cast<const float4*>(xyzq), i0, i1, xf, g.c);
  else
    atom_loop<T, L, M0, M1>(s, reinterpret_cast<const Rec64*>(xyzq), i0, i1, xf, g.c);
  warp_reduce_store<T, L, M0, M1>(s, wb, partials + (long long)tile.id * MomTraits<T>::row);
}

template <typename T, int L, int C, int KM>
__device__ __forceinline__ void run_tile(const MomTile& tile, const MomJob* __restrict__ jobs,
                                         const SysGeom* __restrict__ geoms, double* __restrict__ partials, T* wb,
                                         Xform<T>* xf_w) {
  using P = Plan<T, L, KM>;
  if constexpr (C < P::nch) {
    if (tile.chunk == C)
      run_chunk<T, L, P::m0(C), P::m0(C + 1)>(tile, jobs, geoms, partials, wb, xf_w);
    else
      run_tile<T, L, C + 1, KM>(tile, jobs, geoms, partials, wb, xf_w);
  }
}

// Code of the tile's own degree: a chain of compile-time degrees, one compare per degree.
template <typename T, int L, int KM>
__device__ __forceinline__ void run_tile_any(int Lt, const MomTile& tile, const MomJob* __restrict__ jobs,
                                             const SysGeom* __restrict__ geoms, double* __restrict__ partials, T* wb,
                                             Xform<T>* xf_w) {
  if constexpr (L <= kLmaxMax) {
    if (Lt == L)
      run_tile<T, L, 0, KM>(tile, jobs, geoms, partials, wb, xf_w);
    else
      run_tile_any<T, L + 1, KM>(Lt, tile, jobs, geoms, partials, wb, xf_w);
  }
}

// Persistent kernel: every warp pulls warp tiles from the shared counter until none are
// left, so warps never wait for each other.  counter[0] is the work counter and counter[32]
// the exit ticket, both zero on entry and left zero on exit.  LK >= 0: every tile has degree
// LK; LK < 0: the tiles may have any degree (one launch for a whole uneven batch), each runs
// the code of its job's degree.  KM: the accumulator budget of the chunk plan.
template <typename T, int LK, int KM>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? moment_ctas(KM) : TCM_MOMENT_CTAS_PER_SM)
    k_moments(const MomJob* __restrict__ jobs, const MomTile* __restrict__ tiles, int n_tiles,
              int* __restrict__ counter, const SysGeom* __restrict__ geoms, double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Xform<T> s_xf[kThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kRow = LK >= 0 ? Plan<T, (LK >= 0 ? LK : 0), KM>::max_nacc() : KM;
  T* wb = reinterpret_cast<T*>(smem) + warp * (kRow * MomTraits<T>::stride);
  pdl_wait();  // the centres and radii of the launch before are complete
  for (;;) {
    int ti = 0;
    if (lane == 0) ti = atomicAdd(counter, 1);
    ti = __shfl_sync(0xffffffffu, ti, 0);
    if (ti >= n_tiles) break;
    const MomTile tile = tiles[ti];
    if constexpr (LK >= 0)
      run_tile<T, LK, 0, KM>(tile, jobs, geoms, partials, wb, &s_xf[warp]);
    else
      run_tile_any<T, 0, KM>(jobs[tile.job].L, tile, jobs, geoms, partials, wb, &s_xf[warp]);
  }
  // the last warp out leaves the work counter and its own ticket at zero for the next launch
  if (lane == 0 && atomicAdd(counter + 32, 1) == (int)(gridDim.x * (kThreads / 32)) - 1) {
    atomicExch(counter, 0);
    atomicExch(counter + 32, 0);
  }
}

template <typename T, int LK, int KM>
int launch_moments_t(const MomJob* jobs, const MomTile* tiles, int n_tiles, int* counter,
                     const SysGeom* geoms, double* partials, int grid, cudaStream_t s) {
  constexpr int smem = (kThreads / 32) * (LK >= 0 ? Plan<T, (LK >= 0 ? LK : 0), KM>::max_nacc() : KM) *
                       MomTraits<T>::stride * (int)sizeof(T);
  if (smem > 40 * 1024) {  // with the kernel's static shared memory (under 1 KB) it may pass 48 KB
    if (cudaFuncSetAttribute(k_moments<T, LK, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return -1;
  }
  return launch_pdl(k_moments<T, LK, KM>, dim3(grid), dim3(kThreads), smem, s, jobs, tiles, n_tiles, counter, geoms,
                    partials) == cudaSuccess
             ? 0
             : -1;
}

}  // namespace tcm
