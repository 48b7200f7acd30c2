// Kernels around the moment pass:
//   a1  centre and radius of a system (Section II: any centre; the centroid by default)
//   a3  cross-tile reduction of the moment partials in double, fixed order, plus the
//       deferred normalisation F_lm a^l                                  (Eq. (multipole))
//   a4  irregular solid harmonics of the separation vector R0            (Eq. (Formula))
//   a5  two-center contraction in double                                 (Eq. (Formula))
//   a6  exact pairwise Coulomb sum in double                             (Eq. (Coulomb))
#include <cuda_runtime.h>

#include "tcm_internal.h"

namespace tcm {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
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
__device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_max(r);
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

constexpr int kGeomThreads = 256;

// a1, pass 1: per-tile sums of the coordinates (double).
__global__ void __launch_bounds__(kGeomThreads) k_geom_sum(const GeomJob* __restrict__ gj,
                                                           const GeomTile* __restrict__ gt,
                                                           double* __restrict__ gpart) {
  __shared__ double sh[32];
  const GeomTile tile = gt[blockIdx.x];
  const GeomJob j = gj[tile.gjob];
  const long long i0 = (long long)tile.t * kGeomTileAtoms;
  const long long i1 = min(j.n, i0 + (long long)kGeomTileAtoms);
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kGeomThreads) {
    double x, y, z, q;
    load_xyz(j.xyzq, j.dtype, i, x, y, z, q);
    sx += x;
    sy += y;
    sz += z;
  }
  sx = block_sum(sx, sh);
  sy = block_sum(sy, sh);
  sz = block_sum(sz, sh);
  if (threadIdx.x == 0) {
    double* o = gpart + 4LL * (j.tile_base + tile.t);
    o[0] = sx;
    o[1] = sy;
    o[2] = sz;
  }
}

// a1, pass 2: centroid from the tile sums (fixed order), one thread per system.
__global__ void k_geom_center(const GeomJob* __restrict__ gj, int n, const double* __restrict__ gpart,
                              SysGeom* __restrict__ geoms) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const GeomJob j = gj[k];
  if (!j.need_center) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int t = 0; t < j.n_tiles; ++t)
    for (int d = 0; d < 3; ++d) s[d] += gpart[4LL * (j.tile_base + t) + d];
  const double inv = j.n > 0 ? 1.0 / (double)j.n : 0.0;
  for (int d = 0; d < 3; ++d) geoms[j.geom].c[d] = s[d] * inv;
}

// a1, pass 3: per-tile max of |x - c|^2.
__global__ void __launch_bounds__(kGeomThreads) k_geom_rmax(const GeomJob* __restrict__ gj,
                                                            const GeomTile* __restrict__ gt,
                                                            const SysGeom* __restrict__ geoms,
                                                            double* __restrict__ gpart) {
  __shared__ double sh[32];
  const GeomTile tile = gt[blockIdx.x];
  const GeomJob j = gj[tile.gjob];
  const double cx = geoms[j.geom].c[0], cy = geoms[j.geom].c[1], cz = geoms[j.geom].c[2];
  const long long i0 = (long long)tile.t * kGeomTileAtoms;
  const long long i1 = min(j.n, i0 + (long long)kGeomTileAtoms);
  double mx = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kGeomThreads) {
    double x, y, z, q;
    load_xyz(j.xyzq, j.dtype, i, x, y, z, q);
    const double dx = x - cx, dy = y - cy, dz = z - cz;
    mx = fmax(mx, dx * dx + dy * dy + dz * dz);
  }
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) gpart[4LL * (j.tile_base + tile.t) + 3] = mx;
}

// a1, pass 4: radius.
__global__ void k_geom_radius(const GeomJob* __restrict__ gj, int n, const double* __restrict__ gpart,
                              SysGeom* __restrict__ geoms) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const GeomJob j = gj[k];
  if (!j.need_radius) return;
  double mx = 0.0;
  for (int t = 0; t < j.n_tiles; ++t) mx = fmax(mx, gpart[4LL * (j.tile_base + t) + 3]);
  geoms[j.geom].a = sqrt(mx);
}

// a3: one CTA per moment job.  Sums the job's tile partials of each component in
// tile order (double) and applies F_lm a^l.  cmap[cmap_off[L] + p] = (chunk, slot)
// of packed component p.
__global__ void __launch_bounds__(256) k_finalize(const MomJob* __restrict__ jobs, const double* __restrict__ partials,
                                                  const SysGeom* __restrict__ geoms, const int2* __restrict__ cmap,
                                                  const int* __restrict__ cmap_off, const double* __restrict__ ftab,
                                                  int kmax) {
  __shared__ double apow[kLmaxMax + 1];
  const MomJob& job = jobs[blockIdx.x];
  const int L = job.L;
  const int tpc = job.tiles_per_chunk;
  const double a = scale_radius(geoms[job.geom].a);  // the moment kernels scaled by 1/a
  if (threadIdx.x <= L) {
    double p = 1.0;
    for (int k = 0; k < (int)threadIdx.x; ++k) p *= a;
    apow[threadIdx.x] = p;
  }
  __syncthreads();
  const int ncomp = (L + 1) * (L + 1);
  const int2* map = cmap + cmap_off[L];
  for (int p = threadIdx.x; p < ncomp; p += blockDim.x) {
    const int2 cs = map[p];
    const double* base = partials + (long long)(job.tile_base + cs.x * tpc) * kmax + cs.y;
    double s = 0.0;
    for (int t = 0; t < tpc; ++t) s += base[(long long)t * kmax];
    int l = (int)sqrt((double)p);
    while (l * l > p) --l;
    while ((l + 1) * (l + 1) <= p) ++l;
    const int r = p - l * l;
    const int m = (r + 1) >> 1;
    job.out[p] = ftab[l * (kLmaxMax + 1) + m] * apow[l] * s;
  }
}

// a4 + a5: one CTA per energy.
//   Qhat_lm = Q_lm / sqrt((l+m)! (l-m)!)                    (m >= 0, complex)
//   J_LM    = (-1)^M (L-M)! P_L^M(cos t) e^{-i M p} / R^{L+1}  (L <= 2 Lmax, M >= 0)
//           = sqrt((L+M)!(L-M)!) sqrt(4pi/(2L+1)) Y*_LM(R0hat) / R^{L+1}
// With the stretched 3j symbol (L = l1 + l2) Eq. (Formula) becomes
//   U = sum (-1)^l2 Qhat^A_l1m1 Qhat^B_l2m2 J_{l1+l2, m1+m2},
// and for real charges Qhat_l,-m = (-1)^m conj(Qhat_lm), J_L,-M = (-1)^M conj(J_LM),
// so U = sum_{l1, m1>=0} w_m1 Re(Qhat^A_l1m1 V_l1m1) with w = 1 (m1 = 0) or 2.
// J is built by the recurrences
//   J_00 = 1/R,  J_k+1,k+1 = -(2k+1) (x - iy)/R^2 J_kk,
//   J_M+1,M = (2M+1) z J_MM / R^2,
//   J_L+1,M = ((2L+1) z J_LM - (L^2 - M^2) J_L-1,M) / R^2.
constexpr int kContractThreads = 256;

__global__ void __launch_bounds__(kContractThreads) k_contract(const PairDesc* __restrict__ items,
                                                               const MomJob* __restrict__ jobs,
                                                               const SysGeom* __restrict__ geoms,
                                                               const double* __restrict__ isf,
                                                               double* __restrict__ E, int32_t* __restrict__ status) {
  extern __shared__ double2 sm2[];
  __shared__ double sh[32];
  const PairDesc d = items[blockIdx.x];
  const int L = d.L;
  const double x = d.R0[0], y = d.R0[1], z = d.R0[2];
  const double R2 = x * x + y * y + z * z;
  const double R = sqrt(R2);
  const double aA = geoms[d.geomA].a, aB = geoms[d.geomB].a;
  if (!(R > aA + aB)) {  // Eq. (mainCond) violated: the expansion does not converge
    if (threadIdx.x == 0) {
      E[blockIdx.x] = __longlong_as_double(0x7ff8000000000000LL);
      if (status) status[blockIdx.x] = TCM_ENOTCONV;
    }
    return;
  }
  const int nq = (L + 1) * (L + 2) / 2;
  const int LL = 2 * L;
  double2* qa = sm2;
  double2* qb = sm2 + nq;
  double2* J = sm2 + 2 * nq;
  const double* pa = jobs[d.jobA].out;
  const double* pb = jobs[d.jobB].out;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    int l = (int)((sqrt(8.0 * k + 1.0) - 1.0) * 0.5);
    while (l * (l + 1) / 2 > k) --l;
    while ((l + 1) * (l + 2) / 2 <= k) ++l;
    const int m = k - l * (l + 1) / 2;
    const double f = isf[l * (kLmaxMax + 1) + m];
    if (m == 0) {
      qa[k] = make_double2(pa[l * l] * f, 0.0);
      qb[k] = make_double2(pb[l * l] * f, 0.0);
    } else {
      qa[k] = make_double2(pa[l * l + 2 * m - 1] * f, pa[l * l + 2 * m] * f);
      qb[k] = make_double2(pb[l * l + 2 * m - 1] * f, pb[l * l + 2 * m] * f);
    }
  }
  const double iR2 = 1.0 / R2;
  for (int M = threadIdx.x; M <= LL; M += blockDim.x) {
    double jr = 1.0 / R, ji = 0.0;
    const double wr = x * iR2, wi = -y * iR2;  // (x - iy) / R^2
    for (int k = 0; k < M; ++k) {
      const double f = -(2.0 * k + 1.0);
      const double nr = f * (jr * wr - ji * wi);
      const double ni = f * (jr * wi + ji * wr);
      jr = nr;
      ji = ni;
    }
    J[M * (M + 1) / 2 + M] = make_double2(jr, ji);
    if (M + 1 <= LL) {
      double pr = jr, pi = ji;
      const double f = (2.0 * M + 1.0) * z * iR2;
      double cr = f * jr, ci = f * ji;
      J[(M + 1) * (M + 2) / 2 + M] = make_double2(cr, ci);
      for (int Lp = M + 1; Lp < LL; ++Lp) {
        const double a1 = (2.0 * Lp + 1.0) * z * iR2;
        const double a2 = (double)(Lp * Lp - M * M) * iR2;
        const double nr = a1 * cr - a2 * pr;
        const double ni = a1 * ci - a2 * pi;
        pr = cr;
        pi = ci;
        cr = nr;
        ci = ni;
        J[(Lp + 1) * (Lp + 2) / 2 + M] = make_double2(cr, ci);
      }
    }
  }
  __syncthreads();
  // Work items (l1, m1 >= 0, l2): T = sum_m2 Qhat^B_l2m2 J_{l1+l2, m1+m2}.
  const int nwork = nq * (L + 1);
  double acc = 0.0;
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    const int k1 = w / (L + 1);
    const int l2 = w - k1 * (L + 1);
    int l1 = (int)((sqrt(8.0 * k1 + 1.0) - 1.0) * 0.5);
    while (l1 * (l1 + 1) / 2 > k1) --l1;
    while ((l1 + 1) * (l1 + 2) / 2 <= k1) ++l1;
    const int m1 = k1 - l1 * (l1 + 1) / 2;
    const int Lp = l1 + l2;
    const double2* Jr = J + Lp * (Lp + 1) / 2;
    const double2* qr = qb + l2 * (l2 + 1) / 2;
    double2 b = qr[0];
    double2 j = Jr[m1];
    double tr = b.x * j.x - b.y * j.y;
    double ti = b.x * j.y + b.y * j.x;
    for (int m2 = 1; m2 <= l2; ++m2) {
      b = qr[m2];
      j = Jr[m1 + m2];  // + m2
      tr += b.x * j.x - b.y * j.y;
      ti += b.x * j.y + b.y * j.x;
      // - m2: Qhat^B_l2,-m2 = (-1)^m2 conj(b)
      if (m2 <= m1) {  // J_{L, m1-m2}, non-negative order
        j = Jr[m1 - m2];
        const double s = (m2 & 1) ? -1.0 : 1.0;
        tr += s * (b.x * j.x + b.y * j.y);
        ti += s * (b.x * j.y - b.y * j.x);
      } else {  // J_{L, m1-m2} = (-1)^(m2-m1) conj(J_{L, m2-m1}); total sign (-1)^m1 conj(b j)
        j = Jr[m2 - m1];
        const double s = (m1 & 1) ? -1.0 : 1.0;
        tr += s * (b.x * j.x - b.y * j.y);
        ti -= s * (b.x * j.y + b.y * j.x);
      }
    }
    const double2 a = qa[k1];
    const double re = a.x * tr - a.y * ti;
    const double wgt = (m1 > 0 ? 2.0 : 1.0) * ((l2 & 1) ? -1.0 : 1.0);
    acc += wgt * re;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    E[blockIdx.x] = acc;
    if (status) status[blockIdx.x] = TCM_OK;
  }
}

// a6: exact pairwise sum.  One thread per atom of A; B staged through shared memory
// already rotated and translated: b' = R0 + rot (x_b - c_B).  Double precision.
constexpr int kDirectThreads = 256;

__global__ void __launch_bounds__(kDirectThreads) k_direct(const void* __restrict__ a, long long na, int dta,
                                                           const void* __restrict__ b, long long nb, int dtb,
                                                           const SysGeom* __restrict__ geo, const double* __restrict__ xf,
                                                           double* __restrict__ part) {
  __shared__ double4 sb[kDirectThreads];
  __shared__ double sh[32];
  const double* cA = geo[0].c;
  const double* cB = geo[1].c;
  const double* rot = xf;
  const double* R0 = xf + 9;
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
    double4 v = make_double4(1e300, 1e300, 1e300, 0.0);
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
        const double4 w = sb[k];
        const double dx = w.x - ax, dy = w.y - ay, dz = w.z - az;
        acc += w.w * rsqrt(dx * dx + dy * dy + dz * dz);
      }
    }
  }
  acc = block_sum(acc * qa, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_direct_final(const double* __restrict__ part, int nblk, double* __restrict__ E) {
  __shared__ double sh[32];
  double s = 0.0;
  // each thread sums a contiguous stripe, then a fixed-order block sum
  const int per = (nblk + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  for (int k = b0; k < min(nblk, b0 + per); ++k) s += part[k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *E = s;
}

}  // namespace

int launch_geom(const GeomJob* gjobs, int n_gjobs, const GeomTile* gtiles, int n_gtiles, double* gpart,
                SysGeom* geoms, cudaStream_t s) {
  if (n_gjobs <= 0) return 0;
  const int nb = (n_gjobs + 127) / 128;
  k_geom_sum<<<n_gtiles, kGeomThreads, 0, s>>>(gjobs, gtiles, gpart);
  k_geom_center<<<nb, 128, 0, s>>>(gjobs, n_gjobs, gpart, geoms);
  k_geom_rmax<<<n_gtiles, kGeomThreads, 0, s>>>(gjobs, gtiles, geoms, gpart);
  k_geom_radius<<<nb, 128, 0, s>>>(gjobs, n_gjobs, gpart, geoms);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_finalize(const MomJob* jobs, int n_jobs, const double* partials, const SysGeom* geoms, const int2* cmap,
                    const int* cmap_off, const double* ftab, int kmax, cudaStream_t s) {
  if (n_jobs <= 0) return 0;
  k_finalize<<<n_jobs, 256, 0, s>>>(jobs, partials, geoms, cmap, cmap_off, ftab, kmax);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_contract(const PairDesc* items, int n_items, int Lmax_items, const MomJob* jobs, const SysGeom* geoms,
                    const double* isf, double* E, int32_t* status, cudaStream_t s) {
  if (n_items <= 0) return 0;
  const int nq = (Lmax_items + 1) * (Lmax_items + 2) / 2;
  const int nj = (2 * Lmax_items + 1) * (2 * Lmax_items + 2) / 2;
  const int smem = (2 * nq + nj) * (int)sizeof(double2);
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return -1;
  }
  k_contract<<<n_items, kContractThreads, smem, s>>>(items, jobs, geoms, isf, E, status);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int direct_blocks(long long na) { return (int)((na + kDirectThreads - 1) / kDirectThreads); }

int launch_direct(const void* a, long long na, int dta, const void* b, long long nb, int dtb, const SysGeom* geo,
                  const double* xf, double* part, int nblk, double* E, cudaStream_t s) {
  if (nblk > 0) k_direct<<<nblk, kDirectThreads, 0, s>>>(a, na, dta, b, nb, dtb, geo, xf, part);
  k_direct_final<<<1, 256, 0, s>>>(part, nblk, E);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tcm
