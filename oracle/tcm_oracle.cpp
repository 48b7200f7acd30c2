// Plain CPU oracle for the two-center multipole (TCM) method.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
// calls this file; only the tests, the package's smoke check and the CPU
// baseline leg of the benchmark do.  It shares no code, header, table or
// constant generator with the CUDA path.
//
// Everything is written out from the definitions in the paper, in double
// precision, with Neumaier-compensated sums and a long-double factorial table
// for the coupling coefficients:
//   * Eq. (Coulomb)  : exact pairwise energy U = sum_ij q_i q_j / |R0 + r_j - r_i|
//   * Eq. (multipole): Q_lm = sum_i q_i r_i^l sqrt(4 pi/(2l+1)) Y_lm(theta_i, phi_i)
//   * Eq. (3j)       : Wigner 3j symbols from the general Racah sum
//   * Eq. (Formula)  : U_mult = sum_{l1,l2<=Lmax} sum_{m1,m2} (-1)^(l1+M) R0^-(L+1)
//                        sqrt(4 pi (2L)! / ((2l1)! (2l2)!)) 3j(l1 l2 L; m1 m2 -M)
//                        Q^A_l1m1 Q^B_l2m2 Y*_LM(R0hat),  L = l1+l2, M = m1+m2
// Spherical harmonics are orthonormal with the Condon-Shortley phase (the
// convention of Varshalovich, which the paper follows); Y_lm for m >= 0 comes
// from std::sph_legendre and Y_l,-m = (-1)^m conj(Y_lm).
//
// Readings of the paper taken here:
//   * moments use Y_lm (not its conjugate), as Eq. (multipole) prints them, and
//     the separation harmonic is conjugated, as Eq. (Formula) prints it;
//   * l1 and l2 each run over 0..Lmax independently (square truncation), so L
//     reaches 2 Lmax (Section II, text after Eq. (Formula));
//   * the centre of a system is the centroid of its positions with unit
//     masses unless the caller gives one (Section II allows any point);
//   * a rotation of a system acts about its centre: r' = Rot (x - c).
//
// Complex moments are exchanged as two arrays (re, im) of (L+1)^2 values
// indexed l*l + l + m for m = -l..l.
//
// Build: g++ -std=c++17 -O2 -fPIC -shared -ffp-contract=off (see build.py).
// -ffp-contract=off keeps the arithmetic identical on x86-64 and aarch64.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

// Neumaier (improved Kahan) compensated sum.
struct CSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// n! in long double for 0 <= n <= 400 (filled once).
struct FactTable {
  long double f[401];
  FactTable() {
    f[0] = 1.0L;
    for (int n = 1; n <= 400; ++n) f[n] = f[n - 1] * (long double)n;
  }
};
const FactTable& facts() {
  static FactTable t;
  return t;
}
long double fact(int n) { return facts().f[n]; }

// Orthonormal Y_lm(theta, phi) with Condon-Shortley phase, any m in [-l, l].
void ylm(int l, int m, double theta, double phi, double* re, double* im) {
  int am = m < 0 ? -m : m;
  double p = std::sph_legendre((unsigned)l, (unsigned)am, theta);  // Y_l|m|(theta, 0)
  double cr = p * std::cos(am * phi), ci = p * std::sin(am * phi);
  if (m < 0) {  // Y_l,-m = (-1)^m conj(Y_lm)
    double sgn = (am % 2) ? -1.0 : 1.0;
    cr = sgn * cr;
    ci = -sgn * ci;
  }
  *re = cr;
  *im = ci;
}

// Wigner 3j symbol by the Racah sum (general formula, any admissible arguments).
double threej(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  long double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) /
                    fact(j1 + j2 + j3 + 1);
  long double pre = tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                    fact(j3 + m3) * fact(j3 - m3);
  int kmin = 0;
  if (j2 - j3 - m1 > kmin) kmin = j2 - j3 - m1;
  if (j1 - j3 + m2 > kmin) kmin = j1 - j3 + m2;
  int kmax = j1 + j2 - j3;
  if (j1 - m1 < kmax) kmax = j1 - m1;
  if (j2 + m2 < kmax) kmax = j2 + m2;
  long double sum = 0.0L;
  for (int k = kmin; k <= kmax; ++k) {
    long double den = fact(k) * fact(j3 - j2 + k + m1) * fact(j3 - j1 + k - m2) *
                      fact(j1 + j2 - j3 - k) * fact(j1 - k - m1) * fact(j2 - k + m2);
    sum += ((k % 2) ? -1.0L : 1.0L) / den;
  }
  int ph = j1 - j2 - m3;
  long double sgn = (((ph % 2) + 2) % 2) ? -1.0L : 1.0L;
  return (double)(sgn * std::sqrt(pre) * sum);
}

// Position of atom i relative to the centre, optionally rotated about it.
void rel_pos(const double* xyzq, int64_t i, const double* c, const double* rot, double* r) {
  double d[3] = {xyzq[4 * i + 0] - c[0], xyzq[4 * i + 1] - c[1], xyzq[4 * i + 2] - c[2]};
  if (rot) {
    for (int a = 0; a < 3; ++a) r[a] = rot[3 * a + 0] * d[0] + rot[3 * a + 1] * d[1] + rot[3 * a + 2] * d[2];
  } else {
    r[0] = d[0];
    r[1] = d[1];
    r[2] = d[2];
  }
}

int idx(int l, int m) { return l * l + l + m; }

}  // namespace

extern "C" {

int oracle_abi_version(void) { return 1; }

// Centre = centroid of positions (unit masses); radius a = max_i |x_i - c|.
void oracle_center_radius(int64_t n, const double* xyzq, double* center, double* radius) {
  CSum sx, sy, sz;
  for (int64_t i = 0; i < n; ++i) {
    sx.add(xyzq[4 * i + 0]);
    sy.add(xyzq[4 * i + 1]);
    sz.add(xyzq[4 * i + 2]);
  }
  double inv = n > 0 ? 1.0 / (double)n : 0.0;
  center[0] = sx.value() * inv;
  center[1] = sy.value() * inv;
  center[2] = sz.value() * inv;
  double a = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double dx = xyzq[4 * i + 0] - center[0], dy = xyzq[4 * i + 1] - center[1],
           dz = xyzq[4 * i + 2] - center[2];
    double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    if (r > a) a = r;
  }
  *radius = a;
}

void oracle_ylm(int l, int m, double theta, double phi, double* re, double* im) {
  ylm(l, m, theta, phi, re, im);
}

double oracle_threej(int j1, int j2, int j3, int m1, int m2, int m3) {
  return threej(j1, j2, j3, m1, m2, m3);
}

// Eq. (multipole): Q_lm = sum_i q_i r_i^l sqrt(4 pi / (2l+1)) Y_lm(theta_i, phi_i),
// for 0 <= l <= L and -l <= m <= l, about centre c, positions optionally rotated.
// xyzq: n records (x, y, z, q).  rot: row-major 3x3 or NULL.
void oracle_moments(int64_t n, const double* xyzq, const double* center, const double* rot, int L,
                    double* q_re, double* q_im) {
  const int ncomp = (L + 1) * (L + 1);
  std::vector<CSum> acc_re(ncomp), acc_im(ncomp);
  for (int64_t i = 0; i < n; ++i) {
    double r3[3];
    rel_pos(xyzq, i, center, rot, r3);
    double q = xyzq[4 * i + 3];
    double r = std::sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
    double theta = r > 0.0 ? std::acos(std::fmax(-1.0, std::fmin(1.0, r3[2] / r))) : 0.0;
    double phi = std::atan2(r3[1], r3[0]);
    for (int l = 0; l <= L; ++l) {
      double w = q * std::pow(r, l) * std::sqrt(4.0 * kPi / (2 * l + 1));
      for (int m = -l; m <= l; ++m) {
        double yr, yi;
        ylm(l, m, theta, phi, &yr, &yi);
        acc_re[idx(l, m)].add(w * yr);
        acc_im[idx(l, m)].add(w * yi);
      }
    }
  }
  for (int k = 0; k < ncomp; ++k) {
    q_re[k] = acc_re[k].value();
    q_im[k] = acc_im[k].value();
  }
}

// Eq. (Formula), resolved per (l1, l2) block: blocks[l1*(L+1)+l2] holds the real
// part of the block sum, blocks_im the imaginary part (zero for real charges).
void oracle_tcm_blocks(int L, const double* qa_re, const double* qa_im, const double* qb_re,
                       const double* qb_im, const double* R0, double* blocks, double* blocks_im) {
  double R = std::sqrt(R0[0] * R0[0] + R0[1] * R0[1] + R0[2] * R0[2]);
  double theta = std::acos(std::fmax(-1.0, std::fmin(1.0, R0[2] / R)));
  double phi = std::atan2(R0[1], R0[0]);
  for (int l1 = 0; l1 <= L; ++l1) {
    for (int l2 = 0; l2 <= L; ++l2) {
      int LL = l1 + l2;
      long double pref = std::sqrt(4.0L * (long double)kPi * fact(2 * LL) /
                                   (fact(2 * l1) * fact(2 * l2)));
      double scale = (double)pref / std::pow(R, LL + 1);
      CSum sr, si;
      for (int m1 = -l1; m1 <= l1; ++m1) {
        for (int m2 = -l2; m2 <= l2; ++m2) {
          int M = m1 + m2;
          double tj = threej(l1, l2, LL, m1, m2, -M);
          if (tj == 0.0) continue;
          double sgn = (((l1 + M) % 2) + 2) % 2 ? -1.0 : 1.0;
          double yr, yi;
          ylm(LL, M, theta, phi, &yr, &yi);
          yi = -yi;  // Y*_LM
          // (a + ib)(c + id)(e + if)
          double ar = qa_re[idx(l1, m1)], ai = qa_im[idx(l1, m1)];
          double br = qb_re[idx(l2, m2)], bi = qb_im[idx(l2, m2)];
          double pr = ar * br - ai * bi, pi = ar * bi + ai * br;
          double tr = pr * yr - pi * yi, ti = pr * yi + pi * yr;
          double f = sgn * scale * tj;
          sr.add(f * tr);
          si.add(f * ti);
        }
      }
      blocks[l1 * (L + 1) + l2] = sr.value();
      if (blocks_im) blocks_im[l1 * (L + 1) + l2] = si.value();
    }
  }
}

// Eq. (Formula): the truncated two-center energy U_mult; *im_out gets Im(U).
double oracle_tcm_energy(int L, const double* qa_re, const double* qa_im, const double* qb_re,
                         const double* qb_im, const double* R0, double* im_out) {
  std::vector<double> b((L + 1) * (L + 1)), bi((L + 1) * (L + 1));
  oracle_tcm_blocks(L, qa_re, qa_im, qb_re, qb_im, R0, b.data(), bi.data());
  CSum s, si;
  for (size_t k = 0; k < b.size(); ++k) {
    s.add(b[k]);
    si.add(bi[k]);
  }
  if (im_out) *im_out = si.value();
  return s.value();
}

// Eq. (Coulomb): U = sum_i sum_j q_i q_j / |R0 + r_j^B - r_i^A|, with r^A about
// centre cA, r^B about cB and rotated by rotB (NULL = identity).
// *abs_out (optional) receives sum_ij |q_i q_j| / |R0 + r_j^B - r_i^A|, the scale against
// which rounding in the signed sum is measured.
double oracle_direct(int64_t na, const double* a, const double* ca, int64_t nb, const double* b,
                     const double* cb, const double* rotb, const double* R0, double* abs_out) {
  std::vector<double> rb(3 * (size_t)nb);
  for (int64_t j = 0; j < nb; ++j) rel_pos(b, j, cb, rotb, &rb[3 * j]);
  CSum s, sa;
  for (int64_t i = 0; i < na; ++i) {
    double ra[3];
    rel_pos(a, i, ca, nullptr, ra);
    double qi = a[4 * i + 3];
    CSum row, rowa;
    for (int64_t j = 0; j < nb; ++j) {
      double dx = R0[0] + rb[3 * j + 0] - ra[0];
      double dy = R0[1] + rb[3 * j + 1] - ra[1];
      double dz = R0[2] + rb[3 * j + 2] - ra[2];
      double inv = 1.0 / std::sqrt(dx * dx + dy * dy + dz * dz);
      row.add(b[4 * j + 3] * inv);
      rowa.add(std::fabs(b[4 * j + 3]) * inv);
    }
    s.add(qi * row.value());
    sa.add(std::fabs(qi) * rowa.value());
  }
  if (abs_out) *abs_out = sa.value();
  return s.value();
}

}  // extern "C"
