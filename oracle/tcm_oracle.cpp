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
//   * forces and torques (the paper names them as a use of Eq. (Formula) but prints no
//     formula): the gradient of Eq. (Formula) in R0 through the textbook derivatives of
//     Y_LM, the derivative of Eq. (multipole) under a rotation of a system about its
//     centre, and the exact pairwise forces and torques of Eq. (Coulomb)
// Spherical harmonics are orthonormal with the Condon-Shortley phase (the
// convention of Varshalovich, which the paper follows); Y_lm for m >= 0 comes
// from std::sph_legendre (from the hypergeometric series within 1.1 degrees of a
// pole, where the library loses digits) and Y_l,-m = (-1)^m conj(Y_lm).
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

// Y_lm(theta, 0), 0 <= m <= l, within sin^2(theta/2) < 1e-4 of the north pole, where the
// library function (which works from cos theta) loses the digits of sin^m theta.  From the
// Ferrers function as a terminating hypergeometric series in s = sin^2(theta/2):
//   P_l^m(cos t) = (-1)^m sin^m t (l+m)! / (2^m m! (l-m)!) 2F1(m-l, l+m+1; m+1; s),
// whose terms fall by a factor <= l^2 s / (m+1) < 0.25 here for l <= 48 (no cancellation beyond a digit in long double).
double ylm0_near_pole(int l, int m, double sin_t, double s) {
  long double f = 1.0L, t = 1.0L;
  for (int k = 0; k < l - m; ++k) {
    t *= (long double)(m - l + k) * (l + m + 1 + k) / ((long double)(m + 1 + k) * (k + 1)) * s;
    f += t;
  }
  long double norm = std::sqrt((2 * l + 1) / (4.0L * (long double)kPi) * fact(l + m) / fact(l - m)) /
                     (std::pow(2.0L, m) * fact(m));
  long double v = norm * std::pow((long double)sin_t, m) * f;
  return (double)((m % 2) ? -v : v);
}

// Orthonormal Y_lm(theta, phi) with Condon-Shortley phase, any m in [-l, l].
void ylm(int l, int m, double theta, double phi, double* re, double* im) {
  int am = m < 0 ? -m : m;
  const double sh = std::sin(0.5 * theta), ch = std::cos(0.5 * theta);
  double p;  // Y_l|m|(theta, 0)
  if (sh * sh < 1e-4)
    p = ylm0_near_pole(l, am, std::sin(theta), sh * sh);
  else if (ch * ch < 1e-4)  // Y_lm(pi - t, 0) = (-1)^(l+m) Y_lm(t, 0)
    p = ((l + am) % 2 ? -1.0 : 1.0) * ylm0_near_pole(l, am, std::sin(theta), ch * ch);
  else
    p = std::sph_legendre((unsigned)l, (unsigned)am, theta);
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

// Polar angle of v as atan2(|(x, y)|, z): the same angle as acos(z/|v|), without the loss of
// half the digits near the poles that acos has (acos(1 - d) ~ sqrt(2 d)).  0 for v = 0.
double polar_angle(const double* v) { return std::atan2(std::hypot(v[0], v[1]), v[2]); }

// Angular derivatives of Y_lm for the gradients (Section II gives no force formula; these are
// the textbook derivatives of the orthonormal harmonics):
//   dY_lm/dtheta = 1/2 [ c+ e^{-i phi} Y_l,m+1 - c- e^{+i phi} Y_l,m-1 ],
//   c+ = sqrt((l-m)(l+m+1)), c- = sqrt((l+m)(l-m+1))   (ladder form, regular at the poles);
//   (1/sin theta) dY_lm/dphi = i m Y_lm / sin theta, taken near the poles from the sum of the
//   two ladder terms:  m Y_lm / sin theta = -[ c+ e^{-i phi} Y_l,m+1 + c- e^{i phi} Y_l,m-1 ] / (2 cos theta).
void ladder_terms(int l, int m, double th, double ph, double* ar, double* ai, double* br, double* bi) {
  // (ar, ai) = c+ e^{-i phi} Y_l,m+1 ; (br, bi) = c- e^{i phi} Y_l,m-1
  double cp = std::sqrt((double)(l - m) * (l + m + 1)), cm = std::sqrt((double)(l + m) * (l - m + 1));
  double ur = 0.0, ui = 0.0, dr = 0.0, di = 0.0;
  if (m + 1 <= l) ylm(l, m + 1, th, ph, &ur, &ui);
  if (m - 1 >= -l) ylm(l, m - 1, th, ph, &dr, &di);
  const double c = std::cos(ph), s = std::sin(ph);
  *ar = cp * (c * ur + s * ui);
  *ai = cp * (c * ui - s * ur);
  *br = cm * (c * dr - s * di);
  *bi = cm * (c * di + s * dr);
}

void ylm_dtheta(int l, int m, double th, double ph, double* re, double* im) {
  double ar, ai, br, bi;
  ladder_terms(l, m, th, ph, &ar, &ai, &br, &bi);
  *re = 0.5 * (ar - br);
  *im = 0.5 * (ai - bi);
}

void ylm_dphi_over_sin(int l, int m, double th, double ph, double* re, double* im) {
  const double st = std::sin(th);
  double vr, vi;  // m Y / sin theta
  if (st > 0.5) {
    double yr, yi;
    ylm(l, m, th, ph, &yr, &yi);
    vr = m * yr / st;
    vi = m * yi / st;
  } else {
    double ar, ai, br, bi;
    ladder_terms(l, m, th, ph, &ar, &ai, &br, &bi);
    const double k = -1.0 / (2.0 * std::cos(th));
    vr = k * (ar + br);
    vi = k * (ai + bi);
  }
  *re = -vi;  // i (vr + i vi)
  *im = vr;
}

// Spherical unit vectors at (theta, phi).
void sph_frame(double th, double ph, double* rh, double* th_hat, double* ph_hat) {
  const double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
  rh[0] = st * cp; rh[1] = st * sp; rh[2] = ct;
  th_hat[0] = ct * cp; th_hat[1] = ct * sp; th_hat[2] = -st;
  ph_hat[0] = -sp; ph_hat[1] = cp; ph_hat[2] = 0.0;
}

}  // namespace

extern "C" {

int oracle_abi_version(void) { return 2; }

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
    double theta = polar_angle(r3);
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
  double theta = polar_angle(R0);
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

// Force on B, F = -grad_R0 U_mult, from Eq. (Formula) as printed: the separation factor
// Y*_LM(R0hat) / R0^(L+1) is replaced by its gradient
//   -(L+1) Y*/R^(L+2) Rhat + (dY/dtheta)*/R^(L+2) thetahat + (i M Y / sin theta)*/R^(L+2) phihat.
// force[3] gets the real force; block_norm[l1*(L+1)+l2] (optional) the length of each
// (l1, l2) block's force vector, the scale of its rounding.
void oracle_tcm_force(int L, const double* qa_re, const double* qa_im, const double* qb_re, const double* qb_im,
                      const double* R0, double* force, double* block_norm) {
  double R = std::sqrt(R0[0] * R0[0] + R0[1] * R0[1] + R0[2] * R0[2]);
  double theta = polar_angle(R0);
  double phi = std::atan2(R0[1], R0[0]);
  double rh[3], thh[3], phh[3];
  sph_frame(theta, phi, rh, thh, phh);
  CSum tot[3];
  for (int l1 = 0; l1 <= L; ++l1) {
    for (int l2 = 0; l2 <= L; ++l2) {
      int LL = l1 + l2;
      long double pref = std::sqrt(4.0L * (long double)kPi * fact(2 * LL) / (fact(2 * l1) * fact(2 * l2)));
      double scale = (double)pref / std::pow(R, LL + 2);
      CSum g[3];
      for (int m1 = -l1; m1 <= l1; ++m1) {
        for (int m2 = -l2; m2 <= l2; ++m2) {
          int M = m1 + m2;
          double tj = threej(l1, l2, LL, m1, m2, -M);
          if (tj == 0.0) continue;
          double sgn = (((l1 + M) % 2) + 2) % 2 ? -1.0 : 1.0;
          double yr, yi, tr, ti, pr_, pi_;
          ylm(LL, M, theta, phi, &yr, &yi);
          ylm_dtheta(LL, M, theta, phi, &tr, &ti);
          ylm_dphi_over_sin(LL, M, theta, phi, &pr_, &pi_);
          // the separation harmonic enters conjugated
          yi = -yi;
          ti = -ti;
          pi_ = -pi_;
          double ar = qa_re[idx(l1, m1)], ai = qa_im[idx(l1, m1)];
          double br = qb_re[idx(l2, m2)], bi = qb_im[idx(l2, m2)];
          double qr = ar * br - ai * bi, qi = ar * bi + ai * br;
          double f = sgn * scale * tj;
          // Re[(qr + i qi) v] for v = -(L+1) Y*, (dY/dtheta)*, (i M Y / sin theta)*
          double vR = -(LL + 1) * (qr * yr - qi * yi);
          double vT = qr * tr - qi * ti;
          double vP = qr * pr_ - qi * pi_;
          for (int d = 0; d < 3; ++d) g[d].add(f * (vR * rh[d] + vT * thh[d] + vP * phh[d]));
        }
      }
      double bn = 0.0;
      for (int d = 0; d < 3; ++d) {
        double v = g[d].value();
        tot[d].add(-v);  // force = -gradient
        bn += v * v;
      }
      if (block_norm) block_norm[l1 * (L + 1) + l2] = std::sqrt(bn);
    }
  }
  for (int d = 0; d < 3; ++d) force[d] = tot[d].value();
}

// Derivative of Eq. (multipole) under a rotation of the system about its centre: with every
// position moved to r + eps n x r, dQ_lm/deps = sum_i q_i sqrt(4 pi/(2l+1)) n . (r x grad)(r^l Y_lm)
// and (r x grad)(r^l Y) = r^l [ phihat dY/dtheta - thetahat (1/sin theta) dY/dphi ].
// Positions are taken about the centre, after the optional rotation rot.
void oracle_moments_rotderiv(int64_t n, const double* xyzq, const double* center, const double* rot, int L,
                             const double* axis, double* d_re, double* d_im) {
  const int ncomp = (L + 1) * (L + 1);
  std::vector<CSum> acc_re(ncomp), acc_im(ncomp);
  for (int64_t i = 0; i < n; ++i) {
    double r3[3];
    rel_pos(xyzq, i, center, rot, r3);
    double q = xyzq[4 * i + 3];
    double r = std::sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
    if (r == 0.0) continue;  // n x r = 0: the atom does not move
    double theta = polar_angle(r3);
    double phi = std::atan2(r3[1], r3[0]);
    double rh[3], thh[3], phh[3];
    sph_frame(theta, phi, rh, thh, phh);
    const double nphi = axis[0] * phh[0] + axis[1] * phh[1] + axis[2] * phh[2];
    const double nth = axis[0] * thh[0] + axis[1] * thh[1] + axis[2] * thh[2];
    for (int l = 0; l <= L; ++l) {
      double w = q * std::pow(r, l) * std::sqrt(4.0 * kPi / (2 * l + 1));
      for (int m = -l; m <= l; ++m) {
        double tr, ti, pr_, pi_;
        ylm_dtheta(l, m, theta, phi, &tr, &ti);
        ylm_dphi_over_sin(l, m, theta, phi, &pr_, &pi_);
        acc_re[idx(l, m)].add(w * (nphi * tr - nth * pr_));
        acc_im[idx(l, m)].add(w * (nphi * ti - nth * pi_));
      }
    }
  }
  for (int k = 0; k < ncomp; ++k) {
    d_re[k] = acc_re[k].value();
    d_im[k] = acc_im[k].value();
  }
}

// Eq. (Coulomb) differentiated: the exact force on B, F_B = sum_ij q_i q_j d_ij / |d_ij|^3 with
// d_ij = R0 + r_j^B - r_i^A, and the torques on A and on B about their centres,
// tau_A = sum_i r_i^A x (-F_i), tau_B = sum_j r_j^B x F_j (r^B rotated by rotB).
// out[9] = F_B, tau_A, tau_B.  *abs_out (optional) = sum_ij |q_i q_j| / |d_ij|^2.
void oracle_direct_forces(int64_t na, const double* a, const double* ca, int64_t nb, const double* b,
                          const double* cb, const double* rotb, const double* R0, double* out, double* abs_out) {
  std::vector<double> rb(3 * (size_t)nb);
  for (int64_t j = 0; j < nb; ++j) rel_pos(b, j, cb, rotb, &rb[3 * j]);
  std::vector<CSum> fj(3 * (size_t)nb);
  CSum TA[3], sa;
  for (int64_t i = 0; i < na; ++i) {
    double ra[3];
    rel_pos(a, i, ca, nullptr, ra);
    double qi = a[4 * i + 3];
    CSum fi[3];
    for (int64_t j = 0; j < nb; ++j) {
      double d[3] = {R0[0] + rb[3 * j + 0] - ra[0], R0[1] + rb[3 * j + 1] - ra[1], R0[2] + rb[3 * j + 2] - ra[2]};
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double r = std::sqrt(r2);
      double w = qi * b[4 * j + 3] / (r2 * r);
      for (int k = 0; k < 3; ++k) {
        fj[3 * j + k].add(w * d[k]);
        fi[k].add(-w * d[k]);
      }
      sa.add(std::fabs(qi * b[4 * j + 3]) / r2);
    }
    double f[3] = {fi[0].value(), fi[1].value(), fi[2].value()};
    TA[0].add(ra[1] * f[2] - ra[2] * f[1]);
    TA[1].add(ra[2] * f[0] - ra[0] * f[2]);
    TA[2].add(ra[0] * f[1] - ra[1] * f[0]);
  }
  CSum F[3], TB[3];
  for (int64_t j = 0; j < nb; ++j) {
    double f[3] = {fj[3 * j].value(), fj[3 * j + 1].value(), fj[3 * j + 2].value()};
    const double* r = &rb[3 * j];
    for (int k = 0; k < 3; ++k) F[k].add(f[k]);
    TB[0].add(r[1] * f[2] - r[2] * f[1]);
    TB[1].add(r[2] * f[0] - r[0] * f[2]);
    TB[2].add(r[0] * f[1] - r[1] * f[0]);
  }
  for (int k = 0; k < 3; ++k) {
    out[k] = F[k].value();
    out[3 + k] = TA[k].value();
    out[6 + k] = TB[k].value();
  }
  if (abs_out) *abs_out = sa.value();
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
