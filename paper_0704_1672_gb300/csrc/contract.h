// Descriptors and launchers of the kernels after the moment pass: the contraction (Eq. (Formula)
// in the frame where R0hat = z), the Wigner rotation of cached moments, and the direct sum
// (Eq. (Coulomb)).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tcm_internal.h"

namespace tcm {

// How the contraction receives B's moments.
constexpr int kBLab = 0;      // lab frame: rotated by the frame rotation W (R0hat -> z) like A's
constexpr int kBInFrame = 1;  // already in the frame (the rotation was applied to B's atoms)
constexpr int kBRotate = 2;   // lab frame, rotated by Mb = W rotB with the Wigner D in the kernel

struct PairDesc {  // one energy: moments of jobA and jobB at lmax L, separation R0
  int jobA, jobB;
  int geomA, geomB;
  int L;
  int b_mode;      // kBLab, kBInFrame or kBRotate
  long long rot;   // kBRotate: index of the Euler record (EulerZYZ) of Mb = W rotB, which takes
                   // B's lab-frame moments into the frame, in the call's rotation array
  double fr[6];    // R0 by its frame W = R_y(-b) R_z(-a) (pair_frame): 1/R, R, cos b, sin b, cos a, sin a
};

// A rotation M = R_z(-gamma) R_y(-beta) R_z(-alpha), beta in [0, pi], as (cos beta, sin beta,
// e^{i alpha}, e^{i gamma}).
struct EulerZYZ {
  double cb, sb;
  double ea[2], eg[2];
};

// Euler record of a rotation matrix (row-major) through its unit quaternion (largest-component
// extraction): with q = (w, x, y, z),
//   cos(beta/2) = |(w, z)|,  sin(beta/2) = |(x, y)|,
//   e^{i(alpha+gamma)/2} = (w - i z) / cos(beta/2),  e^{i(alpha-gamma)/2} = (-y + i x) / sin(beta/2),
// which stays accurate near beta = 0 and pi (where only alpha+gamma, resp. alpha-gamma, matters).
__host__ __device__ inline EulerZYZ euler_zyz(const double* M) {
  const double t = M[0] + M[4] + M[8];
  double w, x, y, z;
  if (t > 0.0) {
    const double s = 2.0 * sqrt(t + 1.0);
    w = 0.25 * s; x = (M[7] - M[5]) / s; y = (M[2] - M[6]) / s; z = (M[3] - M[1]) / s;
  } else if (M[0] > M[4] && M[0] > M[8]) {
    const double s = 2.0 * sqrt(1.0 + M[0] - M[4] - M[8]);
    w = (M[7] - M[5]) / s; x = 0.25 * s; y = (M[1] + M[3]) / s; z = (M[2] + M[6]) / s;
  } else if (M[4] > M[8]) {
    const double s = 2.0 * sqrt(1.0 + M[4] - M[0] - M[8]);
    w = (M[2] - M[6]) / s; x = (M[1] + M[3]) / s; y = 0.25 * s; z = (M[5] + M[7]) / s;
  } else {
    const double s = 2.0 * sqrt(1.0 + M[8] - M[0] - M[4]);
    w = (M[3] - M[1]) / s; x = (M[2] + M[6]) / s; y = (M[5] + M[7]) / s; z = 0.25 * s;
  }
  const double n = 1.0 / sqrt(w * w + x * x + y * y + z * z);
  w *= n; x *= n; y *= n; z *= n;
  const double ch = sqrt(w * w + z * z), sh = sqrt(x * x + y * y);
  const double pr = ch > 0.0 ? w / ch : 1.0, pi = ch > 0.0 ? -z / ch : 0.0;   // p = e^{i(alpha+gamma)/2}
  const double qr = sh > 0.0 ? -y / sh : 1.0, qi = sh > 0.0 ? x / sh : 0.0;   // q = e^{i(alpha-gamma)/2}
  EulerZYZ e;
  e.cb = (ch - sh) * (ch + sh);
  e.sb = 2.0 * ch * sh;
  e.ea[0] = pr * qr - pi * qi;  // p q
  e.ea[1] = pr * qi + pi * qr;
  e.eg[0] = pr * qr + pi * qi;  // p conj(q)
  e.eg[1] = pi * qr - pr * qi;
  return e;
}

struct RotDesc {  // one moment set rotated about its centre: out = moments of (M x) from in
  const double* in;
  double* out;
  int L, pad_;
  double M[9];
};

// G (optional, device, 9 doubles per item): force on B, torque on A, torque on B (lab frame).
// rots: device, one EulerZYZ per kBRotate item (PairDesc.rot), or null when there is none.
int launch_contract(const PairDesc* items, int n_items, int Lmax_items, const MomJob* jobs,
                    const SysGeom* geoms, const double* ztab, const double* rots, double* E, int32_t* status,
                    double* G, cudaStream_t s);
int contract_smem_bytes(int L);
int rotate_smem_bytes(int L);
int launch_rotate_moments(const RotDesc* sets, int n_sets, int Lmax_sets, const double* ztab, cudaStream_t s);
int contract_table_size();
void contract_tables(double* t);  // host: fills contract_table_size() doubles

// Rotation W = R_y(-beta) R_z(-alpha) taking R0hat to the z axis (row-major).
__host__ __device__ inline void frame_rotation(const double* R0, double* W) {
  const double x = R0[0], y = R0[1], z = R0[2];
  const double R = sqrt(x * x + y * y + z * z);
  const double rho = sqrt(x * x + y * y);
  const double cb = z / R, sb = rho / R;
  const double ca = rho > 0.0 ? x / rho : 1.0, sa = rho > 0.0 ? y / rho : 0.0;
  W[0] = cb * ca; W[1] = cb * sa; W[2] = -sb;
  W[3] = -sa;     W[4] = ca;      W[5] = 0.0;
  W[6] = sb * ca; W[7] = sb * sa; W[8] = cb;
}
// Host: the frame record PairDesc.fr of R0 (cos b = z/R, sin b = rho/R, e^{ia} = (x + iy)/rho,
// e^{ia} = 1 on the z axis).
inline void pair_frame(const double* R0, PairDesc& d) {
  const double x = R0[0], y = R0[1], z = R0[2];
  const double rho = sqrt(x * x + y * y);
  const double R = sqrt(x * x + y * y + z * z);
  d.fr[0] = 1.0 / R;
  d.fr[1] = R;
  d.fr[2] = z / R;
  d.fr[3] = rho / R;
  d.fr[4] = rho > 0.0 ? x / rho : 1.0;
  d.fr[5] = rho > 0.0 ? y / rho : 0.0;
}
int launch_direct(const void* a, long long na, int dta, const void* b, long long nb, int dtb,
                  const SysGeom* geo /* device: [A, B] centres */,
                  const double* xf /* device: per item rot[9], R0[3] */, int n_items,
                  double* part /* n_items x nblk */, int nblk, double* E /* device, n_items */, cudaStream_t s);
int direct_blocks(long long na);

// Sets the calling thread's tcm_last_error() message; returns code.
int record_error(int code, const char* msg);

}  // namespace tcm
