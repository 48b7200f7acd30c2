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
  double R0[3];
  long long rot;   // kBRotate: index of the 3x3 rotation (W rotB) taking B's lab-frame moments
                   // into the frame, in the call's rotation array
};

struct RotDesc {  // one moment set rotated about its centre: out = moments of (M x) from in
  const double* in;
  double* out;
  int L, pad_;
  double M[9];
};

// G (optional, device, 9 doubles per item): force on B, torque on A, torque on B (lab frame).
// rots: device, 9 doubles per kBRotate item (PairDesc.rot), or null when there is none.
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
int launch_direct(const void* a, long long na, int dta, const void* b, long long nb, int dtb,
                  const SysGeom* geo /* device: [A, B] centres */,
                  const double* xf /* device: per item rot[9], R0[3] */, int n_items,
                  double* part /* n_items x nblk */, int nblk, double* E /* device, n_items */, cudaStream_t s);
int direct_blocks(long long na);

// Sets the calling thread's tcm_last_error() message; returns code.
int record_error(int code, const char* msg);

}  // namespace tcm
