// Descriptors and launchers of the contraction (Eq. (Formula) in the frame where R0hat = z)
// and of the Wigner rotation of cached moments.
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
  double Mb[9];    // kBRotate: rotation taking B's lab-frame moments into the frame
};

struct RotDesc {  // one moment set rotated about its centre: out = moments of (M x) from in
  const double* in;
  double* out;
  int L, pad_;
  double M[9];
};

// G (optional, device, 9 doubles per item): force on B, torque on A, torque on B (lab frame).
int launch_contract(const PairDesc* items, int n_items, int Lmax_items, const MomJob* jobs,
                    const SysGeom* geoms, const double* ztab, double* E, int32_t* status, double* G,
                    cudaStream_t s);
int contract_smem_bytes(int L);
int rotate_smem_bytes(int L);
int launch_rotate_moments(const RotDesc* sets, int n_sets, int Lmax_sets, const double* ztab, cudaStream_t s);
int contract_table_size();
void contract_tables(double* t);  // host: fills contract_table_size() doubles

}  // namespace tcm
