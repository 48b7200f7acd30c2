// tcm_moments_noalloc: the moment pass of tcm_moments without any device allocation.
//
// Some callers cannot allocate device memory: code that runs where cudaMalloc/cudaFree
// would synchronise the device and break its latency budget, host applications whose
// own allocator owns every byte of device memory, and plug-ins that are not allowed to
// create allocations of their own.  tcm_moments needs a context, and a context
// allocates (tables at creation, scratch on first use).  This entry point instead keeps
// everything it needs -- the coefficient tables, the job and tile descriptors, the
// centre/radius partials, the low-degree sums and the per-tile moment partials -- in one
// file-scope __device__ array of fixed size, so a call allocates nothing.  The caller
// passes the coordinates and the output buffer, as for tcm_moments.
//
// The array exists once per device (every GPU that loads the library holds it until the
// process exits) and all calls on a device share it: two calls whose work overlaps on
// the GPU race on it, so calls must be serialised (one stream, or events).  Each call
// rewrites the descriptors and clears the work counters before its kernels run.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "contract.h"

using namespace tcm;

namespace {

constexpr long long kNaMaxAtoms = TCM_NOALLOC_MAX_ATOMS;
constexpr int kNaTileAtoms = 4096;                                   // atoms per tile, both precisions
constexpr int kNaTilesPerChunk = (int)(kNaMaxAtoms / kNaTileAtoms);  // 64
constexpr int kNaMaxChunks = 10;                                     // most chunks of any (precision, Lmax)
constexpr int kNaPartialDoubles = kNaTilesPerChunk * 800;            // max over plans of chunks * kmax = 800
constexpr int kNaMaxTiles = kNaTilesPerChunk * kNaMaxChunks;
// system-pass rows: sys_tile_atoms gives at most 128 tiles up to 65,536 atoms and 1,024-atom tiles
// above (256 for the largest request), plus the sum row
constexpr int kNaSysTiles = (int)((kNaMaxAtoms + 1023) / 1024) + 1;
constexpr int kNaCompTotal = 5525;  // sum over L = 0..24 of (L+1)^2

// Layout of the scratch array (byte offsets, 256-byte aligned sections).
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffPartials = 0;
constexpr size_t kOffTiles = align256(kOffPartials + sizeof(double) * kNaPartialDoubles);
constexpr size_t kOffJob = align256(kOffTiles + sizeof(MomTile) * kNaMaxTiles);
constexpr size_t kOffGeom = align256(kOffJob + sizeof(MomJob));
constexpr size_t kOffSJob = align256(kOffGeom + sizeof(SysGeom));
constexpr size_t kOffSTiles1 = align256(kOffSJob + sizeof(SysJob));
constexpr size_t kOffSTiles2 = align256(kOffSTiles1 + sizeof(SysTile) * kNaSysTiles);
constexpr size_t kOffSPart = align256(kOffSTiles2 + sizeof(SysTile) * kNaSysTiles);
constexpr size_t kOffCounters = align256(kOffSPart + sizeof(double) * kSysPart * kNaSysTiles);
constexpr int kNaImapInts = 4 * kNaCompTotal;  // room for the (chunk, slot) maps of plans 0 and 1
constexpr size_t kOffImapOff = align256(kOffCounters + sizeof(int) * 64);
constexpr size_t kOffImap = align256(kOffImapOff + sizeof(int) * 2 * (kLmaxMax + 2));
constexpr size_t kOffFmap = align256(kOffImap + sizeof(int) * kNaImapInts);
constexpr size_t kScratchBytes = align256(kOffFmap + sizeof(double) * kNaImapInts);
// The size stated in include/tcm.h (TCM_NOALLOC_SCRATCH_BYTES) must be this layout's.
static_assert(kScratchBytes == TCM_NOALLOC_SCRATCH_BYTES, "tcm.h states the wrong scratch size");

// The scratch.  In host code this name is only a stand-in for the symbol; kernels get
// the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_tcm_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
char* g_scratch_ptr[kMaxDevices] = {};  // device address of the scratch, per device

int na_err(int code, const char* msg) { return record_error(code, msg); }

// Once per device, with that device current: the scratch address and the tables.
int setup_device(int dev, char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev]) {
    *out = g_scratch_ptr[dev];
    return TCM_OK;
  }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_tcm_noalloc_scratch);
  if (e != cudaSuccess) return na_err(TCM_ECUDA, "tcm_moments_noalloc: cudaGetSymbolAddress of the scratch failed");
  char* base = static_cast<char*>(ptr);
  std::vector<double> fmap;
  std::vector<int> imap_off, imap;
  finalize_tables(imap_off, imap, fmap);
  // only the chunk plans this entry point runs: 0 (double kernels) and 1 (the float kernel's
  // default budget), the first two blocks of the tables
  const size_t n_off = 2 * (kLmaxMax + 2);
  const size_t n_map = (size_t)imap_off[n_off - 1];
  if (imap_off.size() < n_off || n_map > (size_t)kNaImapInts)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: internal table size mismatch");
  if (cudaMemcpy(base + kOffFmap, fmap.data(), n_map * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + kOffImapOff, imap_off.data(), n_off * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + kOffImap, imap.data(), n_map * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: copying the tables into the scratch failed");
  // A copy from pageable host memory may return before the data reach the device; the
  // kernels of this call may run on another (non-blocking) stream, so wait for the tables.
  if (cudaDeviceSynchronize() != cudaSuccess)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: waiting for the table copies failed");
  g_scratch_ptr[dev] = base;
  *out = base;
  return TCM_OK;
}

// Writes one call's descriptors into the scratch and clears the work counters.  The
// descriptors travel as kernel arguments, so no host staging buffer is involved.
__global__ void k_noalloc_prepare(char* base, MomJob job, SysGeom geom, SysJob sjob, int nch, int tpc) {
  MomTile* tiles = reinterpret_cast<MomTile*>(base + kOffTiles);
  SysTile* t1 = reinterpret_cast<SysTile*>(base + kOffSTiles1);
  SysTile* t2 = reinterpret_cast<SysTile*>(base + kOffSTiles2);
  int* counters = reinterpret_cast<int*>(base + kOffCounters);
  if (threadIdx.x == 0) {
    *reinterpret_cast<MomJob*>(base + kOffJob) = job;
    *reinterpret_cast<SysGeom*>(base + kOffGeom) = geom;
    *reinterpret_cast<SysJob*>(base + kOffSJob) = sjob;
  }
  for (int k = threadIdx.x; k < 64; k += blockDim.x) counters[k] = 0;
  for (int k = threadIdx.x; k < sjob.n_tiles; k += blockDim.x) t1[k] = t2[k] = SysTile{0, k};
  for (int k = threadIdx.x; k < nch * tpc; k += blockDim.x) tiles[k] = MomTile{0, k / tpc, k % tpc, k};
}

}  // namespace

extern "C" int tcm_moments_noalloc(const tcm_system* s, const double* rot, int lmax, int precision, double* q_out,
                                   double* geom_out, void* cuda_stream) {
  if (!s || !q_out) return na_err(TCM_EINVAL, "tcm_moments_noalloc: null argument");
  if (lmax < 0 || lmax > TCM_LMAX_MAX) return na_err(TCM_EINVAL, "tcm_moments_noalloc: lmax outside [0, 24]");
  if (precision != TCM_FP64 && precision != TCM_MIXED) return na_err(TCM_EINVAL, "tcm_moments_noalloc: bad precision");
  if (s->n < 0 || s->n > kNaMaxAtoms)
    return na_err(TCM_EINVAL, "tcm_moments_noalloc: atom count outside [0, TCM_NOALLOC_MAX_ATOMS = 262144]");
  if (s->dtype != TCM_F32 && s->dtype != TCM_F64) return na_err(TCM_EINVAL, "tcm_moments_noalloc: bad dtype");
  if (s->n > 0 && (!s->xyzq || (reinterpret_cast<uintptr_t>(s->xyzq) & 15u)))
    return na_err(TCM_EINVAL, "tcm_moments_noalloc: coordinates null or not 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(q_out) & 15u) || (geom_out && (reinterpret_cast<uintptr_t>(geom_out) & 7u)))
    return na_err(TCM_EINVAL, "tcm_moments_noalloc: misaligned output");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: no usable CUDA device");
  char* base = nullptr;
  int rc = setup_device(dev, &base);
  if (rc != TCM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  const int plan = precision == TCM_FP64 ? 0 : 1;
  const int kmax = plan_kmax(plan);
  const int nch = moments_nchunks(plan, lmax);
  const int tpc = (int)std::max<long long>(1, (s->n + kNaTileAtoms - 1) / kNaTileAtoms);
  if (nch > kNaMaxChunks || nch * kmax > 800 || tpc > kNaTilesPerChunk)
    return na_err(TCM_EINVAL, "tcm_moments_noalloc: request exceeds the fixed scratch");
  MomJob job{};
  job.xyzq = s->xyzq;
  job.n = s->n;
  job.dtype = s->dtype;
  job.L = lmax;
  job.geom = 0;
  job.tiles_per_chunk = tpc;
  job.atoms_per_tile = (int)((s->n + tpc - 1) / tpc);
  job.tile_base = 0;
  job.plan = plan;
  for (int k = 0; k < 9; ++k) job.rot[k] = rot ? rot[k] : ((k % 4 == 0) ? 1.0 : 0.0);
  job.out = q_out;
  SysGeom geom{};
  for (int d = 0; d < 3; ++d) {
    geom.c[d] = s->has_center ? s->center[d] : 0.0;
    geom.chi[d] = (float)geom.c[d];
    geom.clo[d] = (float)(geom.c[d] - (double)geom.chi[d]);
  }
  geom.a = s->radius >= 0.0 ? s->radius : 0.0;
  // the pass over the atoms before the moment pass, as tcm_moments plans it: the centroid when
  // no centre is given, the radius when no radius is given, and the low-degree sums of the
  // mixed path (its degrees l <= 2)
  SysJob sj{};
  sj.xyzq = s->xyzq;
  sj.n = s->n;
  sj.dtype = s->dtype;
  sj.geom = 0;
  sj.need_center = s->has_center ? 0 : 1;
  sj.need_radius = (sj.need_center || s->radius < 0.0) ? 1 : 0;
  sj.need_low = precision == TCM_MIXED ? 1 : 0;
  sj.atoms_per_tile = sys_tile_atoms(s->n);
  sj.n_tiles = (int)std::max<long long>(1, (s->n + sj.atoms_per_tile - 1) / sj.atoms_per_tile);
  sj.tile_base = 0;
  sj.first1 = sj.need_center ? 0 : -1;  // the tile lists are written by k_noalloc_prepare
  sj.first2 = 0;
  sj.sum_row = sj.n_tiles;  // the row after the tile rows
  if (sj.n_tiles + 1 > kNaSysTiles) return na_err(TCM_EINVAL, "tcm_moments_noalloc: request exceeds the fixed scratch");
  job.low_base = sj.sum_row;
  job.low_tiles = sj.need_low ? 1 : 0;
  const int n1 = sj.need_center ? sj.n_tiles : 0;
  const int n2 = (sj.need_radius || sj.need_low) ? sj.n_tiles : 0;

  MomJob* d_job = reinterpret_cast<MomJob*>(base + kOffJob);
  SysGeom* d_geom = reinterpret_cast<SysGeom*>(base + kOffGeom);
  k_noalloc_prepare<<<1, 256, 0, st>>>(base, job, geom, sj, nch, tpc);
  if (cudaPeekAtLastError() != cudaSuccess) return na_err(TCM_ECUDA, "tcm_moments_noalloc: launch failed");
  if ((n1 > 0 || n2 > 0) &&
      launch_sys(reinterpret_cast<SysJob*>(base + kOffSJob), reinterpret_cast<SysTile*>(base + kOffSTiles1), n1,
                 reinterpret_cast<SysTile*>(base + kOffSTiles2), n2, reinterpret_cast<double*>(base + kOffSPart),
                 reinterpret_cast<int*>(base + kOffCounters) + 40, d_geom, st) != 0)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: centre/radius launch failed");
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: cudaDeviceGetAttribute failed");
  const int n_tiles = nch * tpc;
  if (launch_moments(plan, lmax, d_job, reinterpret_cast<MomTile*>(base + kOffTiles), n_tiles,
                     reinterpret_cast<int*>(base + kOffCounters), d_geom, reinterpret_cast<double*>(base + kOffPartials),
                     std::min((n_tiles + kThreads / 32 - 1) / (kThreads / 32), 2 * num_sms), st) != 0)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: moment launch failed");
  if (launch_finalize(d_job, 1, reinterpret_cast<double*>(base + kOffPartials), d_geom,
                      reinterpret_cast<int*>(base + kOffImap), reinterpret_cast<double*>(base + kOffFmap),
                      reinterpret_cast<int*>(base + kOffImapOff), reinterpret_cast<double*>(base + kOffSPart),
                      st) != 0)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: finalisation launch failed");
  if (geom_out && cudaMemcpyAsync(geom_out, d_geom, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return na_err(TCM_ECUDA, "tcm_moments_noalloc: copy of the centre and radius failed");
  return TCM_OK;
}
