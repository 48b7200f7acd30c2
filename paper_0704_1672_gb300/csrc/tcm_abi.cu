// C ABI of libtcm.so (include/tcm.h): argument checks, the context (tables, scratch,
// descriptor staging) and the host-side planning of moment jobs and tiles.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <unordered_map>
#include <new>
#include <tuple>
#include <vector>

#include "contract.h"

using namespace tcm;

namespace {

thread_local char g_err[512] = "";

int set_err(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

#define TRY_CUDA(expr)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess) return set_err(TCM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));           \
  } while (0)
#define TRY(expr)                   \
  do {                              \
    int r_ = (expr);                \
    if (r_ != TCM_OK) return r_;    \
  } while (0)
#define TRY_LAUNCH(expr)                                                                                 \
  do {                                                                                                   \
    if ((expr) != 0) {                                                                                   \
      cudaError_t e_ = cudaGetLastError();                                                               \
      return set_err(TCM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                                \
    }                                                                                                    \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Stage {  // pinned host staging slot for one call's descriptors
  void* host = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool pending = false;
};

constexpr int kStages = 4;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Layout of one call's descriptor block: add() records where each host array goes (256-byte
// aligned offsets); upload() copies the arrays straight into a pinned staging buffer and
// sends the block with a single copy.  The arrays must stay unchanged until upload().
struct Packer {
  struct Span {
    const void* p;
    size_t bytes;
    size_t off;
  };
  std::vector<Span> spans;
  size_t size = 0;
  template <typename T>
  size_t add(const std::vector<T>& v) {
    const size_t off = align_up(size);
    spans.push_back(Span{v.data(), v.size() * sizeof(T), off});
    size = off + std::max<size_t>(v.size() * sizeof(T), 1);
    return off;
  }
  // two arrays of one type back to back (one device array), without concatenating them on the host
  template <typename T>
  size_t add2(const std::vector<T>& a, const std::vector<T>& b) {
    const size_t off = align_up(size);
    spans.push_back(Span{a.data(), a.size() * sizeof(T), off});
    spans.push_back(Span{b.data(), b.size() * sizeof(T), off + a.size() * sizeof(T)});
    size = off + std::max<size_t>((a.size() + b.size()) * sizeof(T), 1);
    return off;
  }
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

struct tcm_ctx {
  int device = 0;
  int num_sms = 0;
  int lmax_cap = 0;
  cudaStream_t stream = nullptr;
  // tables
  double* d_fmap = nullptr;  // F_lm of the component each (chunk, slot) holds
  double* d_ztab = nullptr;  // contraction tables (factorials, 1/sqrt((l+m)!(l-m)!), the rows of d^l(pi/2))
  int* d_imap = nullptr;      // (chunk, slot) -> packed component, both precisions
  int* d_imap_off = nullptr;  // [precision][L] offsets into d_imap
  // scratch
  DevBuf desc, partials, gpart, systk, systiles, counters, moms, escr, dpart, tiles;
  Stage stage[kStages];
  int stage_next = 0;
  void* pinned_small = nullptr;  // 256 B for small device->host reads
  // moment-pass tiling per [TCM_FP64, TCM_MIXED][L]: atoms per lane of a warp tile, and the
  // resident CTAs per SM the persistent grid is sized for
  int atoms_per_thread[2][kLmaxMax + 1];
  int ctas_per_sm[2][kLmaxMax + 1];
  int plan_l[kLmaxMax + 1];  // mixed path: the float kernel's chunk plan per degree (1 or 2)
  int64_t cfg_gen = 0;       // bumped by every tiling or chunking change (part of the graph key)
  // phase profiling
  bool prof = false;
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> ev_pool;
  int64_t launches[TCM_NPHASES] = {};
  double host_ms = 0.0;  // TCM_PHASE_HOST: wall time inside the batched calls while profiling
  // CUDA-graph replay of the batched launch sequence
  bool rotate_cached = false;  // rotated B sides from the moment cache by Wigner rotation
  int graphs = 1;  // 0: launch directly; 1: capture a shape seen twice in a row; 2: capture every new shape
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<long long> gkey, gkey_seen;
  int64_t graph_captures = 0, graph_launches = 0;
};

namespace {

cudaEvent_t pool_event(tcm_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Records an event pair around one phase when profiling is on, and counts launches.
struct PhaseScope {
  tcm_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(tcm_ctx* c_, int ph, int nlaunch) : c(c_), phase(ph) {
    c->launches[ph] += nlaunch;
    if (c->prof && (a = pool_event(c)) != nullptr) cudaEventRecord(a, c->stream);
  }
  ~PhaseScope() {
    if (!a) return;
    cudaEvent_t b = pool_event(c);
    if (!b) {
      c->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, c->stream);
    c->marks.push_back({phase, a, b});
  }
};

int dev_ensure(tcm_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return TCM_OK;
  size_t nc = std::max(bytes, b.cap + b.cap / 2);
  nc = align_up(std::max<size_t>(nc, kAlign));
  if (b.p) {
    TRY_CUDA(cudaStreamSynchronize(c->stream));
    TRY_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  if (cudaMalloc(&b.p, nc) != cudaSuccess) {
    cudaGetLastError();
    return set_err(TCM_ENOMEM, "cudaMalloc of %zu bytes failed", nc);
  }
  b.cap = nc;
  return TCM_OK;
}

// Copy the packed descriptors to the device through a pinned slot; returns the
// device base address in *dbase.
int upload(tcm_ctx* c, const Packer& pk, char** dbase) {
  const size_t bytes = std::max<size_t>(pk.size, 1);
  TRY(dev_ensure(c, c->desc, bytes));
  Stage& st = c->stage[c->stage_next];
  c->stage_next = (c->stage_next + 1) % kStages;
  if (st.pending) {
    TRY_CUDA(cudaEventSynchronize(st.ev));
    st.pending = false;
  }
  if (st.cap < bytes) {
    if (st.host) TRY_CUDA(cudaFreeHost(st.host));
    st.host = nullptr;
    st.cap = 0;
    const size_t nc = align_up(std::max<size_t>(bytes * 2, 4096));
    if (cudaHostAlloc(&st.host, nc, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return set_err(TCM_ENOMEM, "cudaHostAlloc of %zu bytes failed", nc);
    }
    st.cap = nc;
  }
  for (const Packer::Span& sp : pk.spans)
    if (sp.bytes) std::memcpy(static_cast<char*>(st.host) + sp.off, sp.p, sp.bytes);
  TRY_CUDA(cudaMemcpyAsync(c->desc.p, st.host, bytes, cudaMemcpyHostToDevice, c->stream));
  TRY_CUDA(cudaEventRecord(st.ev, c->stream));
  st.pending = true;
  *dbase = static_cast<char*>(c->desc.p);
  return TCM_OK;
}

int check_system(const tcm_system* s, const char* what) {
  if (!s) return set_err(TCM_EINVAL, "%s: null system", what);
  if (s->n < 0) return set_err(TCM_EINVAL, "%s: negative atom count", what);
  if (s->dtype != TCM_F32 && s->dtype != TCM_F64) return set_err(TCM_EINVAL, "%s: dtype must be TCM_F32 or TCM_F64", what);
  if (s->n > 0 && !s->xyzq) return set_err(TCM_EINVAL, "%s: null coordinate pointer", what);
  if (s->n > 0 && !aligned16(s->xyzq)) return set_err(TCM_EINVAL, "%s: coordinates must be 16-byte aligned", what);
  if (s->has_center && !(std::isfinite(s->center[0]) && std::isfinite(s->center[1]) && std::isfinite(s->center[2])))
    return set_err(TCM_EINVAL, "%s: non-finite centre", what);
  if (s->moments) {
    if (!s->has_center || !(s->radius >= 0.0))
      return set_err(TCM_EINVAL, "%s: a moment cache needs the centre and radius it was taken with", what);
    if (s->moments_lmax < 0 || s->moments_lmax > TCM_LMAX_MAX || !aligned16(s->moments))
      return set_err(TCM_EINVAL, "%s: bad moment cache (lmax or alignment)", what);
  }
  return TCM_OK;
}

bool geom_known(const tcm_system& s) { return s.has_center && s.radius >= 0.0; }

// Moment-job planning -------------------------------------------------------------


struct Plan {
  std::vector<MomJob> jobs;
  std::vector<MomGroup> groups;    // (job, chunk) groups, largest tiles first; expanded on the device
  int n_tiles = 0;
  // FP64 (one launch per degree): the tiles of L are [tile_begin[L], tile_begin[L+1]); mixed
  // (one launch per chunk plan over all degrees): the tiles of plan p are
  // [tile_begin[p - 1], tile_begin[p])
  int tile_begin[kLmaxMax + 2] = {};
  int n_tile_ids = 0;
  size_t moms_doubles = 0;
};

void plan_job(tcm_ctx* c, int precision, MomJob& j, int& next_id) {
  j.plan = precision == TCM_FP64 ? 0 : c->plan_l[j.L];
  const int nch = moments_nchunks(j.plan, j.L);
  const long long per_tile = 32LL * c->atoms_per_thread[precision == TCM_FP64 ? 0 : 1][j.L];  // one warp
  long long tpc = (j.n + per_tile - 1) / per_tile;
  if (tpc < 1) tpc = 1;
  j.tiles_per_chunk = (int)tpc;
  j.atoms_per_tile = (int)((j.n + tpc - 1) / tpc);
  j.tile_base = next_id;
  next_id += nch * (int)tpc;
}


// The (job, chunk) groups in decreasing order of their tiles' cost (largest first, so the
// persistent warps finish together).  FP64: grouped by degree (one launch per degree); mixed:
// grouped by chunk plan (one launch per plan present, usually one), one order over all degrees.  The tiles themselves are written on the device
// (k_expand_tiles), so the host work is O(groups log groups).
void build_tiles(int precision, Plan& P) {
  // one 32-bit key per group: [degree (FP64) or chunk plan (mixed), 5 bits] [largest cost first,
  // 27 bits]; a stable sort keeps ties in their planning order, so the order is deterministic.
  // The sort is a least-significant-digit radix sort (three passes of 11 bits): for the tens of
  // thousands of groups of a large batch it takes a fraction of a comparison sort's time.
  struct Group {
    int job, chunk;
  };
  std::vector<Group> g;
  std::vector<uint32_t> key;
  g.reserve(P.jobs.size() * 2);
  key.reserve(P.jobs.size() * 2);
  const bool by_degree = precision == TCM_FP64;
  for (int ji = 0; ji < (int)P.jobs.size(); ++ji) {
    const MomJob& j = P.jobs[ji];
    const int nch = moments_nchunks(j.plan, j.L);
    const double* cc = moments_chunk_costs(j.plan, j.L);
    for (int ch = 0; ch < nch; ++ch) {
      const double cost = cc[ch] * (double)j.atoms_per_tile;
      const uint32_t cq = (uint32_t)std::min(cost, 134217727.0);  // 27 bits
      key.push_back(((uint32_t)(by_degree ? j.L : j.plan - 1) << 27) | (134217727u - cq));
      g.push_back(Group{ji, ch});
    }
  }
  const size_t n = key.size();
  std::vector<uint32_t> order(n), k2(n), o2(n);
  for (size_t i = 0; i < n; ++i) order[i] = (uint32_t)i;
  for (int shift = 0; shift < 32; shift += 11) {
    uint32_t count[2049] = {};
    for (size_t i = 0; i < n; ++i) ++count[((key[i] >> shift) & 2047u) + 1];
    for (int b = 0; b < 2048; ++b) count[b + 1] += count[b];
    for (size_t i = 0; i < n; ++i) {
      const uint32_t d = (key[i] >> shift) & 2047u;
      k2[count[d]] = key[i];
      o2[count[d]++] = order[i];
    }
    key.swap(k2);
    order.swap(o2);
  }
  P.groups.clear();
  P.groups.reserve(n);
  int first = 0;
  size_t gi = 0;
  for (int L = 0; L <= kLmaxMax; ++L) {
    P.tile_begin[L] = first;
    for (; gi < n; ++gi) {
      const Group& gr = g[order[gi]];
      if ((by_degree ? P.jobs[gr.job].L : P.jobs[gr.job].plan - 1) != L) break;
      const int nt = P.jobs[gr.job].tiles_per_chunk;
      P.groups.push_back(MomGroup{gr.job, gr.chunk, nt, first});
      first += nt;
    }
  }
  P.tile_begin[kLmaxMax + 1] = first;
  P.n_tiles = first;
}

// Moment-phase launches of a plan (for the launch counts of a replayed graph): FP64 one per
// degree present, mixed one per chunk plan present.
int moment_launches(int precision, const Plan& P) {
  const int nb = precision == TCM_FP64 ? kLmaxMax + 1 : kNumPlans - 1;
  int n = 0;
  for (int k = 0; k < nb; ++k) n += P.tile_begin[k + 1] > P.tile_begin[k];
  return n;
}

// Queue the moment pass (step a2/a3) for every job of the plan.
// The moment kernels' work counters and exit tickets (counters[L], counters[32 + L]) are zero
// on entry and left zero by every launch, so they are cleared once, when allocated.
int ensure_moment_buffers(tcm_ctx* c, int precision, const Plan& P) {
  TRY(dev_ensure(c, c->partials, (size_t)std::max(P.n_tile_ids, 1) * plan_row(precision == TCM_FP64 ? 0 : 1) *
                                     sizeof(double)));
  TRY(dev_ensure(c, c->tiles, (size_t)std::max(P.n_tiles, 1) * sizeof(MomTile)));
  void* before = c->counters.p;
  TRY(dev_ensure(c, c->counters, 64 * sizeof(int)));
  if (c->counters.p != before) {
    TRY_CUDA(cudaMemsetAsync(c->counters.p, 0, 64 * sizeof(int), c->stream));
  }
  return TCM_OK;
}

// Counter slots of the moment kernels (zero on entry, left zero): [L] and [32 + L] for the
// per-degree FP64 launches, [kAnyCounter + p] and [32 + kAnyCounter + p] for the mixed launch of
// chunk plan p over all degrees.
constexpr int kAnyCounter = kLmaxMax;  // + plan (1 or 2)

int run_moments(tcm_ctx* c, int precision, const Plan& P, const MomJob* d_jobs, const SysGeom* d_geoms,
                cudaStream_t st) {
  TRY(ensure_moment_buffers(c, precision, P));
  int* counters = static_cast<int*>(c->counters.p);
  double* parts = static_cast<double*>(c->partials.p);
  MomTile* tiles = static_cast<MomTile*>(c->tiles.p);
  if (precision == TCM_FP64) {
    int ngroups = 0;
    for (int L = 0; L <= kLmaxMax; ++L) ngroups += P.tile_begin[L + 1] > P.tile_begin[L];
    PhaseScope ps(c, TCM_PHASE_MOMENTS, ngroups);
    for (int L = 0; L <= kLmaxMax; ++L) {
      const int b = P.tile_begin[L], e = P.tile_begin[L + 1];
      if (e == b) continue;
      const int cps = c->ctas_per_sm[0][L];
      const int grid = std::min((e - b + kThreads / 32 - 1) / (kThreads / 32), cps * c->num_sms);  // warp tiles
      TRY_LAUNCH(launch_moments(0, L, d_jobs, tiles + b, e - b, counters + L, d_geoms, parts, grid, st));
    }
  } else if (P.n_tiles > 0) {
    PhaseScope ps(c, TCM_PHASE_MOMENTS, moment_launches(precision, P));
    for (int p = 1; p < kNumPlans; ++p) {
      const int b = P.tile_begin[p - 1], e = P.tile_begin[p];
      if (e == b) continue;
      int cps = 1;  // the grid: the largest CTAs per SM of the plan's degrees, within its kernel's limit
      for (const MomJob& j : P.jobs)
        if (j.plan == p) cps = std::max(cps, c->ctas_per_sm[1][j.L]);
      cps = std::min(cps, moment_ctas(plan_kmax(p)));
      const int grid = std::min((e - b + kThreads / 32 - 1) / (kThreads / 32), cps * c->num_sms);
      TRY_LAUNCH(launch_moments(p, -1, d_jobs, tiles + b, e - b, counters + kAnyCounter + p, d_geoms, parts, grid,
                                st));
    }
  }
  {
    PhaseScope ps(c, TCM_PHASE_FINALIZE, 1);
    TRY_LAUNCH(launch_finalize(d_jobs, (int)P.jobs.size(), parts, d_geoms, c->d_imap, c->d_fmap, c->d_imap_off,
                               static_cast<double*>(c->gpart.p), st));
  }
  return TCM_OK;
}

// The pass over the systems' atoms before the moment pass (syspass.cu): step a1 for the systems
// whose centre or radius is not given, and the low-degree sums of the mixed path for every
// system with a computed moment job.
struct SysPlan {
  std::vector<SysJob> jobs;
  int n1 = 0, n2 = 0;            // tiles of pass 1 (centroid) and pass 2 (radius, low-degree sums)
  std::vector<int> of_system;   // system -> index of its SysJob, or -1
  int rows = 0;
};

// used[s]: system s takes part in the call; low[s]: its low-degree sums are needed.
void plan_sys(const tcm_system* systems, int n_systems, const std::vector<char>& used, const std::vector<char>& low,
              SysPlan& S) {
  S.of_system.assign(std::max(n_systems, 0), -1);
  for (int s = 0; s < n_systems; ++s) {
    if (!used[s]) continue;
    const tcm_system& sy = systems[s];
    const bool nc = !sy.has_center;
    const bool nr = nc || sy.radius < 0.0;  // a radius given without its centre is recomputed
    const bool nl = !low.empty() && low[s];
    if (!nc && !nr && !nl) continue;
    SysJob j{};
    j.xyzq = sy.xyzq;
    j.n = sy.n;
    j.dtype = sy.dtype;
    j.geom = s;
    j.need_center = nc;
    j.need_radius = nr;
    j.need_low = nl;
    j.atoms_per_tile = sys_tile_atoms(sy.n);
    j.n_tiles = (int)std::max<long long>(1, (sy.n + j.atoms_per_tile - 1) / j.atoms_per_tile);
    j.tile_base = S.rows;
    S.rows += j.n_tiles;
    j.sum_row = -1;
    const int ji = (int)S.jobs.size();
    j.first1 = nc ? S.n1 : -1;
    j.first2 = (nr || nl) ? S.n2 : -1;
    if (nc) S.n1 += j.n_tiles;
    if (nr || nl) S.n2 += j.n_tiles;
    S.of_system[s] = ji;
    S.jobs.push_back(j);
  }
  for (SysJob& j : S.jobs)  // one sum row per system after the tile rows
    if (j.need_low) j.sum_row = S.rows++;
}

// Mixed path: every computed moment job takes its degrees l <= 2 from its system's low sums.
void link_low(const SysPlan& S, Plan& P) {
  for (MomJob& j : P.jobs) {
    const int si = S.of_system[j.geom];
    if (si < 0 || !S.jobs[si].need_low) continue;
    j.low_base = S.jobs[si].sum_row;
    j.low_tiles = 1;
  }
}

// Partial rows and tickets of the system pass; the tickets are zeroed when allocated and every
// launch leaves them zero.
int ensure_sys_buffers(tcm_ctx* c, const SysPlan& S) {
  TRY(dev_ensure(c, c->gpart, (size_t)std::max(S.rows, 1) * kSysPart * sizeof(double)));
  void* before = c->systk.p;
  TRY(dev_ensure(c, c->systk, std::max<size_t>(2 * S.jobs.size(), 64) * sizeof(int)));
  if (c->systk.p != before) TRY_CUDA(cudaMemsetAsync(c->systk.p, 0, c->systk.cap, c->stream));
  TRY(dev_ensure(c, c->systiles, (size_t)std::max(S.n1 + S.n2, 1) * sizeof(SysTile)));
  return TCM_OK;
}

int run_sys(tcm_ctx* c, const SysPlan& S, const SysJob* d_sj, SysGeom* d_geo, cudaStream_t st) {
  if (S.jobs.empty()) return TCM_OK;
  PhaseScope ps(c, TCM_PHASE_GEOM, sys_launches(S.n1, S.n2));
  SysTile* t1 = static_cast<SysTile*>(c->systiles.p);
  TRY_LAUNCH(launch_sys(d_sj, t1, S.n1, t1 + S.n1, S.n2, static_cast<double*>(c->gpart.p),
                        static_cast<int*>(c->systk.p), d_geo, st));
  return TCM_OK;
}

// The tile lists of the call (moment pass and system pass), written on the device from the
// groups and system jobs: the first launch of a call (it depends on nothing queued before it).
int run_expand(tcm_ctx* c, const std::vector<MomGroup>& groups, const MomJob* d_jobs, const MomGroup* d_groups,
               const SysPlan& S, const SysJob* d_sj, cudaStream_t st) {
  if (groups.empty() && S.jobs.empty()) return TCM_OK;
  PhaseScope ps(c, TCM_PHASE_GEOM, 1);
  SysTile* t1 = static_cast<SysTile*>(c->systiles.p);
  TRY_LAUNCH(launch_expand_tiles(d_groups, (int)groups.size(), d_jobs, static_cast<MomTile*>(c->tiles.p), d_sj,
                                 (int)S.jobs.size(), t1, t1 + S.n1, st));
  return TCM_OK;
}

SysGeom host_geom(const tcm_system& s) {
  SysGeom g{};
  for (int d = 0; d < 3; ++d) {
    g.c[d] = s.has_center ? s.center[d] : 0.0;
    g.chi[d] = (float)g.c[d];
    g.clo[d] = (float)(g.c[d] - (double)g.chi[d]);
  }
  g.a = s.radius >= 0.0 ? s.radius : 0.0;
  return g;
}

void identity(double* r) {
  for (int k = 0; k < 9; ++k) r[k] = (k % 4 == 0) ? 1.0 : 0.0;
}

// Host tables --------------------------------------------------------------------

int build_tables(tcm_ctx* c) {
  std::vector<double> fmap;
  std::vector<int> imap_off, imap;
  finalize_tables(imap_off, imap, fmap);
  TRY_CUDA(cudaMalloc(&c->d_fmap, fmap.size() * sizeof(double)));
  TRY_CUDA(cudaMalloc(&c->d_imap, imap.size() * sizeof(int)));
  TRY_CUDA(cudaMalloc(&c->d_imap_off, imap_off.size() * sizeof(int)));
  TRY_CUDA(cudaMemcpy(c->d_fmap, fmap.data(), fmap.size() * sizeof(double), cudaMemcpyHostToDevice));
  TRY_CUDA(cudaMemcpy(c->d_imap, imap.data(), imap.size() * sizeof(int), cudaMemcpyHostToDevice));
  TRY_CUDA(cudaMemcpy(c->d_imap_off, imap_off.data(), imap_off.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<double> zt(contract_table_size());
  contract_tables(zt.data());
  TRY_CUDA(cudaMalloc(&c->d_ztab, zt.size() * sizeof(double)));
  TRY_CUDA(cudaMemcpy(c->d_ztab, zt.data(), zt.size() * sizeof(double), cudaMemcpyHostToDevice));
  return TCM_OK;
}

void free_ctx(tcm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_fmap);
  cudaFree(c->d_ztab);
  cudaFree(c->d_imap);
  cudaFree(c->d_imap_off);
  for (DevBuf* b : {&c->desc, &c->partials, &c->gpart, &c->systk, &c->systiles, &c->counters, &c->moms, &c->escr,
                     &c->dpart, &c->tiles})
    cudaFree(b->p);
  for (auto& st : c->stage) {
    if (st.host) cudaFreeHost(st.host);
    if (st.ev) cudaEventDestroy(st.ev);
  }
  if (c->pinned_small) cudaFreeHost(c->pinned_small);
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

int check_ctx(tcm_ctx* c) {
  if (!c) return set_err(TCM_EINVAL, "null context");
  TRY_CUDA(cudaSetDevice(c->device));
  return TCM_OK;
}

}  // namespace

int tcm::record_error(int code, const char* msg) { return set_err(code, "%s", msg); }

extern "C" {

const char* tcm_last_error(void) { return g_err; }

int tcm_ctx_create(tcm_ctx_t* out, int lmax_cap, void* cuda_stream) {
  if (!out) return set_err(TCM_EINVAL, "tcm_ctx_create: null output pointer");
  *out = nullptr;
  if (lmax_cap < 0 || lmax_cap > TCM_LMAX_MAX)
    return set_err(TCM_EINVAL, "tcm_ctx_create: lmax_cap %d outside [0, %d]", lmax_cap, TCM_LMAX_MAX);
  tcm_ctx* c = new (std::nothrow) tcm_ctx();
  if (!c) return set_err(TCM_ENOMEM, "tcm_ctx_create: host allocation failed");
  for (int L = 0; L <= kLmaxMax; ++L) {
    c->atoms_per_thread[0][L] = 32;  // FP64: 32 atoms per lane (1,024 per warp tile)
    c->atoms_per_thread[1][L] = 64;  // mixed: 64 atoms per lane (2,048 per warp tile)
    c->ctas_per_sm[0][L] = c->ctas_per_sm[1][L] = TCM_MOMENT_CTAS_PER_SM;
    c->plan_l[L] = 1;
  }
  int rc = TCM_OK;
  do {
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
      rc = set_err(TCM_ECUDA, "tcm_ctx_create: no usable CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    c->lmax_cap = lmax_cap;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if ((rc = build_tables(c)) != TCM_OK) break;
    for (auto& st : c->stage)
      if (cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming) != cudaSuccess) {
        rc = set_err(TCM_ECUDA, "tcm_ctx_create: cudaEventCreate failed");
        break;
      }
    if (rc != TCM_OK) break;
    if (cudaHostAlloc(&c->pinned_small, 256, cudaHostAllocDefault) != cudaSuccess) {
      rc = set_err(TCM_ENOMEM, "tcm_ctx_create: cudaHostAlloc failed");
      break;
    }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c->cap_stream = nullptr;  // graphs unavailable; calls launch directly
    }
  } while (0);
  if (rc != TCM_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return TCM_OK;
}

void tcm_ctx_destroy(tcm_ctx_t c) { free_ctx(c); }

int tcm_ctx_set_stream(tcm_ctx_t c, void* cuda_stream) {
  TRY(check_ctx(c));
  TRY_CUDA(cudaStreamSynchronize(c->stream));
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return TCM_OK;
}

int tcm_ctx_set_tiling(tcm_ctx_t c, int precision, int atoms_per_lane) {
  TRY(check_ctx(c));
  if (precision != TCM_FP64 && precision != TCM_MIXED) return set_err(TCM_EINVAL, "tcm_ctx_set_tiling: bad precision");
  if (atoms_per_lane < 1 || atoms_per_lane > 4096)
    return set_err(TCM_EINVAL, "tcm_ctx_set_tiling: atoms_per_lane outside [1, 4096]");
  for (int L = 0; L <= kLmaxMax; ++L) c->atoms_per_thread[precision == TCM_FP64 ? 0 : 1][L] = atoms_per_lane;
  ++c->cfg_gen;
  return TCM_OK;
}

int tcm_ctx_set_tiling_l(tcm_ctx_t c, int precision, int lmax, int atoms_per_lane, int ctas_per_sm) {
  TRY(check_ctx(c));
  if (precision != TCM_FP64 && precision != TCM_MIXED) return set_err(TCM_EINVAL, "tcm_ctx_set_tiling_l: bad precision");
  if (lmax < 0 || lmax > kLmaxMax) return set_err(TCM_EINVAL, "tcm_ctx_set_tiling_l: lmax outside [0, %d]", kLmaxMax);
  if (atoms_per_lane < 1 || atoms_per_lane > 4096)
    return set_err(TCM_EINVAL, "tcm_ctx_set_tiling_l: atoms_per_lane outside [1, 4096]");
  const int cmax = precision == TCM_FP64 ? TCM_MOMENT_CTAS_PER_SM : moment_ctas(kKmaxF32Small);
  if (ctas_per_sm < 1 || ctas_per_sm > cmax)
    return set_err(TCM_EINVAL, "tcm_ctx_set_tiling_l: ctas_per_sm outside [1, %d]", cmax);
  c->atoms_per_thread[precision == TCM_FP64 ? 0 : 1][lmax] = atoms_per_lane;
  c->ctas_per_sm[precision == TCM_FP64 ? 0 : 1][lmax] = ctas_per_sm;
  ++c->cfg_gen;
  return TCM_OK;
}

int tcm_ctx_get_tiling_l(tcm_ctx_t c, int precision, int lmax, int* atoms_per_lane, int* ctas_per_sm) {
  TRY(check_ctx(c));
  if (precision != TCM_FP64 && precision != TCM_MIXED) return set_err(TCM_EINVAL, "tcm_ctx_get_tiling_l: bad precision");
  if (lmax < 0 || lmax > kLmaxMax) return set_err(TCM_EINVAL, "tcm_ctx_get_tiling_l: lmax outside [0, %d]", kLmaxMax);
  if (atoms_per_lane) *atoms_per_lane = c->atoms_per_thread[precision == TCM_FP64 ? 0 : 1][lmax];
  if (ctas_per_sm) *ctas_per_sm = c->ctas_per_sm[precision == TCM_FP64 ? 0 : 1][lmax];
  return TCM_OK;
}

int tcm_ctx_set_chunking_l(tcm_ctx_t c, int lmax, int kmax) {
  TRY(check_ctx(c));
  if (lmax < 0 || lmax > kLmaxMax) return set_err(TCM_EINVAL, "tcm_ctx_set_chunking_l: lmax outside [0, %d]", kLmaxMax);
  if (kmax != plan_kmax(1) && kmax != plan_kmax(2))
    return set_err(TCM_EINVAL, "tcm_ctx_set_chunking_l: kmax %d is not %d or %d", kmax, plan_kmax(1), plan_kmax(2));
  c->plan_l[lmax] = kmax == plan_kmax(1) ? 1 : 2;
  ++c->cfg_gen;
  return TCM_OK;
}

int tcm_ctx_get_chunking_l(tcm_ctx_t c, int lmax, int* kmax, int* n_chunks) {
  TRY(check_ctx(c));
  if (lmax < 0 || lmax > kLmaxMax) return set_err(TCM_EINVAL, "tcm_ctx_get_chunking_l: lmax outside [0, %d]", kLmaxMax);
  if (kmax) *kmax = plan_kmax(c->plan_l[lmax]);
  if (n_chunks) *n_chunks = moments_nchunks(c->plan_l[lmax], lmax);
  return TCM_OK;
}

int tcm_ctx_set_graphs(tcm_ctx_t c, int mode) {
  TRY(check_ctx(c));
  if (mode < 0 || mode > 2) return set_err(TCM_EINVAL, "tcm_ctx_set_graphs: mode %d outside [0, 2]", mode);
  c->graphs = mode;
  return TCM_OK;
}

int tcm_ctx_graph_stats(tcm_ctx_t c, int64_t* captures, int64_t* launches) {
  TRY(check_ctx(c));
  if (captures) *captures = c->graph_captures;
  if (launches) *launches = c->graph_launches;
  return TCM_OK;
}

int tcm_ctx_set_profiling(tcm_ctx_t c, int enable) {
  TRY(check_ctx(c));
  c->prof = enable != 0;
  return TCM_OK;
}

int tcm_ctx_read_profile(tcm_ctx_t c, double* ms, int64_t* launches) {
  TRY(check_ctx(c));
  TRY_CUDA(cudaStreamSynchronize(c->stream));
  double acc[TCM_NPHASES] = {};
  acc[TCM_PHASE_HOST] = c->host_ms;
  c->host_ms = 0.0;
  for (auto& m : c->marks) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) acc[m.phase] += t;
    c->ev_pool.push_back(m.a);
    c->ev_pool.push_back(m.b);
  }
  c->marks.clear();
  for (int k = 0; k < TCM_NPHASES; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = c->launches[k];
    c->launches[k] = 0;
  }
  return TCM_OK;
}

int tcm_prepare(tcm_ctx_t c, tcm_system* s) {
  TRY(check_ctx(c));
  TRY(check_system(s, "tcm_prepare"));
  if (geom_known(*s)) return TCM_OK;
  std::vector<char> used(1, 1);
  SysPlan S;
  plan_sys(s, 1, used, {}, S);
  std::vector<SysGeom> geoms{host_geom(*s)};
  Packer pk;
  const size_t o_geo = pk.add(geoms), o_sj = pk.add(S.jobs);
  TRY(ensure_sys_buffers(c, S));
  char* base = nullptr;
  TRY(upload(c, pk, &base));
  SysGeom* d_geo = reinterpret_cast<SysGeom*>(base + o_geo);
  const SysJob* d_sj = reinterpret_cast<SysJob*>(base + o_sj);
  TRY(run_expand(c, {}, nullptr, nullptr, S, d_sj, c->stream));
  TRY(run_sys(c, S, d_sj, d_geo, c->stream));
  TRY_CUDA(cudaMemcpyAsync(c->pinned_small, d_geo, sizeof(SysGeom), cudaMemcpyDeviceToHost, c->stream));
  TRY_CUDA(cudaStreamSynchronize(c->stream));
  const SysGeom* g = static_cast<const SysGeom*>(c->pinned_small);
  for (int d = 0; d < 3; ++d) s->center[d] = g->c[d];
  s->has_center = 1;
  s->radius = g->a;
  return TCM_OK;
}

int tcm_moments(tcm_ctx_t c, const tcm_system* s, const double* rot, int lmax, int precision, tcm_moments_t* out) {
  TRY(check_ctx(c));
  TRY(check_system(s, "tcm_moments"));
  if (!out || !out->q) return set_err(TCM_EINVAL, "tcm_moments: null output");
  if (!aligned16(out->q)) return set_err(TCM_EINVAL, "tcm_moments: output must be 16-byte aligned");
  if (lmax < 0 || lmax > c->lmax_cap)
    return set_err(TCM_EINVAL, "tcm_moments: lmax %d outside [0, %d]", lmax, c->lmax_cap);
  if (precision != TCM_FP64 && precision != TCM_MIXED) return set_err(TCM_EINVAL, "tcm_moments: bad precision");
  Plan P;
  MomJob j{};
  j.xyzq = s->xyzq;
  j.n = s->n;
  j.dtype = s->dtype;
  j.L = lmax;
  j.geom = 0;
  if (rot)
    std::memcpy(j.rot, rot, 9 * sizeof(double));
  else
    identity(j.rot);
  j.out = out->q;
  int next = 0;
  plan_job(c, precision, j, next);
  P.jobs.push_back(j);
  P.n_tile_ids = next;
  build_tiles(precision, P);
  std::vector<char> used(1, 1), low(1, precision == TCM_MIXED ? 1 : 0);
  SysPlan S;
  plan_sys(s, 1, used, low, S);
  link_low(S, P);
  std::vector<SysGeom> geoms{host_geom(*s)};
  Packer pk;
  const size_t o_geo = pk.add(geoms), o_job = pk.add(P.jobs), o_tile = pk.add(P.groups), o_sj = pk.add(S.jobs);
  TRY(ensure_moment_buffers(c, precision, P));
  TRY(ensure_sys_buffers(c, S));
  char* base = nullptr;
  TRY(upload(c, pk, &base));
  SysGeom* d_geo = reinterpret_cast<SysGeom*>(base + o_geo);
  const SysJob* d_sj = reinterpret_cast<SysJob*>(base + o_sj);
  TRY(run_expand(c, P.groups, reinterpret_cast<MomJob*>(base + o_job), reinterpret_cast<MomGroup*>(base + o_tile), S,
                 d_sj, c->stream));
  TRY(run_sys(c, S, d_sj, d_geo, c->stream));
  TRY(run_moments(c, precision, P, reinterpret_cast<MomJob*>(base + o_job), d_geo, c->stream));
  out->lmax = lmax;
  if (!geom_known(*s)) {
    TRY_CUDA(cudaMemcpyAsync(c->pinned_small, d_geo, sizeof(SysGeom), cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(cudaStreamSynchronize(c->stream));
    const SysGeom* g = static_cast<const SysGeom*>(c->pinned_small);
    for (int d = 0; d < 3; ++d) out->center[d] = g->c[d];
    out->radius = g->a;
  } else {
    for (int d = 0; d < 3; ++d) out->center[d] = s->center[d];
    out->radius = s->radius;
  }
  return TCM_OK;
}

int tcm_energy(tcm_ctx_t c, const tcm_moments_t* A, const tcm_moments_t* B, const double* R0, int lmax, double* E) {
  TRY(check_ctx(c));
  if (!A || !B || !R0 || !E || !A->q || !B->q) return set_err(TCM_EINVAL, "tcm_energy: null argument");
  if (lmax < 0 || lmax > c->lmax_cap || lmax > A->lmax || lmax > B->lmax)
    return set_err(TCM_EINVAL, "tcm_energy: lmax %d exceeds the moments' lmax or the context cap", lmax);
  const double R = std::sqrt(R0[0] * R0[0] + R0[1] * R0[1] + R0[2] * R0[2]);
  if (!(R > A->radius + B->radius))
    return set_err(TCM_ENOTCONV, "tcm_energy: |R0| = %.17g <= a_A + a_B = %.17g (Eq. (mainCond))", R,
                   A->radius + B->radius);
  std::vector<MomJob> jobs(2);
  std::memset(jobs.data(), 0, 2 * sizeof(MomJob));
  jobs[0].out = A->q;
  jobs[0].L = A->lmax;
  jobs[1].out = B->q;
  jobs[1].L = B->lmax;
  std::vector<SysGeom> geoms(2);
  std::memset(geoms.data(), 0, 2 * sizeof(SysGeom));
  geoms[0].a = A->radius;
  geoms[1].a = B->radius;
  std::vector<PairDesc> items(1);
  items[0] = PairDesc{0, 1, 0, 1, lmax, kBLab, 0, {}};
  pair_frame(R0, items[0]);
  Packer pk;
  const size_t o_job = pk.add(jobs), o_geo = pk.add(geoms), o_it = pk.add(items);
  char* base = nullptr;
  TRY(upload(c, pk, &base));
  TRY(dev_ensure(c, c->escr, 64));
  double* dE = static_cast<double*>(c->escr.p);
  {
    PhaseScope ps(c, TCM_PHASE_CONTRACT, 1);
    TRY_LAUNCH(launch_contract(reinterpret_cast<PairDesc*>(base + o_it), 1, lmax,
                               reinterpret_cast<MomJob*>(base + o_job), reinterpret_cast<SysGeom*>(base + o_geo),
                               c->d_ztab, nullptr, dE, nullptr, nullptr, c->stream));
  }
  TRY_CUDA(cudaMemcpyAsync(c->pinned_small, dE, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TRY_CUDA(cudaStreamSynchronize(c->stream));
  *E = *static_cast<const double*>(c->pinned_small);
  return TCM_OK;
}

int tcm_rotate_moments(tcm_ctx_t c, int64_t n, const tcm_moments_t* in, const double* rot, tcm_moments_t* out) {
  TRY(check_ctx(c));
  if (n < 0) return set_err(TCM_EINVAL, "tcm_rotate_moments: negative count");
  if (n == 0) return TCM_OK;
  if (!in || !rot || !out) return set_err(TCM_EINVAL, "tcm_rotate_moments: null argument");
  if (n > (1LL << 30)) return set_err(TCM_EINVAL, "tcm_rotate_moments: too many sets");
  std::vector<RotDesc> sets(n);
  int Lmax = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!in[i].q || !out[i].q) return set_err(TCM_EINVAL, "tcm_rotate_moments: set %lld has a null moment pointer", (long long)i);
    if (out[i].lmax < 0 || out[i].lmax > c->lmax_cap || out[i].lmax > in[i].lmax)
      return set_err(TCM_EINVAL, "tcm_rotate_moments: set %lld: output lmax %d outside [0, min(input lmax %d, cap %d)]",
                     (long long)i, out[i].lmax, in[i].lmax, c->lmax_cap);
    for (int k = 0; k < 9; ++k)
      if (!std::isfinite(rot[9 * i + k])) return set_err(TCM_EINVAL, "tcm_rotate_moments: set %lld: non-finite rotation", (long long)i);
    sets[i].in = in[i].q;
    sets[i].out = out[i].q;
    sets[i].L = out[i].lmax;
    std::memcpy(sets[i].M, rot + 9 * i, 9 * sizeof(double));
    Lmax = std::max(Lmax, out[i].lmax);
    for (int d = 0; d < 3; ++d) out[i].center[d] = in[i].center[d];
    out[i].radius = in[i].radius;
  }
  Packer pk;
  const size_t o_set = pk.add(sets);
  char* base = nullptr;
  TRY(upload(c, pk, &base));
  PhaseScope ps(c, TCM_PHASE_CONTRACT, 1);
  TRY_LAUNCH(launch_rotate_moments(reinterpret_cast<RotDesc*>(base + o_set), (int)n, Lmax, c->d_ztab, c->stream));
  return TCM_OK;
}

int tcm_ctx_set_rotate_cached(tcm_ctx_t c, int enable) {
  TRY(check_ctx(c));
  c->rotate_cached = enable != 0;
  return TCM_OK;
}

namespace {
int energy_batch(tcm_ctx_t c, int n_systems, const tcm_system* systems, int64_t n_items, const tcm_pair_item* items,
                 int precision, double* E, int32_t* status, double* G);
}

namespace {
// The batched call, with its host wall time added to TCM_PHASE_HOST while profiling is on.
int timed_batch(tcm_ctx_t c, int n_systems, const tcm_system* systems, int64_t n_items, const tcm_pair_item* items,
                int precision, double* E, int32_t* status, double* G) {
  const auto t0 = std::chrono::steady_clock::now();
  const int rc = energy_batch(c, n_systems, systems, n_items, items, precision, E, status, G);
  if (c && c->prof) c->host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}
}  // namespace

int tcm_energy_batch(tcm_ctx_t c, int n_systems, const tcm_system* systems, int64_t n_items, const tcm_pair_item* items,
                     int precision, double* E, int32_t* status) {
  return timed_batch(c, n_systems, systems, n_items, items, precision, E, status, nullptr);
}

int tcm_gradients_batch(tcm_ctx_t c, int n_systems, const tcm_system* systems, int64_t n_items,
                        const tcm_pair_item* items, int precision, double* E, double* G, int32_t* status) {
  if (n_items > 0 && !G) return set_err(TCM_EINVAL, "tcm_gradients_batch: null gradient output");
  return timed_batch(c, n_systems, systems, n_items, items, precision, E, status, G);
}

namespace {
int energy_batch(tcm_ctx_t c, int n_systems, const tcm_system* systems, int64_t n_items, const tcm_pair_item* items,
                 int precision, double* E, int32_t* status, double* G) {
  TRY(check_ctx(c));
  if (n_items < 0 || n_systems < 0) return set_err(TCM_EINVAL, "tcm_energy_batch: negative count");
  if (n_items == 0) return TCM_OK;
  if (!systems || !items || !E) return set_err(TCM_EINVAL, "tcm_energy_batch: null argument");
  if (n_items > (1LL << 30)) return set_err(TCM_EINVAL, "tcm_energy_batch: too many items");
  if (precision != TCM_FP64 && precision != TCM_MIXED) return set_err(TCM_EINVAL, "tcm_energy_batch: bad precision");
  std::vector<char> used(n_systems, 0);
  for (int64_t k = 0; k < n_items; ++k) {
    const tcm_pair_item& it = items[k];
    if (it.a < 0 || it.a >= n_systems || it.b < 0 || it.b >= n_systems)
      return set_err(TCM_EINVAL, "tcm_energy_batch: item %lld refers to a system outside [0, %d)", (long long)k, n_systems);
    if (it.lmax < 0 || it.lmax > c->lmax_cap)
      return set_err(TCM_EINVAL, "tcm_energy_batch: item %lld lmax %d outside [0, %d]", (long long)k, it.lmax, c->lmax_cap);
    used[it.a] = used[it.b] = 1;
  }
  for (int s = 0; s < n_systems; ++s)
    if (used[s]) TRY(check_system(&systems[s], "tcm_energy_batch"));
  // host-known radii: reject non-convergent items before any work is queued
  for (int64_t k = 0; k < n_items; ++k) {
    const tcm_pair_item& it = items[k];
    if (geom_known(systems[it.a]) && geom_known(systems[it.b])) {
      const double R = std::sqrt(it.R0[0] * it.R0[0] + it.R0[1] * it.R0[1] + it.R0[2] * it.R0[2]);
      const double aa = systems[it.a].radius + systems[it.b].radius;
      if (!(R > aa))
        return set_err(TCM_ENOTCONV, "tcm_energy_batch: item %lld: |R0| = %.17g <= a_A + a_B = %.17g (Eq. (mainCond))",
                       (long long)k, R, aa);
    }
  }
  // moment jobs (A sides and unrotated B sides shared)
  Plan P;
  std::unordered_map<long long, int> job_of;  // unrotated jobs by (system, Lmax)
  job_of.reserve((size_t)std::min<int64_t>(n_items, 1 << 20) * 2);
  P.jobs.reserve((size_t)std::min<int64_t>(n_items, 1 << 20) * 2);
  std::vector<PairDesc> pd(n_items);
  int next_id = 0;
  size_t moff = 0;
  std::vector<size_t> job_moff;
  std::vector<MomJob> cached;  // unrotated sides served from a system's moment cache
  std::map<int, int> cached_of;
  auto get_job = [&](int sys, int L, int rot_item, const double* rot) {
    if (rot_item < 0 && systems[sys].moments && L <= systems[sys].moments_lmax) {
      auto c = cached_of.find(sys);
      if (c != cached_of.end()) return -2 - c->second;
      MomJob j{};
      j.L = systems[sys].moments_lmax;
      j.geom = sys;
      j.out = const_cast<double*>(systems[sys].moments);
      cached.push_back(j);
      cached_of[sys] = (int)cached.size() - 1;
      return -2 - ((int)cached.size() - 1);
    }
    const long long key = (long long)sys * (kLmaxMax + 1) + L;
    if (rot_item < 0) {  // rotated jobs are unique to their item: no lookup
      auto itr = job_of.find(key);
      if (itr != job_of.end()) return itr->second;
    }
    MomJob j{};
    j.xyzq = systems[sys].xyzq;
    j.n = systems[sys].n;
    j.dtype = systems[sys].dtype;
    j.L = L;
    j.geom = sys;
    if (rot)
      std::memcpy(j.rot, rot, 9 * sizeof(double));
    else
      identity(j.rot);
    plan_job(c, precision, j, next_id);
    job_moff.push_back(moff);
    moff += (size_t)(L + 1) * (L + 1);
    const int id = (int)P.jobs.size();
    P.jobs.push_back(j);
    if (rot_item < 0) job_of[key] = id;
    return id;
  };
  std::vector<EulerZYZ> rots;  // Euler record of W rotB per rotate-from-cache item
  for (int64_t k = 0; k < n_items; ++k) {
    const tcm_pair_item& it = items[k];
    const int ja = get_job(it.a, it.lmax, -1, nullptr);
    int jb;
    if (it.has_rot && c->rotate_cached && systems[it.b].moments && it.lmax <= systems[it.b].moments_lmax) {
      // B's cached lab-frame moments, taken into the frame by W rotB inside the contraction
      double W[9];
      frame_rotation(it.R0, W);
      jb = get_job(it.b, it.lmax, -1, nullptr);
      pd[k] = PairDesc{ja, jb, it.a, it.b, it.lmax, kBRotate, (long long)rots.size(), {}};
      pair_frame(it.R0, pd[k]);
      double M[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          M[3 * i + j] = W[3 * i + 0] * it.rotB[0 + j] + W[3 * i + 1] * it.rotB[3 + j] + W[3 * i + 2] * it.rotB[6 + j];
      rots.push_back(euler_zyz(M));
      continue;
    }
    if (it.has_rot) {
      // B is moved per item anyway: fold the rotation W that takes R0hat to z into its
      // atom transform, so the contraction receives B's moments already in that frame.
      double W[9], M[9];
      frame_rotation(it.R0, W);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          M[3 * i + j] = W[3 * i + 0] * it.rotB[0 + j] + W[3 * i + 1] * it.rotB[3 + j] + W[3 * i + 2] * it.rotB[6 + j];
      jb = get_job(it.b, it.lmax, (int)k, M);
    } else {
      jb = get_job(it.b, it.lmax, -1, nullptr);
    }
    pd[k] = PairDesc{ja, jb, it.a, it.b, it.lmax, it.has_rot ? kBInFrame : kBLab, 0, {}};
    pair_frame(it.R0, pd[k]);
  }
  P.n_tile_ids = next_id;
  TRY(dev_ensure(c, c->moms, std::max<size_t>(moff, 1) * sizeof(double)));
  for (size_t ji = 0; ji < P.jobs.size(); ++ji) P.jobs[ji].out = static_cast<double*>(c->moms.p) + job_moff[ji];
  build_tiles(precision, P);
  std::vector<char> low(n_systems, 0);
  if (precision == TCM_MIXED)
    for (const MomJob& j : P.jobs) low[j.geom] = 1;
  SysPlan S;
  plan_sys(systems, n_systems, used, low, S);
  link_low(S, P);
  // cached sides follow the computed jobs in the descriptor array (not finalised)
  const int n_computed = (int)P.jobs.size();
  for (auto& d : pd) {
    if (d.jobA <= -2) d.jobA = n_computed + (-2 - d.jobA);
    if (d.jobB <= -2) d.jobB = n_computed + (-2 - d.jobB);
  }
  int Lmax_items = 0;
  for (int64_t k = 0; k < n_items; ++k) Lmax_items = std::max(Lmax_items, (int)items[k].lmax);
  std::vector<SysGeom> geoms(std::max(n_systems, 1));
  for (int s = 0; s < n_systems; ++s) geoms[s] = host_geom(systems[s]);
  Packer pk;
  const size_t o_geo = pk.add(geoms), o_job = pk.add2(P.jobs, cached), o_tile = pk.add(P.groups), o_sj = pk.add(S.jobs),
               o_it = pk.add(pd), o_rot = pk.add(rots);
  // every buffer the launches touch is sized before anything is queued (no reallocation
  // may happen while a graph is being captured)
  TRY(ensure_sys_buffers(c, S));
  TRY(ensure_moment_buffers(c, precision, P));
  char* base = nullptr;
  TRY(upload(c, pk, &base));
  SysGeom* d_geo = reinterpret_cast<SysGeom*>(base + o_geo);
  const MomJob* d_jobs = reinterpret_cast<MomJob*>(base + o_job);
  auto enqueue = [&](cudaStream_t st) -> int {
    const SysJob* d_sj = reinterpret_cast<SysJob*>(base + o_sj);
    TRY(run_expand(c, P.groups, d_jobs, reinterpret_cast<MomGroup*>(base + o_tile), S, d_sj, st));
    TRY(run_sys(c, S, d_sj, d_geo, st));
    TRY(run_moments(c, precision, P, d_jobs, d_geo, st));
    PhaseScope ps(c, TCM_PHASE_CONTRACT, 1);
    TRY_LAUNCH(launch_contract(reinterpret_cast<PairDesc*>(base + o_it), (int)n_items, Lmax_items, d_jobs, d_geo,
                               c->d_ztab, rots.empty() ? nullptr : reinterpret_cast<double*>(base + o_rot), E,
                               status, G, st));
    return TCM_OK;
  };
  if (!c->graphs || c->prof || !c->cap_stream) return enqueue(c->stream);
  // Replay a captured graph of the launch sequence when this call has the same shape and
  // buffers as the captured one (only the uploaded descriptor contents differ).
  std::vector<long long> key = {precision, G != nullptr, (long long)(uintptr_t)G, (long long)S.jobs.size(),
                                (long long)S.n1, (long long)S.n2, (long long)P.jobs.size(), P.n_tile_ids,
                                (long long)n_items, Lmax_items, (long long)o_geo, (long long)o_job, (long long)o_tile,
                                (long long)o_sj, (long long)o_it, (long long)o_rot, (long long)(uintptr_t)c->systiles.p,
                                (long long)rots.empty(), (long long)(uintptr_t)base, (long long)(uintptr_t)c->gpart.p,
                                (long long)(uintptr_t)c->systk.p, (long long)(uintptr_t)c->partials.p,
                                (long long)(uintptr_t)c->counters.p, (long long)(uintptr_t)E, (long long)(uintptr_t)status,
                                (long long)P.groups.size(), (long long)P.n_tiles, (long long)(uintptr_t)c->tiles.p,
                                (long long)c->cfg_gen};
  for (int L = 0; L <= kLmaxMax + 1; ++L) key.push_back(P.tile_begin[L]);
  if (!c->gexec || key != c->gkey) {
    // by default capture only a shape seen twice in a row: a stream of changing shapes
    // (continuous batching) launches directly instead of paying a capture per call
    if (c->graphs == 1 && key != c->gkey_seen) {
      c->gkey_seen = key;
      return enqueue(c->stream);
    }
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    TRY_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int64_t saved[TCM_NPHASES];
    std::copy(c->launches, c->launches + TCM_NPHASES, saved);
    const int rc = enqueue(c->cap_stream);
    for (int k = 0; k < TCM_NPHASES; ++k) c->launches[k] = saved[k];
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != TCM_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc != TCM_OK ? rc : set_err(TCM_ECUDA, "graph capture failed: %s", cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->gexec = nullptr;
      return set_err(TCM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    }
    c->gkey = key;
    ++c->graph_captures;
  }
  TRY_CUDA(cudaGraphLaunch(c->gexec, c->stream));
  ++c->graph_launches;
  c->launches[TCM_PHASE_GEOM] += (S.jobs.empty() ? 0 : sys_launches(S.n1, S.n2)) +
                                  ((P.groups.empty() && S.jobs.empty()) ? 0 : 1);
  c->launches[TCM_PHASE_MOMENTS] += moment_launches(precision, P);
  c->launches[TCM_PHASE_FINALIZE] += 1;
  c->launches[TCM_PHASE_CONTRACT] += 1;
  return TCM_OK;
}
}  // namespace

namespace {
// Eq. (Coulomb) for n items (B rotated by rotB[9 k] about its centre, at separation R0[3 k]);
// energies to the device array dE.  Asynchronous.
int direct_items(tcm_ctx_t c, const tcm_system* A, const tcm_system* B, int64_t n, const double* rotB,
                 const double* R0, double* dE) {
  tcm_system sys[2] = {*A, *B};
  for (auto& s : sys)
    if (s.has_center) s.radius = std::max(s.radius, 0.0);  // the direct sum needs centres only
  std::vector<char> used(2, 1);
  SysPlan S;
  plan_sys(sys, 2, used, {}, S);
  std::vector<SysGeom> geoms{host_geom(sys[0]), host_geom(sys[1])};
  std::vector<double> xf(12 * (size_t)n);
  for (int64_t k = 0; k < n; ++k) {
    if (rotB)
      std::memcpy(&xf[12 * k], rotB + 9 * k, 9 * sizeof(double));
    else
      identity(&xf[12 * k]);
    for (int d = 0; d < 3; ++d) xf[12 * k + 9 + d] = R0[3 * k + d];
  }
  Packer pk;
  const size_t o_geo = pk.add(geoms), o_xf = pk.add(xf), o_sj = pk.add(S.jobs);
  const int nblk = direct_blocks(A->n);
  TRY(ensure_sys_buffers(c, S));
  TRY(dev_ensure(c, c->dpart, (size_t)std::max<int64_t>(nblk * n, 1) * sizeof(double)));
  char* base = nullptr;
  TRY(upload(c, pk, &base));
  SysGeom* d_geo = reinterpret_cast<SysGeom*>(base + o_geo);
  const SysJob* d_sj = reinterpret_cast<SysJob*>(base + o_sj);
  TRY(run_expand(c, {}, nullptr, nullptr, S, d_sj, c->stream));
  TRY(run_sys(c, S, d_sj, d_geo, c->stream));
  const int nlaunch = (int)((n + 65534) / 65535) * (nblk > 0 ? 2 : 1);
  PhaseScope ps(c, TCM_PHASE_DIRECT, nlaunch);
  TRY_LAUNCH(launch_direct(A->xyzq, A->n, A->dtype, B->xyzq, B->n, B->dtype, d_geo,
                           reinterpret_cast<double*>(base + o_xf), (int)n, static_cast<double*>(c->dpart.p), nblk, dE,
                           c->stream));
  return TCM_OK;
}
}  // namespace

int tcm_direct(tcm_ctx_t c, const tcm_system* A, const tcm_system* B, const double* rotB, const double* R0, double* E) {
  TRY(check_ctx(c));
  TRY(check_system(A, "tcm_direct A"));
  TRY(check_system(B, "tcm_direct B"));
  if (!R0 || !E) return set_err(TCM_EINVAL, "tcm_direct: null argument");
  TRY(dev_ensure(c, c->escr, 64));
  double* dE = static_cast<double*>(c->escr.p);
  TRY(direct_items(c, A, B, 1, rotB, R0, dE));
  TRY_CUDA(cudaMemcpyAsync(c->pinned_small, dE, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TRY_CUDA(cudaStreamSynchronize(c->stream));
  *E = *static_cast<const double*>(c->pinned_small);
  return TCM_OK;
}

int tcm_direct_batch(tcm_ctx_t c, const tcm_system* A, const tcm_system* B, int64_t n_items, const double* rotB,
                     const double* R0, double* E) {
  TRY(check_ctx(c));
  TRY(check_system(A, "tcm_direct_batch A"));
  TRY(check_system(B, "tcm_direct_batch B"));
  if (n_items < 0) return set_err(TCM_EINVAL, "tcm_direct_batch: negative count");
  if (n_items == 0) return TCM_OK;
  if (!R0 || !E) return set_err(TCM_EINVAL, "tcm_direct_batch: null argument");
  if (n_items > (1LL << 30)) return set_err(TCM_EINVAL, "tcm_direct_batch: too many items");
  if ((int64_t)direct_blocks(A->n) * n_items > (1LL << 34))
    return set_err(TCM_EINVAL, "tcm_direct_batch: A's blocks x items exceeds the partial-sum buffer limit");
  return direct_items(c, A, B, n_items, rotB, R0, E);
}

}  // extern "C"
