/*
 * tcm.h -- C ABI of the GB300 two-center multipole (TCM) library (libtcm.so).
 *
 * The method (Solov'yov, Yakubovich, Solov'yov, Greiner, "Two center multipole
 * expansion method: application to macromolecular systems") computes the Coulomb
 * interaction energy of two separated charge systems A and B,
 *
 *   Eq. (Coulomb):    U = sum_i sum_j q_i q_j / |R0 + r_j^B - r_i^A|,
 *
 * where r^A, r^B are positions about each system's centre and R0 points from the
 * centre of A to the centre of B, in two steps:
 *
 *   Eq. (multipole):  Q_lm = sum_i q_i r_i^l sqrt(4 pi / (2l+1)) Y_lm(theta_i, phi_i)
 *                     for each system, 0 <= l <= Lmax, and
 *   Eq. (Formula):    U_mult = sum_{l1,l2=0}^{Lmax} sum_{m1,m2} (-1)^(l1+M) R0^-(L+1)
 *                       sqrt(4 pi (2L)! / ((2 l1)! (2 l2)!)) (l1 l2 L; m1 m2 -M)
 *                       Q^A_{l1 m1} Q^B_{l2 m2} Y*_{LM}(R0hat),  L = l1 + l2, M = m1 + m2,
 *
 * valid when |R0| exceeds the sum of the two system radii (Eq. (mainCond)).
 *
 * Conventions
 *   - Y_lm: orthonormal spherical harmonics with the Condon-Shortley phase.
 *   - Moments use Y_lm (not Y*_lm) and the separation harmonic is conjugated, as the
 *     paper prints them; l1 and l2 each run over 0..Lmax (square truncation).
 *   - Units follow the input: charges in e and distances in Angstrom give energies in
 *     e^2/Angstrom (multiply by 332.06 for kcal/mol).
 *   - Packed moments: (Lmax+1)^2 doubles; degree l starts at index l*l and holds
 *     Re Q_l0, Re Q_l1, Im Q_l1, ..., Re Q_ll, Im Q_ll.  For real charges
 *     Q_l,-m = (-1)^m conj(Q_lm), so m < 0 is not stored.
 *   - A rotation acts about the system's own centre: r' = rot * (x - c), rot
 *     row-major 3x3.  Moments are reported in the frame after rotation.
 *
 * Memory and threads
 *   - Coordinate records, packed moments and batch energy outputs are DEVICE
 *     pointers owned by the caller; the context owns its scratch (grown on first
 *     use, never freed until tcm_ctx_destroy) and its tables.
 *   - All work is queued on the context's stream.  Calls that return a host value
 *     (tcm_energy, tcm_direct, tcm_prepare, tcm_moments when it must compute a
 *     centre or radius) synchronise that stream; the others are asynchronous.
 *   - A context is used by one host thread at a time.
 *   - The calls stage their descriptors through pinned host buffers and may wait on the
 *     host for a staging slot, so they cannot be captured into a caller's CUDA graph; the
 *     library captures and replays its own launch sequence instead (tcm_ctx_set_graphs).
 *
 * Errors
 *   Every call returns a tcm_status; nothing throws across the ABI.  On failure
 *   tcm_last_error() returns a message for the calling thread.
 */
#ifndef TCM_H_
#define TCM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest Lmax with compiled kernels.  Moments use (Lmax+1)^2 components; the
 * contraction evaluates irregular harmonics up to order 2 Lmax. */
#define TCM_LMAX_MAX 24

typedef enum {
  TCM_OK = 0,
  TCM_EINVAL = 1,    /* bad argument: null pointer, Lmax out of range, misaligned buffer, bad dtype */
  TCM_ENOTCONV = 2,  /* |R0| <= a_A + a_B: the expansion does not converge (Eq. (mainCond)) */
  TCM_ENOMEM = 3,    /* device or pinned host allocation failed */
  TCM_ECUDA = 4,     /* a CUDA runtime call or kernel launch failed */
  TCM_ETIMEOUT = 5   /* reserved: a bounded device-side wait ran out */
} tcm_status;

typedef enum { TCM_F32 = 0, TCM_F64 = 1 } tcm_dtype;

typedef enum {
  TCM_FP64 = 0,  /* every step in double precision */
  TCM_MIXED = 1  /* moment recurrence and per-atom products in float on radius-scaled
                    coordinates; block partials, cross-block reduction, tables and the
                    contraction in double */
} tcm_precision;

typedef struct tcm_ctx* tcm_ctx_t;

/* One charge system. */
typedef struct {
  const void* xyzq; /* device: n records (x, y, z, q); float[4] (16-byte aligned) for
                       TCM_F32, double[4] (16-byte aligned) for TCM_F64 */
  int64_t n;        /* number of charges, >= 0 */
  int32_t dtype;    /* tcm_dtype */
  int32_t has_center; /* nonzero: center[] is the system centre; zero: the centroid of the
                         positions (unit masses) is used */
  double center[3];
  double radius;    /* a = max_i |x_i - c| (any a' >= a is also accepted); < 0: computed */
  const double* moments; /* optional device cache: packed moments about center (from tcm_moments,
                            lmax moments_lmax); batches use it for every unrotated side with
                            lmax <= moments_lmax instead of recomputing; requires has_center and
                            radius >= 0; NULL = none */
  int32_t moments_lmax;
  int32_t pad_;
} tcm_system;

/* Moments of one system (output of tcm_moments, input of tcm_energy). */
typedef struct {
  double* q;        /* device: (lmax+1)^2 packed doubles, caller-owned */
  int32_t lmax;
  int32_t pad_;
  double center[3]; /* centre the moments are taken about */
  double radius;    /* system radius about that centre */
} tcm_moments_t;

/* One (pair, orientation) of a batch. */
typedef struct {
  int32_t a, b;     /* indices into the batch's systems array */
  int32_t lmax;     /* 0 <= lmax <= TCM_LMAX_MAX */
  int32_t has_rot;  /* nonzero: rotB applies to B about its centre */
  double rotB[9];
  double R0[3];     /* centre of A -> centre of B */
} tcm_pair_item;

/* Create a context on the current CUDA device, bound to cuda_stream (a cudaStream_t;
 * NULL = legacy default stream).  lmax_cap (0..TCM_LMAX_MAX) bounds the Lmax of every
 * later call.  On success *ctx is set; on failure *ctx is NULL. */
int tcm_ctx_create(tcm_ctx_t* ctx, int lmax_cap, void* cuda_stream);

/* Release the context and everything it owns.  Synchronises its stream.  NULL is a no-op. */
void tcm_ctx_destroy(tcm_ctx_t ctx);

/* Rebind the context to another stream (takes effect for later calls). */
int tcm_ctx_set_stream(tcm_ctx_t ctx, void* cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char* tcm_last_error(void);

/* Phases of the path, for tracing and benchmarks. */
typedef enum {
  TCM_PHASE_GEOM = 0,     /* a1: centre and radius; set-up of the moment pass (tile list, low-degree sums) */
  TCM_PHASE_MOMENTS = 1,  /* a2: per-atom moment accumulation and per-tile CTA reduction */
  TCM_PHASE_FINALIZE = 2, /* a3: cross-tile reduction in double and normalisation */
  TCM_PHASE_CONTRACT = 3, /* a4 + a5: irregular harmonics at R0 and the two-center contraction */
  TCM_PHASE_DIRECT = 4,   /* a6: exact pairwise sum */
  TCM_PHASE_HOST = 5,     /* host wall time inside tcm_energy_batch / tcm_gradients_batch (planning,
                             descriptor staging and upload, launching or graph replay); no kernels */
  TCM_NPHASES = 6
} tcm_phase;

/* Tiling of the moment pass for one precision, every degree: each warp of the moment kernels
 * takes tiles of 32 x atoms_per_lane atoms (1..4096; defaults 64 for TCM_MIXED, 32 for
 * TCM_FP64).  A system's tiles, and so the rounding of its moments, depend only on its
 * atom count, its Lmax and this setting.  Used by the autotuner. */
int tcm_ctx_set_tiling(tcm_ctx_t ctx, int precision, int atoms_per_lane);

/* The moment-pass tiling of one degree lmax in [0, TCM_LMAX_MAX] at one precision: atoms per
 * lane of a warp tile (as above) and the resident CTAs per SM that the persistent grid of
 * that degree's launch is sized for (grid = min(work, ctas_per_sm x SMs) CTAs of four warps):
 * [1, 2] for TCM_FP64, [1, 3] for TCM_MIXED, where a launch's grid is held to what its
 * kernel is compiled for (2 CTAs per SM at the 160-accumulator chunk budget, 3 at 96; see
 * tcm_ctx_set_chunking_l).  Defaults: 32 (FP64) or 64 (mixed) atoms per lane, 2 CTAs per SM.
 * Set by the autotuner; results stay within the stated tolerances for any setting (only the
 * summation order of the atom sums changes).  tcm_ctx_get_tiling_l reads the current
 * setting. */
int tcm_ctx_set_tiling_l(tcm_ctx_t ctx, int precision, int lmax, int atoms_per_lane, int ctas_per_sm);
int tcm_ctx_get_tiling_l(tcm_ctx_t ctx, int precision, int lmax, int* atoms_per_lane, int* ctas_per_sm);

/* The L-chunking of the mixed path's moment pass for one degree lmax in [0, TCM_LMAX_MAX]:
 * each lane keeps at most kmax float accumulators of Eq. (multipole) in registers, so the
 * (lmax+1)^2 components are split into column chunks of at most kmax, each a tile that
 * re-reads its atoms.  kmax = 160 (default; kernel compiled for 2 CTAs per SM) or 96 (more
 * chunks, fewer registers, 3 CTAs per SM).  A batch whose degrees use both budgets runs one
 * moment launch per budget.  Set by the autotuner; like the tiling it changes only the
 * summation order.  tcm_ctx_get_chunking_l reads kmax and the resulting number of chunks
 * (either pointer may be NULL).  TCM_EINVAL for another kmax or lmax. */
int tcm_ctx_set_chunking_l(tcm_ctx_t ctx, int lmax, int kmax);
int tcm_ctx_get_chunking_l(tcm_ctx_t ctx, int lmax, int* kmax, int* n_chunks);

/* CUDA-graph replay of tcm_energy_batch.  A call's launch sequence (tile list, centres and
 * radii, low-degree sums, the moment pass -- one launch over all degrees per chunk budget
 * present in TCM_MIXED, one per degree in TCM_FP64 --, finalisation, contraction) is
 * captured into a graph and replayed by later calls with the same launch shapes, settings
 * and buffers (item count, job and tile counts, tiling and chunking,
 * output pointers); the descriptors are uploaded per call, so the orientations, pairs and
 * systems may change.  mode 0: launch kernel by kernel; mode 1 (default): capture a shape
 * when two calls in a row have it (a stream of changing shapes launches directly instead of
 * paying a capture per call); mode 2: capture every new shape on its first call.  Off while
 * phase timing is on. */
int tcm_ctx_set_graphs(tcm_ctx_t ctx, int mode);

/* Number of graph captures and graph launches so far (either pointer may be NULL). */
int tcm_ctx_graph_stats(tcm_ctx_t ctx, int64_t* captures, int64_t* launches);

/* Enable (1) or disable (0) phase timing: the context then records a CUDA event pair on
 * its stream around every phase it queues.  Off by default. */
int tcm_ctx_set_profiling(tcm_ctx_t ctx, int enable);

/* Synchronise the context stream, then write the milliseconds spent in each phase
 * (ms[TCM_NPHASES], NULL allowed; zero unless profiling was on) and the number of kernels
 * launched per phase (launches[TCM_NPHASES], NULL allowed) since the previous read, and
 * reset both. */
int tcm_ctx_read_profile(tcm_ctx_t ctx, double* ms, int64_t* launches);

/* Step a1 (Section II: the centres may be any point; centroid by default): compute the
 * centroid (if !has_center) and the radius (if radius < 0) of *s on the device, write
 * them into *s and set has_center.  Synchronous. */
int tcm_prepare(tcm_ctx_t ctx, tcm_system* s);

/* Eq. (multipole): moments Q_lm, 0 <= l <= lmax, of system s about its centre, after
 * the optional rotation rot (row-major 3x3 host array, NULL = identity).
 * out->q must hold (lmax+1)^2 doubles on the device; out->lmax, out->center and
 * out->radius are written.  precision is a tcm_precision.  Asynchronous unless the
 * centre or radius has to be computed (then it synchronises once, as tcm_prepare). */
int tcm_moments(tcm_ctx_t ctx, const tcm_system* s, const double* rot, int lmax, int precision,
                tcm_moments_t* out);

/* Eq. (Formula): two-center energy of A and B at separation R0 (host double[3], from
 * the centre of A to the centre of B), truncated at lmax (<= both moment sets' lmax).
 * Returns TCM_ENOTCONV when |R0| <= A->radius + B->radius.  Writes the energy to the
 * host double *E.  Synchronous. */
int tcm_energy(tcm_ctx_t ctx, const tcm_moments_t* A, const tcm_moments_t* B, const double* R0,
               int lmax, double* E);

/* Rotation of cached moments (the moments of a system turned about its centre, without its
 * atoms): for each of the n sets, out[i].q receives the moments, 0 <= l <= out[i].lmax, of the
 * system whose lab-frame moments are in[i].q after the rotation rot + 9 i (row-major 3x3 host
 * array) about its centre -- what tcm_moments with that rotation gives, up to rounding, in
 * O(lmax^3) per set instead of O(atoms x lmax^2).  Each degree l is rotated with its Wigner
 * matrix D^l (Section II: the solid harmonics of a given l transform among themselves); the
 * Euler angles are taken from the rotation's quaternion.
 *   in[i].q, out[i].q: device, packed as tcm_moments_t; out[i].lmax <= in[i].lmax and <= the
 *   context cap; out[i].q may equal in[i].q (in place), sets must not otherwise overlap.
 *   out[i].center and out[i].radius are copied from in[i] (a rotation about the centre changes
 *   neither).
 * Asynchronous on the context stream. */
int tcm_rotate_moments(tcm_ctx_t ctx, int64_t n, const tcm_moments_t* in, const double* rot,
                       tcm_moments_t* out);

/* Rotated sides of tcm_energy_batch from the moment cache (off by default): when on, an item
 * with has_rot whose system b carries a moment cache with moments_lmax >= the item's lmax
 * takes B's moments from that cache, rotated inside the contraction kernel by the Wigner
 * matrices of (frame rotation) x rotB, instead of recomputing them from B's atoms.  The
 * energies agree with the recomputed ones within the stated tolerances. */
int tcm_ctx_set_rotate_cached(tcm_ctx_t ctx, int enable);

/* Batched Eq. (multipole) + Eq. (Formula): for every item, the moments of system a
 * and of system b (rotated by rotB about its centre) at the item's lmax and their
 * two-center energy at R0.  Moment sets shared by several items (same system, lmax
 * and no rotation) are computed once.  Systems without a centre or radius get them
 * on the device (step a1) without a host round trip.
 *   E:      device, n_items doubles (NaN for an item that does not converge)
 *   status: device, n_items int32 (TCM_OK or TCM_ENOTCONV), or NULL
 * Systems that carry a moment cache (tcm_system.moments) reuse it for their unrotated sides
 * (and for rotated sides too under tcm_ctx_set_rotate_cached).
 * Returns TCM_ENOTCONV at once if a host-known radius already violates Eq. (mainCond).
 * Asynchronous; results are ready when the context stream reaches this point.
 * Each item's result does not depend on the other items in the batch. */
int tcm_energy_batch(tcm_ctx_t ctx, int n_systems, const tcm_system* systems, int64_t n_items,
                     const tcm_pair_item* items, int precision, double* E, int32_t* status);

/* Forces and torques with the batched energies (the paper names forces as a use of Eq.
 * (Formula) but prints no formula; these are the exact derivatives of the truncated energy):
 * as tcm_energy_batch, and for every item G[9 k .. 9 k + 8] (device doubles) receives
 *   F_B   = -grad_R0 E   (force on B; the force on A is -F_B),
 *   tau_A = torque on A about its centre,  tau_B = torque on B about its centre,
 * all in the lab frame, as minus the derivative of E under a rotation of that system about
 * its own centre.  With the square truncation tau_A + tau_B + R0 x F_B = 0.  Computed in the
 * frame where R0hat = z from the same moments (O(Lmax^3) per item); NaN for an item that does
 * not converge.  E may be the same buffer tcm_energy_batch would take. */
int tcm_gradients_batch(tcm_ctx_t ctx, int n_systems, const tcm_system* systems, int64_t n_items,
                        const tcm_pair_item* items, int precision, double* E, double* G, int32_t* status);

/* Eq. (Coulomb): exact pairwise energy of A and B (B rotated by rotB about its centre,
 * NULL = identity) with the centre of B at the centre of A plus R0, in double
 * precision.  Writes the host double *E.  Synchronous. */
int tcm_direct(tcm_ctx_t ctx, const tcm_system* A, const tcm_system* B, const double* rotB,
               const double* R0, double* E);

/* Eq. (Coulomb) for many placements of B against A (a potential-energy-surface scan, Section
 * IV): for item k, B rotated by rotB + 9 k (host row-major 3x3 array per item, or NULL for
 * none) about its centre, with its centre at A's centre plus R0 + 3 k (host).  E: device,
 * n_items doubles.  Double precision, one CTA per (item, 256 atoms of A), fixed-order sums.
 * Asynchronous on the context stream. */
int tcm_direct_batch(tcm_ctx_t ctx, const tcm_system* A, const tcm_system* B, int64_t n_items,
                     const double* rotB, const double* R0, double* E);

/* Largest atom count accepted by tcm_moments_noalloc, and the size in bytes of the fixed
 * device array it works in (about 0.69 MiB). */
#define TCM_NOALLOC_MAX_ATOMS 262144
#define TCM_NOALLOC_SCRATCH_BYTES 720128

/* The paper has no counterpart to this call; it exists for callers that cannot allocate
 * device memory.  Examples: code that must not let cudaMalloc/cudaFree synchronise the
 * device in the middle of its work, applications whose own allocator owns all device
 * memory, and plug-ins that are not allowed to create allocations.  A context
 * (tcm_ctx_create) allocates, so such callers use this instead of tcm_moments.
 *
 * It computes the same moments as tcm_moments, of system s, optionally rotated by rot
 * (row-major host double[9], NULL = identity), into q_out (device, (lmax+1)^2 packed
 * doubles, 16-byte aligned).  If center_radius_out is not NULL it receives (device,
 * 4 doubles) the centre and radius used: the given ones, or the centroid and radius
 * computed on the device when s has no centre or no radius.  precision is TCM_FP64 or
 * TCM_MIXED.  The work is queued on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream) and the call returns without waiting.
 *
 * Memory: instead of allocating, the call uses one fixed scratch array of
 * TCM_NOALLOC_SCRATCH_BYTES bytes defined in the library as device memory.  Every GPU that
 * loads the library holds its own copy until the process exits.  All calls on a GPU share
 * that array and it keeps the last call's contents (each call rewrites what it reads), so
 * calls whose work overlaps on the GPU race on it: serialise them (one stream, or events).
 * Limits: 0 <= s->n <= TCM_NOALLOC_MAX_ATOMS and 0 <= lmax <= TCM_LMAX_MAX; larger
 * requests return TCM_EINVAL with a message.
 * Set-up: the first call on each GPU (with that GPU current) looks up the scratch
 * address, copies the coefficient tables into it and waits for the device to finish;
 * make that first call before any stream capture.
 * Errors are reported as by the other calls (status code, tcm_last_error()). */
int tcm_moments_noalloc(const tcm_system* s, const double* rot, int lmax, int precision, double* q_out,
                        double* center_radius_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TCM_H_ */
