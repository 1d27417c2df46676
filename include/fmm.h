/*
 * fmm.h - C ABI of the GB300 relativistic space-charge FMM.
 *
 * The library computes, for N charged particles of a beam, the lab-frame
 * space-charge fields of Section 3 of Kan, Kaertner, Le Borne, Zemke,
 * "A GPU-parallelized interpolation-based fast multipole method for the
 * relativistic space-charge field calculation" (arXiv 2302.07567):
 *
 *   E_i = 1/(4 pi eps0)      sum_{j != i} q_j gamma_j  g(x_i, x_j)       (Eq. 3.1)
 *   B_i = 1/(4 pi eps0 c0)   sum_{j != i} q_j p_j  x  g(x_i, x_j)
 *   g(x_i, x_j) = (x_i - x_j) / ((dx)^2 + (dy)^2 + gbar^2 (dz)^2)^(3/2)   (Eq. 3.2)
 *
 * with gamma_j = sqrt(1 + |p_j|^2) and gbar^2 = 1 + pbar.pbar, pbar the mean
 * momentum.  The sums are evaluated by the barycentric Lagrange dual tree
 * traversal FMM of the paper: a stretched k-d cluster tree (Algs. 1-2,
 * Appendix B), P2M/M2M (Algs. 3-5), the dual tree traversal under the
 * stretched admissibility condition (Eq. 4.x, Algs. 6-8, 11, 17), M2L and
 * P2P (Algs. 9-10) and L2L/L2P (Algs. 13-15).  Every stage runs as CUDA on
 * one GPU.  Units are SI: x in metres, p = gamma*beta dimensionless, q in
 * coulomb, E in V/m, B in tesla; eps0 = 8.8541878128e-12 F/m and
 * c0 = 299792458 m/s.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Device pointers are owned by the caller and must stay valid until the
 *   work queued on `stream` has finished.  Arrays are dense, row-major:
 *   [N,3] means x[3*i + k].
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * - Every function returns an fmm_status; none of them throws, aborts or
 *   prints.  The library never allocates device memory: scratch space comes
 *   from the workspace the caller attaches with fmm_plan_set_workspace.
 * - A plan is not thread safe; use one plan per host thread.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fmm_status {
  FMM_OK = 0,
  FMM_EINVAL = 1,       /* bad argument: N < 1, degree outside 1..12, leaf size < 2,
                           eta not finite or <= 0, unknown precision, NULL pointer  */
  FMM_ENOWORKSPACE = 2, /* no workspace attached, or smaller than required          */
  FMM_EOVERFLOW = 3,    /* an interaction-list capacity was exceeded; raise it with
                           fmm_plan_set_capacity, re-attach a workspace, call again  */
  FMM_ENONFINITE = 4,   /* x or p holds NaN or Inf                                   */
  FMM_ESTATE = 5,       /* fmm_field_adjoint before a successful fmm_field; export of
                           expansions an FMM_RECOMPUTE adjoint overwrote            */
  FMM_ECUDA = 6,        /* a CUDA runtime call failed (see fmm_last_cuda_error)      */
  FMM_EBOUNDS = 7       /* an index check of FMM_BOUNDS_CHECK failed                 */
} fmm_status;

typedef enum fmm_precision {
  FMM_FP64 = 0, /* every stage in double precision                                   */
  FMM_FP32 = 1  /* tree, boxes, gbar, traversal and interpolation setup in FP64;
                   P2M/M2M/M2L/P2P/L2L/L2P arithmetic in FP32 with FP32 accumulators
                   and compensated (Kahan) sums across source clusters and leaves    */
} fmm_precision;

typedef enum fmm_flags {
  FMM_RECOMPUTE = 1u,    /* one set of per-level expansions instead of two: the
                            adjoint's node weights W and adjoint moments Lambda are
                            written over the forward's locals L and multipoles M
                            (with FMM_GBAR_TERM, whose M2L^T reads M, Lambda keeps a
                            buffer of its own), so fmm_plan_workspace_bytes shrinks
                            by about 7.5 (n+1)^3 x (number of clusters) bytes
                            (FP32).  The target-side far field, which reads the
                            leaf locals, runs before the far-field chain that
                            overwrites them: in FP32 without FMM_GBAR_TERM as a
                            kernel of its own, after which the near field and the
                            chain run side by side as without the flag; in FP64 and
                            with FMM_GBAR_TERM inside the near-field kernel, which
                            then runs first, on the caller's stream (no second
                            stream).  A further adjoint call without a new fmm_field
                            recomputes the upward pass, M2L and L2L first;
                            fmm_plan_export of multipoles or locals after an
                            adjoint returns FMM_ESTATE                               */
  FMM_BOUNDS_CHECK = 2u, /* after the traversal (and the adjoint's source-major lists)
                            check on the device: node tables, the leaf order is a
                            permutation, list pairs in range, sorted and matching
                            their CSR offsets, and sum |S_t||S_s| = N^2 over the
                            lists; a failure returns FMM_EBOUNDS before any kernel
                            indexes through the bad value (costs one more wait)     */
  FMM_TIMING = 4u,       /* record CUDA events around each stage (fmm_plan_stats)    */
  FMM_TEST_POLY_KERNEL = 16u, /* test mode, FP64 plans, forward only: the kernel is the
                            polynomial g(R) = R (R_x^2 + R_y^2 + gbar^2 R_z^2 + 1),
                            of degree 3 in each variable, so with n >= 3 every
                            interpolation step is exact (Theorem 1, the lemma of
                            Appendix A) and the FMM equals the direct sum of this g
                            to rounding; E = k_e sum a_j g, B = k_e/c0 sum b_j x g */
  FMM_SIZE_AWARE = 8u,   /* not in the paper: in the traversal (Alg. 17) an admissible
                            pair with |S_t||S_s| < m^2 particle pairs (m = (n+1)^3) is
                            evaluated directly, as P2P of all leaf pairs under it,
                            instead of by M2L: fewer operations and no truncation
                            error for that pair                                     */
  FMM_SERIAL = 64u,      /* run every stage on the caller's stream, one kernel after
                            another.  By default independent branches share the GPU
                            on a second stream the plan owns (FP32 forward: near-field
                            P2P beside M2L and L2L; adjoint: the near field beside the
                            source side's far-field chain), which is faster at every
                            size measured; the serial order gives each kernel the GPU
                            to itself, so its stage time is its own duration (for
                            attributing time per kernel), and each kernel then takes
                            every resident block slot.  Results are bitwise equal.   */
  FMM_GBAR_TERM = 32u    /* adjoint only (not in the paper): gbar is the function
                            sqrt(1 + pbar.pbar), pbar = (1/N) sum_j p_j, of Section 3
                            instead of a constant, so dL/dp gains
                            dL/dgbar * pbar / (N gbar) for every particle.  The tree,
                            its boxes and the lists stay fixed (gbar moves them only
                            through discrete decisions); gbar enters the FMM through
                            the kernel g of Eq. 3.2 alone, and dL/dgbar is the sum,
                            over the same P2P and M2L pairs, of the loss contracted
                            with dg/dgbar = -3 gbar R_z^2 R / (R_x^2 + R_y^2 +
                            gbar^2 R_z^2)^(5/2).  M2L^T then runs its generic kernel. */
} fmm_flags;

typedef struct fmm_plan_s* fmm_plan_t;

/* Create a plan for N particles (Alg. 12, FMM(S, s, N0, eta)).
 *   degree     interpolation degree n, 1..12: (n+1)^3 Chebyshev points per cluster
 *   leaf_size  N0 >= 2: the tree depth is kappa = 0 if N <= N0, else the least
 *              kappa with N0 * 2^kappa >= N (Section 8); every leaf holds at most N0
 *   eta        admissibility parameter of max(diam_s)/dist_s < eta (Eq. 4.x, Alg. 8)
 *   precision  FMM_FP64 or FMM_FP32;  flags: OR of fmm_flags.
 * The plan is host memory only; destroy it with fmm_plan_destroy. */
int fmm_plan_create(fmm_plan_t* out, int64_t N, int degree, int leaf_size, double eta,
                    int precision, unsigned flags);

/* Capacities of the P2P and M2L interaction lists (pairs of clusters) and of
 * the traversal frontier.  0 keeps the default.  Changing a capacity changes
 * the workspace size: query and attach it again afterwards. */
int fmm_plan_set_capacity(fmm_plan_t plan, int64_t p2p_pairs, int64_t m2l_pairs,
                          int64_t frontier_pairs);

/* Bytes of device workspace the plan needs (256-byte aligned start required). */
int fmm_plan_workspace_bytes(fmm_plan_t plan, size_t* bytes);

/* Attach caller-owned device memory of at least fmm_plan_workspace_bytes. The
 * plan keeps the pointer; the caller frees it after fmm_plan_destroy.  Also
 * uploads the plan's node tables (a synchronous copy on the legacy stream). */
int fmm_plan_set_workspace(fmm_plan_t plan, void* device_ptr, size_t bytes);

/* Forward pass: fields of all N particles (Alg. 12).
 *   x, p  device, [N,3] float64;  q  device, [N] float64
 *   E, B  device, [N,3]; float64 for FMM_FP64 plans, float32 for FMM_FP32 plans
 * Rows of E and B follow the input order.  The call queues work on `stream`,
 * waits once on it after the traversal (to read the list sizes and the device
 * error flags) and returns; the remaining kernels may still be running.  In
 * FP32 plans part of the work (M2L, L2L) runs on a second stream the plan
 * owns, beside the near field; the call joins it into `stream`, so work
 * queued later on `stream` is ordered after all of it.
 * On FMM_EOVERFLOW / FMM_ENONFINITE nothing is written to E and B. */
int fmm_field(fmm_plan_t plan, const double* x, const double* p, const double* q,
              void* E, void* B, void* stream);

/* Forward pass of a tracking step (not in the paper, whose Alg. 12 builds
 * the tree and the lists for every field evaluation).  The tree's membership
 * (which particles form each cluster) and the P2P and M2L lists of the last
 * successful fmm_field or fmm_field_reuse on this plan are kept; gbar, every
 * cluster's box (the bounding box of its unchanged members at the new
 * positions, Section 2) and every stage after the tree are recomputed.  If
 * every M2L pair is still admissible (Alg. 8) under the new boxes and gbar,
 * the kept lists are used as they are: they still partition all N^2 particle
 * pairs into direct and admissible pairs, so the result carries the FMM's
 * error bound (Section 4), though it may differ from fmm_field on the same
 * input, whose traversal can choose other pairs.  Otherwise, or with no
 * earlier forward on the plan, the call builds tree and lists anew exactly as
 * fmm_field does and sets *rebuilt = 1 (else 0; rebuilt may be NULL).  A call
 * that follows a stale attempt builds at once without trying the kept lists
 * (the next call tries again): on large beams the particles' relative motion
 * carries some of the millions of M2L pairs across the admissibility bound
 * every step, and the wasted attempts then cost every second step only.
 * Arguments, outputs, the one wait on `stream` and the errors as fmm_field;
 * with unchanged x and p the result equals fmm_field's bit for bit. */
int fmm_field_reuse(fmm_plan_t plan, const double* x, const double* p, const double* q, void* E, void* B,
                    void* stream, int* rebuilt);

/* Relativistic Boris push over one time step (not in the paper; the particle
 * pusher a tracking code runs between field evaluations).  With u = p (the
 * momentum gamma beta), a_j = q_j dt / (2 mass c0) and gamma(u) = sqrt(1+|u|^2):
 *   u-  = u + a E,   t = (a c0 / gamma(u-)) B,   s = 2 t / (1 + |t|^2),
 *   u+  = u- + (u- + u- x t) x s,   u' = u+ + a E,   x' = x + c0 dt u' / gamma(u'),
 * E, B the fields at x (V/m, T).  x, p: device [N,3] float64, updated in place
 * (p then lives at the half step); q: device [N] float64 (coulomb); E, B: device
 * [N,3] in the precision field_precision (FMM_FP32: float, FMM_FP64: double), as
 * fmm_field writes them; mass in kg > 0, dt in s.  Asynchronous on `stream`.
 * FMM_EINVAL for NULL pointers, N < 1, a bad precision, mass <= 0 or a
 * non-finite mass or dt. */
int fmm_boris_push(double* x, double* p, const double* q, int64_t N, const void* E, const void* B,
                   int field_precision, double mass, double dt, void* stream);

/* Adjoint of the forward pass of the same plan (not in the paper).  For the
 * loss L = sum_i wE_i . E_i + wB_i . B_i it returns dL/dx [N,3], dL/dp [N,3]
 * and dL/dq [N] (device float64), the exact derivative of the FMM operator
 * with the tree, its boxes, the interaction lists and gbar held fixed at the
 * values of the last fmm_field call (with FMM_GBAR_TERM, gbar follows p).  wE, wB: device [N,3] of the plan's
 * output type.  x, p, q must be the arrays of the last fmm_field call, still
 * unchanged.  Returns FMM_ESTATE if no successful fmm_field preceded it.
 * The source side's far field runs on a second stream the plan owns, beside
 * the target-side kernel on `stream`; the call joins it into `stream` before
 * it returns, so work queued later on `stream` is ordered after all of it. */
int fmm_field_adjoint(fmm_plan_t plan, const double* x, const double* p, const double* q,
                      const void* wE, const void* wB, double* dx, double* dp, double* dq,
                      void* stream);

/* A recorded step (not in the paper): fmm_field and, with wE != NULL,
 * fmm_field_adjoint on these arguments, kept by the plan as two CUDA graphs
 * (the forward, the adjoint) and replayed by fmm_step_graph_launch.  A replay
 * runs the kernels of the calls it recorded in the same order, so on the same
 * input its results equal theirs bit for bit; it spares the host the launch of
 * every kernel (about 300 per forward and adjoint), which bounds the step of a
 * small beam.  The graphs hold the pointers: x, p, q, wE, wB, E, B, dx, dp, dq
 * must stay allocated at these addresses while the graphs exist, and a replay
 * reads what they hold then (a tracking or optimisation loop updates x, p, q,
 * wE, wB in place).  The call first runs the step once as usual, so it
 * returns that step's errors (after FMM_EOVERFLOW the caller grows the
 * capacities and calls again), then records it.  Arguments as fmm_field and
 * fmm_field_adjoint (dx, dp, dq may be NULL when wE is NULL).  FMM_EINVAL for
 * NULL arguments, a legacy default stream (NULL, cudaStreamLegacy or
 * cudaStreamPerThread, which cannot be recorded), FMM_TIMING or
 * FMM_BOUNDS_CHECK (they time or wait on the host); FMM_ECUDA, and no graphs,
 * if recording fails.  fmm_plan_set_capacity, fmm_plan_set_workspace and
 * fmm_plan_destroy drop the graphs. */
int fmm_step_graph_create(fmm_plan_t plan, const double* x, const double* p, const double* q, const void* wE,
                          const void* wB, void* E, void* B, double* dx, double* dp, double* dq, void* stream);

/* Replays the recorded step on `stream` and waits for it: the forward, a read
 * of its list sizes and device error flags, then (if recorded) the adjoint.
 * Returns what fmm_field would return on the arrays' current contents; on
 * FMM_EOVERFLOW or FMM_ENONFINITE the adjoint is not replayed and nothing is
 * written to E, B, dx, dp, dq (the graphs stay; after growing the capacities,
 * which drops them, the caller records anew).  FMM_ESTATE without a recorded
 * step. */
int fmm_step_graph_launch(fmm_plan_t plan, void* stream);

/* Drops the recorded step, if any. */
int fmm_step_graph_destroy(fmm_plan_t plan);

/* Copies `bytes` from src to dst with a kernel on the GPU's SMs (16-byte
 * loads and stores) instead of the copy engine (not in the paper; a helper
 * for callers whose inputs and results live in host memory).  dst and src
 * are device memory of the current device, managed memory, or pinned or
 * registered host memory (cudaHostAlloc, cudaHostRegister), in either
 * direction; both 16-byte aligned and bytes a multiple of 16.  Measured on
 * this GPU: the first copy from or to a 0.4 GB pinned buffer after a 2^24
 * field and adjoint step took 5-8 ms with this kernel and 9-30 ms with
 * cudaMemcpyAsync; with the buffer just copied both take 1.9 ms.  The kernel
 * shares the SMs with whatever else runs.  Asynchronous on `stream`.
 * FMM_EINVAL for NULL or misaligned arguments and for memory a kernel cannot
 * address (pageable host memory, another device's memory). */
int fmm_copy(void* dst, const void* src, size_t bytes, void* stream);

typedef struct fmm_stats {
  int64_t N, nodes, leaves;
  int32_t degree, leaf_size, kappa, precision;
  double eta, gbar, length_unit, mass_unit;
  int64_t p2p_pairs, m2l_pairs;          /* cluster pairs in the interaction lists   */
  double p2p_interactions;               /* sum |S_t||S_s| over P2P pairs minus N     */
  double m2l_interactions;               /* m2l_pairs * (n+1)^6                       */
  int64_t cap_p2p, cap_m2l, cap_frontier;
  /* stage times of the last calls in ms (FMM_TIMING only, else 0):
     forward: 0 setup, 1 tree, 2 upward pass, 3 traversal with the ordering
     of the lists, 4 the host read of the list sizes, 5 M2L, 6 L2L,
     7 P2P+L2P (FP32: the near-field P2P, which runs beside M2L and L2L),
     16 FP32: L2P and the output after both, 13 whole forward, 17 P2M (part of 2);
     adjoint: 8 L2P^T + L2L^T, 9 M2L^T, 10 M2M^T, 11 near-field particle
     kernel (FP32: both roles; else the target side with its far field),
     12 source side (FP32: far field and chain rule; else near + far + chain
     rule), 14 whole adjoint, 15 source-major lists and any recomputation.
     With FMM_SERIAL every stage has the GPU to itself, so a stage time is the
     duration of its own kernels. */
  double stage_ms[18];
} fmm_stats;

/* Copy the plan's dimensions, list sizes and stage times (synchronises the
 * stream of the last call when FMM_TIMING is set). */
int fmm_plan_stats(fmm_plan_t plan, fmm_stats* out);
/* sizeof(fmm_stats) in this build, for bindings to check their layout. */
size_t fmm_stats_bytes(void);

/* Inspection of intermediate results of the last fmm_field, copied to host
 * memory (synchronous).  `bytes` must be at least the size given below, with
 * C = 2^(kappa+1) - 1 nodes numbered breadth first from 1 (Section 8) and
 * m = (degree+1)^3 proxy points ordered nu = nu1 + (n+1) nu2 + (n+1)^2 nu3.
 *   FMM_EXPORT_GBAR       double[1]
 *   FMM_EXPORT_PERM       int32[N]    input index of the particle at leaf-order slot
 *   FMM_EXPORT_NODES      int64[C][2] (first slot, count) of nodes 1..C
 *   FMM_EXPORT_BBOX       double[C][6] (a_x, a_y, a_z, b_x, b_y, b_z) (Section 2)
 *   FMM_EXPORT_AXIS       int32[C]    split axis of Alg. 1, -1 at leaves
 *   FMM_EXPORT_P2P        int32[n][2] (target, source), sorted; n = stats.p2p_pairs
 *   FMM_EXPORT_M2L        int32[n][2] (target, source), sorted; n = stats.m2l_pairs
 *   FMM_EXPORT_MULTIPOLE  double[C][4][m]: sum_j l_nu(x_j) q_j gamma_j and
 *                         sum_j l_nu(x_j) q_j p_j (Section 3, Algs. 3-5)
 *   FMM_EXPORT_LOCAL      double[C][6][m]: cumulative local fields (E_mu, B_mu) of
 *                         Eq. 2.9 without the 1/(4 pi eps0) and 1/c0 prefactors */
typedef enum fmm_export {
  FMM_EXPORT_GBAR = 0, FMM_EXPORT_PERM = 1, FMM_EXPORT_NODES = 2, FMM_EXPORT_BBOX = 3,
  FMM_EXPORT_AXIS = 4, FMM_EXPORT_P2P = 5, FMM_EXPORT_M2L = 6, FMM_EXPORT_MULTIPOLE = 7,
  FMM_EXPORT_LOCAL = 8
} fmm_export;
int fmm_plan_export(fmm_plan_t plan, int what, void* host_dst, size_t bytes);

/* Brute force of Section 5 (Alg. 10 with S_t = S_s = S, i != j) in float64 for
 * the T target rows listed in `targets` (device int64[T]; NULL = all N, T = N).
 * gbar >= 1 is the stretch factor of Eq. 3.2, e.g. fmm_stats.gbar of a plan run
 * on the same particles (FMM_EINVAL otherwise).  E, B: device float64 [T,3].
 * Work is O(T N); it is the reference the library's error reports use. */
int fmm_direct_field(const double* x, const double* p, const double* q, int64_t N,
                     const int64_t* targets, int64_t T, double gbar, double* E, double* B,
                     void* stream);

void fmm_plan_destroy(fmm_plan_t plan);
const char* fmm_strerror(int status);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char* fmm_last_cuda_error(void);
int fmm_version(void);
/* Number of CUDA kernels this process has launched through the library so far
 * (all plans, all threads); differences around a region count its launches. */
int64_t fmm_kernel_launches(void);

/* Measurement helper (the paper has no counterpart): the FP32 fused
 * multiply-add rate of the current device in TFLOP/s (FMA = 2 flop), the peak
 * the library's ALU-bound kernels are reported against.  A kernel on every SM
 * runs independent FMA chains, in the scalar form (paired = 0: one FMA per
 * lane per instruction) or the paired form (paired = 1: two per lane per
 * instruction, as the particle kernels issue their arithmetic); the best of
 * three timed launches after one warm-up counts.  Synchronous, a few ms.
 *   sink  device memory of at least SMs x 8 x 256 floats (written, never read;
 *         FMM_EINVAL if smaller or NULL) */
int fmm_fp32_fma_rate(void* sink, size_t sink_bytes, int paired, double* tflops, void* stream);

/* gbar of a beam without allocating anything (the paper has no counterpart;
 * the value is the gbar of Eq. 3.2 that fmm_field computes, bit for bit).
 * For callers that cannot allocate device memory or attach a workspace: code
 * running during stream capture, allocation-free tracking loops, hosts whose
 * device memory is owned by a pool.  The partial sums live in a fixed scratch
 * array inside the library (~200 KB, held by every GPU that loads the library
 * until exit).
 *   p     device [N,3] float64 momenta;  gbar  device double[1] output
 *   N     1 .. FMM_NOALLOC_MAX_N, else FMM_EINVAL (nothing is launched)
 * The work runs on the device current in the calling thread, and `stream` must
 * belong to that device (FMM_EINVAL otherwise).  The first call on a device looks
 * up the scratch address (cudaGetSymbolAddress) and should come before any stream
 * capture; a cudaDeviceReset invalidates that address, so do not call this entry
 * point on a device after resetting it.  All calls share the scratch array: calls
 * whose work overlaps on the GPU race on it. */
#define FMM_NOALLOC_MAX_N 16777216
int fmm_gamma_bar_noalloc(const double* p, int64_t N, double* gbar, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
