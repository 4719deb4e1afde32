/*
 * arp.h -- C ABI of the asymptotic parareal library for the 1D rotating
 * shallow-water system (Haut & Wingate, "An asymptotic parallel-in-time
 * method for highly oscillatory PDEs").
 *
 * Model (Sec. 6.1, Eq. 6.1 in the generic form of Eq. 1.1):
 *     du/dt + (1/eps) L u = N(u) + D u,   u = (v1, v2, h), x in [0, 2 pi) periodic,
 *     L_k = [[0, -1, i k F^-1/2], [1, 0, 0], [i k F^-1/2, 0, 0]]  (Fourier symbol),
 *     D_k = -nu k^4,   N(u) = -(v1 v1_x, v1 v2_x, (h v1)_x).
 *
 * STATE LAYOUT (every state buffer of this API):
 *     double, complex interleaved (re, im), shape [batch][3][H], H = N/2 + 1,
 *     field order (v1, v2, h), entry [b][f][k] = coefficient u_k of field f with
 *     u_f(x_j) = sum_{k=-N/2+1}^{N/2} u_k e^{i k x_j}, x_j = 2 pi j / N, and
 *     u_{-k} = conj(u_k).  The state space keeps wavenumbers k <= K = (N-1)/3
 *     (2/3 rule); inputs are projected onto it (bins above K are ignored and the
 *     imaginary parts of the k = 0 bins are taken as zero); outputs have exact
 *     zeros above K.
 *
 * OWNERSHIP: the caller owns every buffer passed in; the context owns its
 *     tables, workspaces and the parareal iterates.  Unless a function says
 *     otherwise, pointers are device pointers and work is enqueued on `stream`
 *     (a cudaStream_t passed as void*, NULL = the legacy default stream) and
 *     runs asynchronously; buffers must stay valid until it completes.
 *
 * ERRORS: every call returns an arp_status; nothing aborts and no C++
 *     exception crosses this boundary.  arp_last_error() gives a message for
 *     the last failing call on a context.  Waits inside kernels are bounded:
 *     a wait that gives up makes the call return ARP_ETIMEOUT and leaves the
 *     CUDA context usable, but the parareal iterate is then undefined until
 *     the next arp_set_initial.  After ARP_ECUDA the context should be
 *     destroyed.
 *
 * THREADS: a context may be used by one host thread at a time.
 */
#ifndef ARP_H
#define ARP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct arp_ctx arp_ctx;

typedef enum {
  ARP_OK = 0,
  ARP_EINVAL = 1,       /* invalid argument (size, pointer, option) */
  ARP_ENOMEM = 2,       /* device allocation failed */
  ARP_ECUDA = 3,        /* a CUDA call or kernel launch failed */
  ARP_ETIMEOUT = 4,     /* a bounded wait inside a kernel gave up */
  ARP_ENONFINITE = 5    /* a result contained NaN or Inf */
} arp_status;

typedef enum {
  ARP_FP64 = 0,         /* all arithmetic in FP64 */
  ARP_FP32 = 1,         /* fine and coarse bulk arithmetic in FP32; tables and
                           phases computed in FP64 and rounded; parareal
                           correction and norm in FP64 */
  ARP_TF32X3 = 2,       /* as ARP_FP32, but the real DFTs of the batched stages (the
                           ETDRK4 fine sweep, all states stepped together, and the
                           time average of arp_coarse_avg / arp_coarse_step) run as
                           dense GEMMs on the tensor cores (the library's own
                           tcgen05 kernel) with TF32 operands split into high and
                           low parts (three products, FP32 accumulation); the
                           serial coarse chain and the other fine schemes keep the
                           FP32 FFT path */
  ARP_BF16X2 = 3,       /* as ARP_TF32X3 with BF16 high and low parts (all four
                           products); about 16 significant bits per operand, so
                           its results miss the 1e-5 FP32 bar on the time average */
  ARP_BF16X3 = 4        /* as ARP_TF32X3 with BF16 high, middle and low parts (the
                           six products of order <= 2) */
} arp_precision;

typedef enum {
  ARP_OPT_T0 = 1,          /* averaging window in fast-time units (default dT/eps) */
  ARP_OPT_F = 2,           /* the free parameter F of Eq. 6.1 (default 1) */
  ARP_OPT_PRECISION = 3,   /* an arp_precision value (default ARP_FP64) */
  ARP_OPT_KMAX = 4,        /* iteration cap used by arp_parareal_solve (default 5) */
  ARP_OPT_TOL = 5,         /* stopping tolerance of arp_parareal_solve (default 0) */
  ARP_OPT_CHAIN = 6,       /* serial coarse chain: 0 = automatic (one thread-block cluster,
                              else a cooperative grid with bounded grid barriers, else one
                              launch per step; in FP64 with M > 16 the cooperative grid
                              first), 1 =
                              cooperative grid, 2 = launches, 3 = the cluster only; all give
                              the same result up to rounding (default 0) */
  ARP_OPT_FINE_BLOCK = 7,  /* FP32 fine sweep schedule: 0 = the tuned default for the grid size
                              (chosen offline from GB300 timings), 1 = N/4 threads per slice,
                              2 = N/2 threads (both at least 32, at most 512), 3 = N/8 threads
                              with both FFT lanes per butterfly and the ETDRK4 stage values in
                              shared memory (ETDRK4, N >= 256), 4 = N/8 threads with radix-16
                              transform stages and the stage values in shared memory (ETDRK4,
                              512 <= N <= 2048); where 3 or 4 does not apply the default does;
                              all are within the FP32 error bound, their results differ in the
                              last bits (default 0) */
  ARP_OPT_FINE_SCHEME = 8,  /* fine propagator F: 0 = ETDRK4 (Cox & Matthews, default), 1 = Strang
                               splitting (Algorithm 3: exact linear half steps around a midpoint
                               step of N), 2 = integrating-factor RK4 (classical RK4 on
                               e^{-t(-L/eps+D)} u, the comparator of Sec. 6.2); steps of size
                               h = dT/ceil(dT/dt); used by arp_fine_batch and the parareal
                               iteration */
  ARP_OPT_COARSE_SCHEME = 9,  /* coarse propagator G: 0 = the asymptotic slow solver
                                 (Algorithm 2, default), 1 = one Strang step of size dT of the
                                 full equation (standard parareal, Sec. 6.2); used by
                                 arp_coarse_step and the parareal chain.  arp_coarse_avg always
                                 computes the time average.  Batches (arp_batch_*) accept only
                                 the default schemes (ARP_EINVAL otherwise) */
  ARP_OPT_COARSE_GRID = 10,  /* coarse solver on a coarser spatial grid (Sec. 1's remark on a
                                coarser discretisation for the asymptotic solver): 0 (default) or
                                N = the fine grid; a power of two N_c in [8, N) runs the coarse chain
                                of the parareal iteration on the modes k <= (N_c - 1)/3 of an N_c
                                grid, the higher modes of U following from F - G alone.  Applies to
                                the asymptotic coarse scheme with the cluster chain
                                (ARP_OPT_CHAIN 0); allocates a sub-context of
                                arp_query_bytes(N_c, slices, M, precision) bytes on first use;
                                arp_coarse_avg and arp_coarse_step keep the fine grid */
  ARP_OPT_PIPELINE = 11,  /* arp_parareal_solve as a pipeline across iterations: 0 = off (one
                             level after another), 1 = on with chunks of
                             min(16, max(4, ceil(S/16))) links (default), n >= 2 = chunks
                             of n links.  The SMs are split
                             into two partitions (green contexts): one that holds the coarse
                             chain's thread-block cluster, one for the fine sweeps, which start
                             on a chunk's slices as soon as the chain has produced their start
                             states.  Results, level and change equal the level-by-level solve's
                             bit for bit.  Applies with the cluster chain (ARP_OPT_CHAIN 0 where
                             the automatic choice is the cluster: FP32, or FP64 with M <= 16;
                             or ARP_OPT_CHAIN 3), the asymptotic coarse scheme on the fine
                             grid and the FFT precisions; elsewhere, or where the partition
                             cannot be made, the solve runs level by level.  Allocates one
                             more [slices][3][H] FP64 buffer on first use */
  ARP_OPT_TEST_SKIP_ARRIVAL = 100  /* failure-detection test hook, cleared after one chain
                                      launch.  1 (or any non-zero value but 2): the chain runs
                                      as the cooperative grid and block 0 skips its first
                                      grid-barrier arrival.  2: the chain runs in the
                                      thread-block cluster (where one fits; ARP_OPT_CHAIN 0 or
                                      3) and CTA 0 does not send its first partial sums.
                                      Either way every bounded wait on them gives up (after
                                      about 1 s) and the call returns ARP_ETIMEOUT.  Level by
                                      level only: the pipelined solve is not taken while the
                                      hook is set */
} arp_option;

/*
 * arp_create: a context for one problem.
 *   N      grid points, a power of two in [8, 2048]
 *   eps    Rossby number (> 0; +inf switches the fast term off)
 *   nu     hyperviscosity coefficient (>= 0), D_k = -nu k^4 (Sec. 6.1; the
 *          printed +mu d^4/dx^4 is read as dissipation)
 *   slices number of parareal time slices S >= 1 (Sec. 3)
 *   dT     slice length (coarse step) > 0; the horizon is T = S dT
 *   dt     fine step, 0 < dt <= dT; the fine propagator takes
 *          steps = ceil(dT/dt - 1e-9) ETDRK4 steps of size dT/steps
 *   M      quadrature points of the time average (Eq. 2.2, Algorithm 1), >= 2
 * Computes every table on the device (synchronously) before returning.
 * Returns ARP_EINVAL for invalid sizes, ARP_ENOMEM / ARP_ECUDA on failure;
 * *out is NULL unless ARP_OK.
 */
arp_status arp_create(arp_ctx** out, int N, double eps, double nu, int slices,
                      double dT, double dt, int M);

/* arp_set_option: set an arp_option (tables are rebuilt on the next call that
 * needs them).  ARP_EINVAL for an unknown key or an out-of-range value. */
arp_status arp_set_option(arp_ctx* ctx, int key, double value);

/* arp_query_bytes: device bytes a context with these sizes allocates (for
 * admission control); 0 for invalid sizes. */
size_t arp_query_bytes(int N, int slices, int M, int precision);

/*
 * arp_fine_batch: the fine propagator phi_dT (Sec. 3) applied to `batch`
 * independent states, U_out[b] = F(U_in[b]): `steps` ETDRK4 steps (Cox &
 * Matthews; the fine integrator named in Sec. 6.2) with the stiff linear part
 * exp(h(-L/eps + D)) applied exactly per wavenumber through L's
 * eigen-decomposition (Sec. 6.1) and N(u) formed pseudo-spectrally.
 * U_in, U_out: device, [batch][3][H] complex doubles; may not overlap.
 * batch = 0 is a no-op.  ARP_EINVAL for batch < 0 or NULL buffers.
 */
arp_status arp_fine_batch(arp_ctx* ctx, const double* U_in, double* U_out, int batch,
                          void* stream);

/*
 * arp_coarse_avg: the discretised average of the nonlinearity (Eq. 2.1-2.2,
 * Algorithm 1) for `batch` states:
 *   Nbar(u) = sum_{m=0}^{M-1} w_m e^{s_m L} N(e^{-s_m L} u),
 *   s_m = T0 m / M (fast time), w_m = rho(m/M)/M, rho(s) = C e^{-1/(s(1-s))}
 *   on (0,1) with int_0^1 rho = 1 (Sec. 2).
 * U_in, Nbar_out: device, [batch][3][H] complex doubles; may not overlap.
 * The sum over m is reduced on chip in a fixed order (results do not depend
 * on batch).  batch = 0 is a no-op.
 */
arp_status arp_coarse_avg(arp_ctx* ctx, const double* U_in, double* Nbar_out, int batch,
                          void* stream);

/*
 * arp_coarse_step: the asymptotic slow solver over dT (Algorithm 2) for
 * `batch` states:  w = e^{dT/2 D} u; k1 = Nbar(w); k2 = Nbar(w + dT/2 k1);
 * w = e^{dT/2 D}(w + dT k2); G(u) = e^{-(dT/eps) L} w  (the map back to fast
 * time of Sec. 3; the printed e^{+(dT/eps) L} is read as this).
 * Layout as arp_fine_batch.
 */
arp_status arp_coarse_step(arp_ctx* ctx, const double* U_in, double* U_out, int batch,
                           void* stream);

/* arp_set_initial: u0 for the parareal iteration, one state [3][H].  u0 may be
 * a host or a device pointer.  Resets the iteration (the next
 * arp_parareal_iterate is the coarse predictor). */
arp_status arp_set_initial(arp_ctx* ctx, const double* u0, void* stream);

/*
 * arp_parareal_iterate: one parareal iteration (Eq. 3.1, Algorithm 4).
 * The first call after arp_set_initial is the coarse predictor
 * U_n^0 = G(U_{n-1}^0), n = 1..S, and reports *max_rel_change = +inf.
 * Each later call k >= 1 computes, in this order: F(U_n^{k-1}) for all
 * n < S in parallel; V_n = F(U_n^{k-1}) - G(U_n^{k-1}) (FP64);
 * the serial chain U_{n+1}^k = G(U_n^k) + V_n with U_0^k = u0; and
 * *max_rel_change = max_n ||U_n^k - U_n^{k-1}|| / ||U_n^k|| (L2 over the
 * three fields via Parseval).  Synchronises `stream` to read the norm back.
 * *k_done receives the iteration level just completed.
 * ARP_EINVAL if no initial state was set; ARP_ENONFINITE if the change is
 * NaN or Inf (the iterate is kept).
 */
arp_status arp_parareal_iterate(arp_ctx* ctx, void* stream, int* k_done,
                                double* max_rel_change);

/* arp_parareal_solve: arp_parareal_iterate until k = KMAX or the change is
 * <= TOL (options), starting from the current level.  With ARP_OPT_PIPELINE
 * (default on, where it applies) the levels overlap on the device: the fine
 * sweep of level k starts on a chunk of slices as soon as the chain of level
 * k has produced their start states, on SMs the chain does not use; the
 * result, level and change are the level-by-level solve's, bit for bit.  When
 * the tolerance stops the solve at level k, the fine sweep of level k started
 * speculatively still completes before the work that follows on `stream`.
 * Returns after the last level's change is read; the slices are ready in
 * `stream` order.  ARP_EINVAL if no initial state was set; ARP_ETIMEOUT if a
 * bounded wait of the chain gave up (the iterate is then undefined until the
 * next arp_set_initial). */
arp_status arp_parareal_solve(arp_ctx* ctx, void* stream, int* k_done, double* max_rel_change);

/* arp_get_slices: copy the current iterate U_0..U_S, [(S+1)][3][H] complex
 * doubles, to U (host or device pointer).  Synchronises `stream` when U is a
 * host pointer. */
arp_status arp_get_slices(arp_ctx* ctx, double* U, void* stream);

/* arp_destroy: release the context and everything it owns (NULL is allowed). */
arp_status arp_destroy(arp_ctx* ctx);

/* arp_last_error: message of the last failed call on ctx (or of the last failed
 * arp_create when ctx is NULL); never NULL; valid until the next call. */
const char* arp_last_error(const arp_ctx* ctx);

/*
 * arp_coarse_avg_static: the time average of arp_coarse_avg (FP64, F = 1,
 * T0 = dT/eps) for callers that cannot allocate device memory -- a framework
 * that owns a fixed device-memory budget and forbids allocation after start-up,
 * or a latency-critical loop where cudaMalloc's implicit synchronisation is not
 * acceptable.  It needs no context (arp_create allocates) and allocates
 * nothing: its tables and workspaces live in one 16 MiB file-scope device array
 * that every GPU loading the library holds until the process exits.  The paper
 * has no counterpart to this entry point.
 *   N, eps, dT, M   as for arp_create (the window is T0 = dT/eps)
 *   U_in, Nbar_out  device, [batch][3][H] complex doubles, caller-owned
 * The batch is processed in passes of as many states as the array holds.
 * Returns ARP_EINVAL for invalid sizes and when the tables plus one state's
 * workspace exceed the 16 MiB array (e.g. N = 2048 with M = 256); no message
 * is recorded.  Every call shares the array and overwrites what it needs
 * before reading it (nothing has to start at zero); calls that overlap on the
 * GPU (on different streams, or from different threads) race on it.  The
 * first call on a device looks the array's device address up (once per
 * device); with lazy module loading (the CUDA default) that lookup is also
 * what places the 16 MiB array on the device.  Make that first call at
 * start-up, before the caller's memory budget is fixed and before any stream
 * capture; it returns ARP_ENOMEM if the device has no room for the array.
 */
arp_status arp_coarse_avg_static(int N, double eps, double dT, int M, const double* U_in, double* Nbar_out,
                                 int batch, void* stream);

/*
 * Batches: one parareal iteration of many independent problems at once.
 * arp_batch_create groups `count` existing contexts (not owned; all on the
 * current device); with ctxs == NULL it creates an empty batch with room for
 * `count` members (see arp_batch_reset).  arp_batch_iterate advances every context that has an
 * initial state by one level, exactly as arp_parareal_iterate would (the
 * predictor for contexts at their first call), but runs the work of all
 * contexts of the same grid size and precision in fused launches: one fine
 * sweep over every (problem, slice), one correction, one launch of one
 * thread-block cluster per problem for the serial chains (a context whose
 * chain cannot run as a cluster gets its own chain launch), and one norm over
 * all slices.  The blocks run the same kernel bodies as the single-problem
 * path, so each problem's iterates do not depend on the other members.
 * levels[i] / changes[i] (arrays of `count`, may be NULL) receive context i's
 * level and relative change (+inf after its predictor, NaN if it has no
 * initial state).  Synchronises `stream`.  A context of a batch must not be
 * used by another call while arp_batch_iterate runs.  On ARP_ETIMEOUT or
 * ARP_ENONFINITE the other problems have still advanced; the failing
 * context's arp_last_error tells what happened.
 */
typedef struct arp_batch arp_batch;
arp_status arp_batch_create(arp_batch** out, arp_ctx* const* ctxs, int count);
arp_status arp_batch_iterate(arp_batch* batch, void* stream, int* levels, double* changes);
/* arp_batch_reset: replace the members (count <= the count given at creation;
 * 0 empties the batch) without reallocating; a serving loop calls it when
 * requests join or leave. */
arp_status arp_batch_reset(arp_batch* batch, arp_ctx* const* ctxs, int count);
arp_status arp_batch_destroy(arp_batch* batch);
const char* arp_batch_last_error(const arp_batch* batch);

/* arp_info: sizes of a context: out[0]=N, out[1]=H, out[2]=K, out[3]=slices,
 * out[4]=M, out[5]=fine steps per slice, out[6]=current level k (-1 before the
 * predictor), out[7]=precision, out[8]=the schedule the FP32 ETDRK4 fine sweep
 * runs with (1 to 4 as ARP_OPT_FINE_BLOCK; the tuned default resolved). */
arp_status arp_info(const arp_ctx* ctx, int* out9);

/* arp_alu_peak: the measured plain-ALU peak of the current device: fused
 * multiply-adds of `precision` (ARP_FP32 or ARP_FP64) in independent register
 * chains on every SM, timed with events on `stream` (which it synchronises);
 * *tflops counts 2 flops per FMA.  A measurement aid for roofline fractions.
 * ARP_EINVAL for another precision or a NULL pointer; ARP_ECUDA or ARP_ENOMEM
 * on a CUDA failure. */
arp_status arp_alu_peak(int precision, double* tflops, void* stream);

/* arp_pipeline_info: how the last arp_parareal_solve ran: out[0] = 1 if
 * pipelined (ARP_OPT_PIPELINE), else 0; out[1], out[2] = SMs of the chain and
 * fine partitions, out[3] = links per chunk, out[4] = CTAs of the chain's
 * cluster (0 where no partition was made); out[5] = 1 if a launch or call on
 * the partitions was refused once (for instance by a profiler without support
 * for them) while the CUDA context stayed usable: that solve was redone level
 * by level from u0, with the same result, and the context no longer pipelines.
 * ARP_EINVAL for NULL arguments. */
arp_status arp_pipeline_info(const arp_ctx* ctx, int* out6);

/* arp_gemm_check: the library's split-precision tensor-core GEMM (the
 * contraction behind the DFT-as-GEMM precisions) on caller data, so it can be
 * tested on its own: C[j][i] = sum_k A[i][k] B[j][k] for A (m x k), B (n x k)
 * and C (n x m), all row-major FP32 device buffers owned by the caller;
 * `precision` is ARP_TF32X3, ARP_BF16X2 or ARP_BF16X3 (how A and B are split
 * into the MMA's input type).  Temporary operand buffers are allocated and
 * freed inside the call, which synchronises `stream`.  The paper has no
 * counterpart.  ARP_EINVAL for another precision, non-positive or too large
 * sizes (m, k <= 65536) or NULL pointers; ARP_ENOMEM, ARP_ECUDA, or
 * ARP_ETIMEOUT if a bounded wait of the kernel gave up. */
arp_status arp_gemm_check(int precision, int m, int n, int k, const float* A, const float* B, float* C, void* stream);

/* arp_chain_exchange_bytes: a host-side check of the cluster chain's byte
 * counts (no GPU work, no context).  For a grid of N points, a cluster of
 * `cluster` CTAs (1..16) and CTA `rank`, the bytes that CTA's two mbarriers
 * expect per time average, as the chain kernel arms them: *red_bytes for the
 * partial sums of its own (branch, wavenumber) pairs from every rank,
 * *ws_bytes for the whole state pushed by the owners, in complex values of
 * `precision` (ARP_FP64: 16 bytes, ARP_FP32: 8).  The paper has no
 * counterpart; it exists so the counts can be compared with the bytes the
 * exchanges send.  ARP_EINVAL for sizes outside those ranges or NULL pointers. */
arp_status arp_chain_exchange_bytes(int N, int cluster, int rank, int precision, unsigned* red_bytes,
                                    unsigned* ws_bytes);

#ifdef __cplusplus
}
#endif

#endif /* ARP_H */
