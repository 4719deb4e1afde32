// context.h -- host-side context of the asymptotic parareal library and the
// internal launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "arp.h"
#include "common.cuh"

namespace arp {
struct DftWork;  // dftgemm.cu: DFT matrices, GEMM operands, cuBLAS handle
struct Pipe;     // pipeline.cu: SM partition, streams and events of the pipelined solve
}

struct arp_ctx {
  // problem
  int N = 0, logN = 0, H = 0, K = 0, K1 = 0;
  int slices = 0, M = 0, steps = 0;
  int qc = 1, P = 0;             // nodes per block, node chunks P = ceil(M / qc)
  int cchunk = 1;                // states per pass of arp_coarse_avg / arp_coarse_step
  double eps = 0, nu = 0, dT = 0, dt = 0, h = 0;
  double T0 = 0, F = 1.0, tol = 0.0;
  bool T0_set = false;
  int kmax = 5;
  int precision = ARP_FP64;
  int device = 0;
  int num_sms = 0;               // SMs of the device (the fine sweep's schedule rule)
  bool tables_dirty = true;

  // FP64 tables (always), FP32 copies (rounded from FP64)
  double* inv_sig64 = nullptr;   // [K1]
  double* sk_sig64 = nullptr;    // [K1]
  float* inv_sig32 = nullptr;
  float* sk_sig32 = nullptr;
  arp::cd* etd64 = nullptr;      // [6][3][K1]: E, E2, Q, f1, f2x2, f3
  arp::cf* etd32 = nullptr;
  arp::cf* E_lo32 = nullptr;     // [3][K1]: E - (double)(float)E, rounded to float
  // compact FP32 ETDRK4 tables (E, E2, Q, f1, f2x2, f3, E_lo): [7][K1] complex of
  // the alpha = +1 branch, then [7][K1] float of the (real) alpha = 0 branch
  arp::cf* etd32c = nullptr;
  arp::cd* tw64 = nullptr;       // [N] (twiddle_count(logN) used): per-stage FFT twiddles
  arp::cf* tw32 = nullptr;
  arp::cf* tw16_32 = nullptr;    // [N] (twiddle16_count(logN) used, 512 <= N <= 2048): radix-16 twiddles
  arp::cd* phase64 = nullptr;    // [M][3][K1] e^{-i omega s_m}
  arp::cf* phase32 = nullptr;
  double* weight64 = nullptr;    // [M] w_m
  float* weight32 = nullptr;
  double* dhalf = nullptr;       // [K1] e^{-nu k^4 dT/2}
  arp::cd* gphase = nullptr;     // [3][K1] e^{-i omega dT/eps}
  arp::cd* strang_h64 = nullptr; // [3][K1] e^{lambda dT/2} (the Strang coarse step's half steps)

  // workspaces (sized for `cchunk` states)
  arp::cd* W = nullptr;          // [cchunk][3][K1] eigen, FP64
  arp::cd* W2 = nullptr;         // [cchunk][3][K1]
  arp::cd* partial = nullptr;    // [cchunk][P][3][K1]
  double* rel = nullptr;         // [slices + 1] per-slice relative change
  double* scalar = nullptr;      // [2]: max relative change
  unsigned* sync = nullptr;      // [4]: [0] grid-barrier counter, [1] status (0 ok, else an arp_status)
  arp::cd* part2 = nullptr;      // [P][3][K1] second partial buffer of the chain

  // parareal state, physical spectral FP64, [(slices+1)][3][H] each
  arp::cd* U = nullptr;          // current iterate
  arp::cd* Uold = nullptr;       // previous iterate
  arp::cd* Gc = nullptr;         // G(U_n) of the current iterate, n < slices
  arp::cd* Fb = nullptr;         // F(U_n), n < slices
  arp::cd* V = nullptr;          // F - G
  arp::cd* VT = nullptr;         // [slices][3][K1] e^{dT/2 D} R^H V_n (eigen basis)
  arp::cd* Ge = nullptr;         // [slices][3][K1] G(U_n) in the eigen basis (cluster chain)
  int skip_arrival = 0;          // one-shot failure-detection test hook
  int chain_mode = 0;            // ARP_OPT_CHAIN
  int fine_block = 0;            // ARP_OPT_FINE_BLOCK: 0 per-size default, 1 = N/4, 2 = N/2 threads
  int fine_scheme = 0;           // ARP_OPT_FINE_SCHEME: 0 ETDRK4, 1 Strang splitting, 2 integrating-factor RK4
  int coarse_scheme = 0;         // ARP_OPT_COARSE_SCHEME: 0 asymptotic (Algorithm 2), 1 Strang step of dT
  int coarse_grid = 0;           // ARP_OPT_COARSE_GRID: 0 = the fine grid, else N_c < N for the coarse chain
  arp_ctx* coarse = nullptr;     // owned sub-context on the N_c grid (its tables, chain buffers), made on first use
  arp::DftWork* dft = nullptr;   // ARP_TF32X3 / ARP_BF16X2 workspace, made on first use
  int pipeline = 1;              // ARP_OPT_PIPELINE: 0 off, 1 automatic chunks, n >= 2 links per chunk
  arp::Pipe* pipe = nullptr;     // made by the first pipelined solve
  int last_pipelined = 0;        // whether the last arp_parareal_solve ran pipelined
  int level = -1;                // -1: no initial state; 0: predictor pending
  bool have_initial = false;

  std::string err;
};

namespace arp {

// Stores a message and returns the status.
arp_status fail(arp_ctx* c, arp_status s, const std::string& msg);
arp_status check_cuda(arp_ctx* c, cudaError_t e, const char* what);

// tables.cu (build) and api.cu (rebuild when options changed them)
arp_status build_tables(arp_ctx* c, cudaStream_t s);
arp_status ensure_tables(arp_ctx* c, cudaStream_t s);

// fine.cu: F applied to `batch` physical states.
arp_status launch_fine(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);
// strang64.cu: `steps` Strang steps of size h per state (coarse: one step of
// size dT), and standard parareal's serial chain with the Strang coarse step.
arp_status launch_strang_sweep(arp_ctx* c, const cd* in, cd* out, int batch, bool coarse, cudaStream_t s);
arp_status launch_strang_chain(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s);

// coarse.cu
//   to_eigen: W[b] = (dhalf if use_dhalf) * R^H u[b]
arp_status launch_to_eigen(arp_ctx* c, const cd* u, cd* W, int batch, bool use_dhalf, cudaStream_t s);
//   nbar_partial: partial[b][p] = sum over chunk p of w_m e^{i w s_m} b(R e^{-i w s_m} W[b])
arp_status launch_nbar_partial(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s);
//   reduce epilogues (sum over chunks p in order, then):
enum ReduceMode { kReduceAvg = 0, kReduceMid = 1, kReduceFinal = 2 };
//   kReduceAvg:   out_phys[b] = R Nbar
//   kReduceMid:   W2[b] = W[b] + dT/2 Nbar
//   kReduceFinal: g = gphase * dhalf * (W[b] + dT Nbar); out_phys[b] = R g;
//                 if out2: out2_phys[b] = R g (+ vadd[b] when vadd is given)
arp_status launch_nbar_reduce(arp_ctx* c, int mode, const cd* partial, const cd* W, cd* W2,
                              cd* out_phys, const cd* vadd, cd* out2_phys, int batch, cudaStream_t s);
arp_status coarse_avg(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);
arp_status coarse_step(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);

// chain: the serial coarse chain U_{n+1} = G(U_n) (+ V_n), n = 0..S-1, one
// cooperative persistent launch; Gc_n = G(U_n).  Returns ARP_EINVAL (without
// launching) if the grid cannot be co-resident.
arp_status launch_chain(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s);
// The same chain inside one thread-block cluster (no grid barriers).  Returns
// ARP_EINVAL (without launching) if no suitable cluster can be scheduled.  With
// a range, only links n0 .. n0+nl-1 run: the carried eigen-basis state enters
// from Win (null: from U0) and is stored to Wout (if not null), so consecutive
// ranges give the whole chain's results bit for bit; check_only launches
// nothing and reports whether a cluster fits on the current context's SMs.
// cluster: 0 tries 16 then 8 CTAs, else only that size, already known to fit
// the current context's SMs (no occupancy query).
struct ChainRange {
  int n0 = 0, nl = 0;
  const cd* Win = nullptr;
  cd* Wout = nullptr;
  bool check_only = false;
  int cluster = 0;
};
arp_status launch_cluster_chain(arp_ctx* c, const cd* U0, cd* Ge, const cd* VT, cudaStream_t s,
                                const ChainRange* rg = nullptr);

// parareal.cu
// True where the automatic chain choice (ARP_OPT_CHAIN 0) takes the cooperative
// grid before the cluster: FP64 with more than 16 quadrature nodes, where the
// cluster's CTAs would each transform several nodes on the slow FP64 units
// while the grid gives every node a block of its own.  With at most 16 nodes a
// cluster CTA holds at most one node and the cluster's barriers are cheaper.
inline bool fp64_grid_first(const arp_ctx* c) {
  return c->chain_mode == 0 && c->precision == ARP_FP64 && c->M > 16;
}
arp_status parareal_iterate(arp_ctx* c, cudaStream_t s, int* k_done, double* change);
// The serial chain of one context (cluster, else cooperative grid, else launches).
arp_status run_chain(arp_ctx* c, const cd* V, cudaStream_t s);
// ARP_OK for a zero chain status word, else ARP_ETIMEOUT with a message.
arp_status chain_status(arp_ctx* c, unsigned status);
// api.cu: the coarse-grid sub-context, created or refreshed to match c's options.
arp_status ensure_coarse(arp_ctx* c, cudaStream_t s);
// pipeline.cu: arp_parareal_solve with the levels overlapped (the same results
// bit for bit); *ran false (nothing done) where the SM partition or the chain
// cluster is unavailable.
bool pipeline_eligible(const arp_ctx* c);
arp_status parareal_solve_pipelined(arp_ctx* c, cudaStream_t user, bool* ran, int* k_done, double* change);
arp_status pipeline_info(const arp_ctx* c, int* out);
// After a pipelined solve that ran and failed with ARP_ECUDA: true if the CUDA
// context is still usable (a launch or call on the SM partitions was refused,
// e.g. by a profiler that does not support them, rather than a fault); the
// pipeline is then disabled for c and the caller solves level by level.
bool pipeline_recover(arp_ctx* c);
// fine32.cu: the FP32 ETDRK4 fine sweep's schedule in effect for c (1, 2 or 3).
int fine_schedule_in_effect(const arp_ctx* c);
void pipeline_release(arp_ctx* c);
// dftgemm.cu: the DFT-as-GEMM precisions (ARP_TF32X3, ARP_BF16X2): the time
// average's node terms as one chunk partial [batch][1][3][K1], and the ETDRK4
// fine sweep with all states stepped together.
bool dft_mode(const arp_ctx* c);
arp_status dft_nbar(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s);
arp_status dft_fine(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);
void dft_release(arp_ctx* c);

}  // namespace arp
