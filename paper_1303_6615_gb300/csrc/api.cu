// api.cu -- the C ABI (include/arp.h): argument checks, context memory, and
// dispatch to the kernels.  No exception crosses this boundary.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "context.h"

namespace arp {

arp_status fail(arp_ctx* c, arp_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

arp_status check_cuda(arp_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ARP_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? ARP_ENOMEM : ARP_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

arp_status ensure_tables(arp_ctx* c, cudaStream_t s) {
  if (!c->tables_dirty) return ARP_OK;
  return build_tables(c, s);
}

// The sub-context of ARP_OPT_COARSE_GRID: the same problem on N_c points (its
// tables and chain buffers; its own slices' states are not used), kept in step
// with the options that shape the coarse chain (window, F, precision).
arp_status ensure_coarse(arp_ctx* c, cudaStream_t s) {
  if (c->coarse_grid == 0) return ARP_OK;
  if (!c->coarse) {
    arp_ctx* q = nullptr;
    const arp_status r = arp_create(&q, c->coarse_grid, c->eps, c->nu, c->slices, c->dT, c->dt, c->M);
    if (r != ARP_OK) return fail(c, r, std::string("coarse grid: ") + arp_last_error(nullptr));
    c->coarse = q;
  }
  arp_ctx* q = c->coarse;
  if (q->T0_set != c->T0_set || q->T0 != c->T0 || q->F != c->F) {
    q->T0 = c->T0;
    q->T0_set = c->T0_set;
    q->F = c->F;
    q->tables_dirty = true;
  }
  q->precision = c->precision;
  const arp_status r = ensure_tables(q, s);
  return r == ARP_OK ? ARP_OK : fail(c, r, std::string("coarse grid: ") + q->err);
}

namespace {

thread_local std::string g_create_error;

bool pow2_in_range(int n) { return n >= 8 && n <= 2048 && (n & (n - 1)) == 0; }

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

struct Sizes {
  size_t tables, work, state;
};

// States per pass of the batched time average: all slices, but at most what a
// 32 MiB partial-sum workspace holds (at least one); the parareal path does
// not use this workspace.
int coarse_chunk(int slices, size_t P, size_t K1) {
  const size_t per = P * 3 * K1 * 16;
  size_t c = ((size_t)32 << 20) / per;
  if (c < 1) c = 1;
  return (int)(c < (size_t)slices ? c : (size_t)slices);
}

Sizes sizes_of(int N, int slices, int M) {
  const size_t H = N / 2 + 1, K1 = (N - 1) / 3 + 1, S = slices;
  const size_t qc = (M + kMaxNodeBlocks - 1) / kMaxNodeBlocks;
  const size_t P = (M + qc - 1) / qc;
  const size_t CC = coarse_chunk(slices, P, K1);
  Sizes z;
  z.tables = K1 * (8 + 8 + 4 + 4) + 18 * K1 * (16 + 8) + 3 * K1 * 8 + (size_t)N * (16 + 8 + 8) + (size_t)M * 3 * K1 * (16 + 8) +
             (size_t)M * 12 + K1 * 8 + 3 * K1 * 16 + 3 * K1 * 16 + 7 * K1 * 12;
  z.work = 2 * CC * 3 * K1 * 16 + (CC + 1) * P * 3 * K1 * 16 + (S + 1) * 8 + 16 + 16;
  z.state = 2 * (S + 1) * 3 * H * 16 + 3 * S * 3 * H * 16 + 2 * S * 3 * K1 * 16;
  return z;
}

template <typename P>
arp_status alloc(arp_ctx* c, P** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? ARP_ENOMEM : ARP_ECUDA,
                std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                    cudaGetErrorString(e));
  }
  return ARP_OK;
}

void release(arp_ctx* c) {
  pipeline_release(c);
  dft_release(c);
  void* ptrs[] = {c->E_lo32, c->inv_sig64, c->sk_sig64, c->inv_sig32, c->sk_sig32, c->etd64,   c->etd32, c->tw64,
                  c->tw32,      c->phase64,  c->phase32,   c->weight64,  c->weight32, c->dhalf, c->gphase,
                  c->W,         c->W2,       c->partial,   c->rel,       c->scalar,   c->U,     c->Uold,
                  c->Gc,        c->Fb,       c->V,         c->sync,     c->part2,    c->VT,    c->Ge,
                  c->strang_h64, c->etd32c,  c->tw16_32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

arp_status allocate(arp_ctx* c) {
  const size_t K1 = c->K1, H = c->H, S = c->slices, M = c->M, P = c->P, N = c->N, CC = c->cchunk;
  arp_status r;
#define ARP_ALLOC(ptr, bytes) \
  if ((r = alloc(c, &(ptr), (bytes))) != ARP_OK) return r;
  ARP_ALLOC(c->inv_sig64, K1 * 8);
  ARP_ALLOC(c->sk_sig64, K1 * 8);
  ARP_ALLOC(c->inv_sig32, K1 * 4);
  ARP_ALLOC(c->sk_sig32, K1 * 4);
  ARP_ALLOC(c->etd64, 18 * K1 * 16);
  ARP_ALLOC(c->etd32, 18 * K1 * 8);
  ARP_ALLOC(c->E_lo32, 3 * K1 * 8);
  ARP_ALLOC(c->etd32c, 7 * K1 * 8 + 7 * K1 * 4);
  ARP_ALLOC(c->tw64, N * 16);
  ARP_ALLOC(c->tw32, N * 8);
  ARP_ALLOC(c->tw16_32, N * 8);
  ARP_ALLOC(c->phase64, M * 3 * K1 * 16);
  ARP_ALLOC(c->phase32, M * 3 * K1 * 8);
  ARP_ALLOC(c->weight64, M * 8);
  ARP_ALLOC(c->weight32, M * 4);
  ARP_ALLOC(c->dhalf, K1 * 8);
  ARP_ALLOC(c->gphase, 3 * K1 * 16);
  ARP_ALLOC(c->strang_h64, 3 * K1 * 16);
  ARP_ALLOC(c->W, CC * 3 * K1 * 16);
  ARP_ALLOC(c->W2, CC * 3 * K1 * 16);
  ARP_ALLOC(c->partial, CC * P * 3 * K1 * 16);
  ARP_ALLOC(c->rel, (S + 1) * 8);
  ARP_ALLOC(c->scalar, 16);
  ARP_ALLOC(c->sync, 16);
  ARP_ALLOC(c->part2, P * 3 * K1 * 16);
  ARP_ALLOC(c->U, (S + 1) * 3 * H * 16);
  ARP_ALLOC(c->Uold, (S + 1) * 3 * H * 16);
  ARP_ALLOC(c->Gc, S * 3 * H * 16);
  ARP_ALLOC(c->Fb, S * 3 * H * 16);
  ARP_ALLOC(c->V, S * 3 * H * 16);
  ARP_ALLOC(c->VT, S * 3 * K1 * 16);
  ARP_ALLOC(c->Ge, S * 3 * K1 * 16);
#undef ARP_ALLOC
  cudaError_t e = cudaMemset(c->U, 0, (S + 1) * 3 * H * 16);
  if (e == cudaSuccess) e = cudaMemset(c->Uold, 0, (S + 1) * 3 * H * 16);
  if (e == cudaSuccess) e = cudaMemset(c->Gc, 0, S * 3 * H * 16);
  return check_cuda(c, e, "state initialisation");
}

bool is_host_pointer(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// Projects one state onto the state space in place: bins above K zero, k = 0 real.
__global__ void project_kernel(cd* u, int H, int K1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * H) return;
  const int k = i % H;
  if (k >= K1) u[i] = {0.0, 0.0};
  else if (k == 0) u[i].y = 0.0;
}

}  // namespace
}  // namespace arp

using namespace arp;

extern "C" {

size_t arp_query_bytes(int N, int slices, int M, int precision) {
  if (!pow2_in_range(N) || slices < 1 || M < 2 || precision < ARP_FP64 || precision > ARP_BF16X3) return 0;
  Sizes z = sizes_of(N, slices, M);
  return z.tables + z.work + z.state;
}

arp_status arp_create(arp_ctx** out, int N, double eps, double nu, int slices, double dT, double dt, int M) {
  if (!out) return ARP_EINVAL;
  *out = nullptr;
  auto bad = [](const char* m) {
    g_create_error = m;
    return ARP_EINVAL;
  };
  if (!pow2_in_range(N)) return bad("N must be a power of two in [8, 2048]");
  if (!(eps > 0.0)) return bad("eps must be > 0 (+inf switches the fast term off)");
  if (!(nu >= 0.0) || std::isinf(nu)) return bad("nu must be finite and >= 0");
  if (slices < 1 || slices > (1 << 20)) return bad("slices must lie in [1, 2^20]");
  if (!(dT > 0.0) || std::isinf(dT)) return bad("dT must be finite and > 0");
  if (!(dt > 0.0) || dt > dT * (1.0 + 1e-12)) return bad("dt must satisfy 0 < dt <= dT");
  if (M < 2 || M > (1 << 16)) return bad("M must lie in [2, 65536]");
  const double ratio = std::ceil(dT / dt - 1e-9);
  if (ratio > 1e8) return bad("dT/dt too large");
  arp_ctx* c = new (std::nothrow) arp_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return ARP_ENOMEM;
  }
  c->N = N;
  c->logN = log2i(N);
  c->H = N / 2 + 1;
  c->K = (N - 1) / 3;
  c->K1 = c->K + 1;
  c->slices = slices;
  c->M = M;
  c->qc = (M + kMaxNodeBlocks - 1) / kMaxNodeBlocks;
  c->P = (M + c->qc - 1) / c->qc;
  c->cchunk = coarse_chunk(slices, c->P, c->K1);
  c->eps = eps;
  c->nu = nu;
  c->dT = dT;
  c->dt = dt;
  c->steps = ratio < 1.0 ? 1 : (int)ratio;
  c->h = dT / c->steps;
  arp_status r = check_cuda(c, cudaGetDevice(&c->device), "current device");
  if (r == ARP_OK)
    r = check_cuda(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device), "SM count");
  if (r == ARP_OK) r = allocate(c);
  if (r == ARP_OK) {
    cudaStream_t s;
    r = check_cuda(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    if (r == ARP_OK) {
      r = build_tables(c, s);
      if (r == ARP_OK) r = check_cuda(c, cudaStreamSynchronize(s), "table build");
      cudaStreamDestroy(s);
    }
  }
  if (r != ARP_OK) {
    g_create_error = c->err;
    release(c);
    delete c;
    return r;
  }
  *out = c;
  return ARP_OK;
}

arp_status arp_set_option(arp_ctx* c, int key, double v) {
  if (!c) return ARP_EINVAL;
  switch (key) {
    case ARP_OPT_T0:
      if (!(v > 0.0) || std::isinf(v)) return fail(c, ARP_EINVAL, "T0 must be finite and > 0");
      c->T0 = v;
      c->T0_set = true;
      c->tables_dirty = true;
      return ARP_OK;
    case ARP_OPT_F:
      if (!(v > 0.0) || std::isinf(v)) return fail(c, ARP_EINVAL, "F must be finite and > 0");
      c->F = v;
      c->tables_dirty = true;
      return ARP_OK;
    case ARP_OPT_PRECISION:
      if (v != (double)ARP_FP64 && v != (double)ARP_FP32 && v != (double)ARP_TF32X3 && v != (double)ARP_BF16X2 &&
          v != (double)ARP_BF16X3)
        return fail(c, ARP_EINVAL, "unknown precision");
      c->precision = (int)v;
      return ARP_OK;
    case ARP_OPT_KMAX:
      if (!(v >= 0.0) || v > 1e6 || v != std::floor(v)) return fail(c, ARP_EINVAL, "KMAX must be an integer >= 0");
      c->kmax = (int)v;
      return ARP_OK;
    case ARP_OPT_TOL:
      if (!(v >= 0.0)) return fail(c, ARP_EINVAL, "TOL must be >= 0");
      c->tol = v;
      return ARP_OK;
    case ARP_OPT_CHAIN:
      if (v != 0.0 && v != 1.0 && v != 2.0 && v != 3.0) return fail(c, ARP_EINVAL, "CHAIN must be 0, 1, 2 or 3");
      c->chain_mode = (int)v;
      return ARP_OK;
    case ARP_OPT_FINE_SCHEME:
      if (v != 0.0 && v != 1.0 && v != 2.0)
        return fail(c, ARP_EINVAL, "FINE_SCHEME must be 0 (ETDRK4), 1 (Strang) or 2 (integrating-factor RK4)");
      c->fine_scheme = (int)v;
      return ARP_OK;
    case ARP_OPT_COARSE_SCHEME:
      if (v != 0.0 && v != 1.0) return fail(c, ARP_EINVAL, "COARSE_SCHEME must be 0 (asymptotic) or 1 (Strang)");
      c->coarse_scheme = (int)v;
      return ARP_OK;
    case ARP_OPT_COARSE_GRID: {
      const int n = (int)v;
      if ((double)n != v || (n != 0 && (n < 8 || n > c->N || (n & (n - 1)) != 0)))
        return fail(c, ARP_EINVAL, "COARSE_GRID must be 0 or a power of two in [8, N]");
      c->coarse_grid = (n == c->N) ? 0 : n;
      if (c->coarse && c->coarse->N != c->coarse_grid) {
        arp_destroy(c->coarse);
        c->coarse = nullptr;
      }
      return ARP_OK;
    }
    case ARP_OPT_PIPELINE:
      if (!(v >= 0.0) || v > 1e9 || v != std::floor(v))
        return fail(c, ARP_EINVAL, "PIPELINE must be 0, 1 or a chunk length >= 2");
      c->pipeline = (int)v;
      return ARP_OK;
    case ARP_OPT_FINE_BLOCK:
      if (v != 0.0 && v != 1.0 && v != 2.0 && v != 3.0 && v != 4.0)
        return fail(c, ARP_EINVAL, "FINE_BLOCK must be 0, 1, 2, 3 or 4");
      c->fine_block = (int)v;
      return ARP_OK;
    case ARP_OPT_TEST_SKIP_ARRIVAL:
      c->skip_arrival = v == 2.0 ? 2 : (v != 0.0);
      return ARP_OK;
    default:
      return fail(c, ARP_EINVAL, "unknown option key");
  }
}

arp_status arp_fine_batch(arp_ctx* c, const double* in, double* out, int batch, void* stream) {
  if (!c) return ARP_EINVAL;
  if (batch < 0) return fail(c, ARP_EINVAL, "batch must be >= 0");
  if (batch == 0) return ARP_OK;
  if (!in || !out) return fail(c, ARP_EINVAL, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  arp_status r = ensure_tables(c, s);
  if (r != ARP_OK) return r;
  return launch_fine(c, (const cd*)in, (cd*)out, batch, s);
}

arp_status arp_coarse_avg(arp_ctx* c, const double* in, double* out, int batch, void* stream) {
  if (!c) return ARP_EINVAL;
  if (batch < 0) return fail(c, ARP_EINVAL, "batch must be >= 0");
  if (batch == 0) return ARP_OK;
  if (!in || !out) return fail(c, ARP_EINVAL, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  arp_status r = ensure_tables(c, s);
  if (r != ARP_OK) return r;
  return coarse_avg(c, (const cd*)in, (cd*)out, batch, s);
}

arp_status arp_coarse_step(arp_ctx* c, const double* in, double* out, int batch, void* stream) {
  if (!c) return ARP_EINVAL;
  if (batch < 0) return fail(c, ARP_EINVAL, "batch must be >= 0");
  if (batch == 0) return ARP_OK;
  if (!in || !out) return fail(c, ARP_EINVAL, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  arp_status r = ensure_tables(c, s);
  if (r != ARP_OK) return r;
  return coarse_step(c, (const cd*)in, (cd*)out, batch, s);
}

arp_status arp_set_initial(arp_ctx* c, const double* u0, void* stream) {
  if (!c) return ARP_EINVAL;
  if (!u0) return fail(c, ARP_EINVAL, "NULL initial state");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)3 * c->H * sizeof(cd);
  arp_status r = check_cuda(c, cudaMemcpyAsync(c->U, u0, bytes, cudaMemcpyDefault, s), "initial state copy");
  if (r != ARP_OK) return r;
  project_kernel<<<(3 * c->H + 127) / 128, 128, 0, s>>>(c->U, c->H, c->K1);
  r = check_cuda(c, cudaGetLastError(), "initial state projection");
  if (r != ARP_OK) return r;
  if (is_host_pointer(u0)) {
    r = check_cuda(c, cudaStreamSynchronize(s), "initial state synchronise");
    if (r != ARP_OK) return r;
  }
  c->level = -1;
  c->have_initial = true;
  return ARP_OK;
}

arp_status arp_parareal_iterate(arp_ctx* c, void* stream, int* k_done, double* change) {
  if (!c) return ARP_EINVAL;
  if (!c->have_initial) return fail(c, ARP_EINVAL, "no initial state: call arp_set_initial first");
  cudaStream_t s = (cudaStream_t)stream;
  arp_status r = ensure_tables(c, s);
  if (r != ARP_OK) return r;
  return parareal_iterate(c, s, k_done, change);
}

arp_status arp_parareal_solve(arp_ctx* c, void* stream, int* k_done, double* change) {
  if (!c) return ARP_EINVAL;
  if (!c->have_initial) return fail(c, ARP_EINVAL, "no initial state: call arp_set_initial first");
  cudaStream_t s = (cudaStream_t)stream;
  arp_status r = ensure_tables(c, s);
  if (r != ARP_OK) return r;
  c->last_pipelined = 0;
  if (pipeline_eligible(c) && c->level < c->kmax) {
    bool ran = false;
    r = parareal_solve_pipelined(c, s, &ran, k_done, change);
    if (!ran && r != ARP_OK) {
      // the partition or its streams could not be made: nothing was enqueued,
      // and the pipeline stays off for this context (arp_pipeline_info)
      cudaGetLastError();
      c->err.clear();
      r = ARP_OK;
    } else if (ran && r == ARP_ECUDA && pipeline_recover(c)) {
      // a refused call on the partitions: the level being built may be partial,
      // so solve again from u0 (slice 0 of the iterate, never overwritten) level
      // by level; the iterates are deterministic functions of u0, so the result
      // is the one the pipelined solve would have returned
      c->level = -1;
      r = ARP_OK;
    } else if (ran || r != ARP_OK) {
      return r;
    }
  }
  int k = c->level;
  double ch = INFINITY;
  while (r == ARP_OK && k < c->kmax && !(k >= 1 && ch <= c->tol)) r = arp_parareal_iterate(c, stream, &k, &ch);
  if (k_done) *k_done = k;
  if (change) *change = ch;
  return r;
}

arp_status arp_get_slices(arp_ctx* c, double* U, void* stream) {
  if (!c) return ARP_EINVAL;
  if (!U) return fail(c, ARP_EINVAL, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)(c->slices + 1) * 3 * c->H * sizeof(cd);
  arp_status r = check_cuda(c, cudaMemcpyAsync(U, c->U, bytes, cudaMemcpyDefault, s), "slices copy");
  if (r != ARP_OK) return r;
  if (is_host_pointer(U)) return check_cuda(c, cudaStreamSynchronize(s), "slices synchronise");
  return ARP_OK;
}

arp_status arp_destroy(arp_ctx* c) {
  if (!c) return ARP_OK;
  if (c->coarse) arp_destroy(c->coarse);
  release(c);
  delete c;
  return ARP_OK;
}

arp_status arp_pipeline_info(const arp_ctx* c, int* out6) {
  if (!c || !out6) return ARP_EINVAL;
  return pipeline_info(c, out6);
}

const char* arp_last_error(const arp_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

arp_status arp_info(const arp_ctx* c, int* o) {  // o: 9 values
  if (!c || !o) return ARP_EINVAL;
  o[0] = c->N;
  o[1] = c->H;
  o[2] = c->K;
  o[3] = c->slices;
  o[4] = c->M;
  o[5] = c->steps;
  o[6] = c->level;
  o[7] = c->precision;
  o[8] = fine_schedule_in_effect(c);
  return ARP_OK;
}

}  // extern "C"
