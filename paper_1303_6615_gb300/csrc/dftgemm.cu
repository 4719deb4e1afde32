// dftgemm.cu -- the real DFTs of the nonlinearity as dense GEMMs on the tensor
// cores (precisions ARP_TF32X3 and ARP_BF16X2): the evaluation of N for a batch
// of states, used by the batched time average (one column group per
// (state, quadrature node)) and by a fine sweep that steps all slices in lock
// step (one column group per slice and ETDRK4 stage).
//
// Each field f is a column of real coefficients c = (Re f_0, Re f_1..K, Im f_1..K)
// (R = 2K + 1 rows), and with x_j = 2 pi j / N
//     f(x_j) = sum_r Winv[j][r] c_r,  Winv = [1, 2 cos(k x_j), -2 sin(k x_j)]       (N x R)
//     c_r(p) = sum_j Wfwd[r][j] p(x_j), Wfwd = [cos(k x_j); -sin(k x_j)] / N          (R x N)
// so the four inverse real transforms of a state (v1, h, v1_x, v2_x) are four
// columns of X = Winv A and the three forward ones (the products) three columns
// of Q = Wfwd P.  Both products are split-precision: every operand is split into
// a high and a low part of the input type (TF32-rounded FP32, or BF16) and
//     Winv A ~ Winv_hi A_hi + Winv_hi A_lo + Winv_lo A_hi,
// accumulated in FP32 by cuBLAS (plain library GEMMs; all other steps run in the
// kernels below).  The coefficient dimension is padded to Rp, a multiple of 8,
// with zero rows and columns, so every operand column starts on a 16-byte
// boundary (with R = 2K + 1 odd, the library would otherwise fall back to
// element-aligned kernels).  The dense DFT costs 2 N R flops per column against the FFT's
// ~2.5 N log2 N: this path exists for the precision study, not for speed.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <string>

#include "context.h"
#include "fine_impl.cuh"

namespace arp {

struct DftWork {
  cublasHandle_t blas = nullptr;
  int R = 0;               // padded coefficient rows: 2K + 1 rounded up to a multiple of 8
  size_t cols = 0;         // column capacity of A and X (4 per state-node or slice)
  void* Winv[2] = {nullptr, nullptr};
  void* Wfwd[2] = {nullptr, nullptr};
  void* A[2] = {nullptr, nullptr};
  float* X = nullptr;
  void* P[2] = {nullptr, nullptr};
  float* Q = nullptr;
  int tables_prec = -1;    // precision the DFT matrices were split for
  // fine sweep state, [slices][3][K1] each
  int fine_cap = 0;
  cf *U = nullptr, *ULO = nullptr, *NU = nullptr, *A1 = nullptr, *ACC = nullptr, *XS = nullptr;
};

namespace {

struct SplitTF32 {
  using E = float;
  static constexpr cudaDataType_t kType = CUDA_R_32F;
  static constexpr cublasComputeType_t kCompute = CUBLAS_COMPUTE_32F_FAST_TF32;
  __device__ static void split(float x, E& hi, E& lo) {
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    lo = x - hi;
  }
};

struct SplitBF16 {
  using E = __nv_bfloat16;
  static constexpr cudaDataType_t kType = CUDA_R_16BF;
  static constexpr cublasComputeType_t kCompute = CUBLAS_COMPUTE_32F;
  __device__ static void split(float x, E& hi, E& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  }
};

template <class S>
__global__ void dft_tables_kernel(int N, int K, int R, typename S::E* winv_hi, typename S::E* winv_lo,
                                  typename S::E* wfwd_hi, typename S::E* wfwd_lo) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * R) return;
  const int j = (int)(t % N), r = (int)(t / N);
  if (r > 2 * K) {  // padding
    S::split(0.0f, winv_hi[j + (size_t)N * r], winv_lo[j + (size_t)N * r]);
    S::split(0.0f, wfwd_hi[r + (size_t)R * j], wfwd_lo[r + (size_t)R * j]);
    return;
  }
  const int k = r <= K ? r : r - K;
  const long long m = ((long long)k * j) % N;  // exact argument reduction of k x_j
  double sn, cs;
  sincospi(2.0 * (double)m / (double)N, &sn, &cs);
  const double vinv = r == 0 ? 1.0 : (r <= K ? 2.0 * cs : -2.0 * sn);
  const double vfwd = (r == 0 ? 1.0 : (r <= K ? cs : -sn)) / (double)N;
  S::split((float)vinv, winv_hi[j + (size_t)N * r], winv_lo[j + (size_t)N * r]);
  S::split((float)vfwd, wfwd_hi[r + (size_t)R * j], wfwd_lo[r + (size_t)R * j]);
}

// The four field columns of one state from its eigen amplitudes x (FP32) at k.
template <class S>
__device__ __forceinline__ void pack_columns(const cf x[3], int k, int K, int R, float is, float ss, size_t g,
                                             typename S::E* Ahi, typename S::E* Alo) {
  cf u[3];
  eigen_to_phys<float>(x, is, ss, u);
  const float kk = (float)k;
  const cf F[4] = {u[0], u[2], kk * mul_i(u[0]), kk * mul_i(u[1])};  // v1, h, v1_x, v2_x
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const size_t col = (4 * g + f) * (size_t)R;
    S::split(F[f].x, Ahi[col + k], Alo[col + k]);
    if (k > 0) S::split(F[f].y, Ahi[col + K + k], Alo[col + K + k]);
  }
}

// Column groups (state s, node m): x = e^{-i omega s_m} W_s.
template <class S>
__global__ void dft_pack_avg_kernel(const cd* __restrict__ W, int nb, int M, int K, int R, const cf* __restrict__ ph,
                                    const float* __restrict__ is, const float* __restrict__ ss,
                                    typename S::E* Ahi, typename S::E* Alo) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nb * M * K1) return;
  const int k = (int)(t % K1);
  const size_t g = (size_t)(t / K1);
  const int s = (int)(g / M), m = (int)(g % M);
  cf x[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) x[b] = ph[((size_t)m * 3 + b) * K1 + k] * cvt<float>(W[((size_t)s * 3 + b) * K1 + k]);
  pack_columns<S>(x, k, K, R, is[k], ss[k], g, Ahi, Alo);
}

// Column groups (slice s): the fine sweep's stage inputs.
template <class S>
__global__ void dft_pack_fine_kernel(const cf* __restrict__ X, int S_, int K, int R, const float* __restrict__ is,
                                     const float* __restrict__ ss, typename S::E* Ahi, typename S::E* Alo) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S_ * K1) return;
  const int k = (int)(t % K1);
  const size_t g = (size_t)(t / K1);
  cf x[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) x[b] = X[(g * 3 + b) * K1 + k];
  pack_columns<S>(x, k, K, R, is[k], ss[k], g, Ahi, Alo);
}

// Products at the samples of each column group: -v1 v1_x, -v1 v2_x, -h v1.
template <class S>
__global__ void dft_products_kernel(const float* __restrict__ X, int N, long long groups, typename S::E* Phi,
                                    typename S::E* Plo) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= groups * N) return;
  const int j = (int)(t % N);
  const size_t g = (size_t)(t / N);
  const float v1 = X[j + (size_t)N * (4 * g)], h = X[j + (size_t)N * (4 * g + 1)];
  const float v1x = X[j + (size_t)N * (4 * g + 2)], v2x = X[j + (size_t)N * (4 * g + 3)];
  const float p[3] = {-v1 * v1x, -v1 * v2x, -h * v1};
#pragma unroll
  for (int f = 0; f < 3; ++f) S::split(p[f], Phi[j + (size_t)N * (3 * g + f)], Plo[j + (size_t)N * (3 * g + f)]);
}

// b = R^H (P1, P2, i k P3) of column group g at k from the forward coefficients.
__device__ __forceinline__ void unpack_columns(const float* __restrict__ Q, int k, int K, int R, float is, float ss,
                                               size_t g, cf b[3]) {
  cf P[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const size_t col = (3 * g + f) * (size_t)R;
    P[f] = mk<float>(Q[col + k], k > 0 ? Q[col + K + k] : 0.0f);
  }
  const cf n3[3] = {P[0], P[1], (float)k * mul_i(P[2])};
  phys_to_eigen<float>(n3, is, ss, b);
}

// Block (32 wavenumbers x 8 node chunks) per (state, k-range): each thread sums
// the weighted, back-rotated terms of its chunk of consecutive nodes in node
// order, then the chunk sums are added in chunk order (FP32) -- a fixed order --
// and written as the single chunk partial [nb][1][3][K1].
constexpr int kAvgChunks = 8;
__global__ void __launch_bounds__(32 * kAvgChunks) dft_unpack_avg_kernel(
    const float* __restrict__ Q, int nb, int M, int K, int R, const cf* __restrict__ ph, const float* __restrict__ w,
    const float* __restrict__ is, const float* __restrict__ ss, cd* __restrict__ partial) {
  __shared__ cf part[kAvgChunks][3][32];
  const int K1 = K + 1;
  const int k = blockIdx.x * 32 + threadIdx.x, s = blockIdx.y, y = threadIdx.y;
  const int per = (M + kAvgChunks - 1) / kAvgChunks;
  const int m0 = min(M, y * per), m1 = min(M, m0 + per);
  cf acc[3] = {mk<float>(0, 0), mk<float>(0, 0), mk<float>(0, 0)};
  if (k < K1) {
    for (int m = m0; m < m1; ++m) {
      cf b[3];
      unpack_columns(Q, k, K, R, is[k], ss[k], (size_t)s * M + m, b);
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[q] = acc[q] + w[m] * (conj(ph[((size_t)m * 3 + q) * K1 + k]) * b[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) part[y][q][threadIdx.x] = acc[q];
  __syncthreads();
  if (y == 0 && k < K1) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      cf t = part[0][q][threadIdx.x];
      for (int c = 1; c < kAvgChunks; ++c) t = t + part[c][q][threadIdx.x];
      partial[((size_t)s * 3 + q) * K1 + k] = cvt<double>(t);
    }
  }
}

// Per (slice, k): unpack N of the stage and apply the ETDRK4 combination of
// that stage (the formulas of the FP32 fine sweep: float-pair state, FP32 sum
// of the stage terms), writing the next stage's input XS.
__global__ void dft_fine_stage_kernel(const float* __restrict__ Q, int S_, int K, int R, int stage,
                                      FineTabs<float> tb, cf* U, cf* ULO, cf* NU, cf* A1, cf* ACC,
                                      cf* XS) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S_ * K1) return;
  const int k = (int)(t % K1), s = (int)(t / K1);
  cf bn[3];
  unpack_columns(Q, k, K, R, tb.is[k], tb.ss[k], (size_t)s, bn);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const size_t o = ((size_t)s * 3 + q) * K1 + k;
    cf u = U[o], ulo = ULO[o], nu = NU[o], a1 = A1[o], acc = ACC[o];
    XS[o] = etd32_stage(stage, q * K1 + k, bn[q], u, ulo, nu, a1, acc, tb.etd, tb.E_lo);
    U[o] = u;
    ULO[o] = ulo;
    NU[o] = nu;
    A1[o] = a1;
    ACC[o] = acc;
  }
}

__global__ void dft_fine_load_kernel(const cd* __restrict__ in, int S_, int H, int K, FineTabs<float> tb, cf* U,
                                     cf* ULO, cf* XS) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S_ * K1) return;
  const int k = (int)(t % K1), s = (int)(t / K1);
  cd a[3];
  load_eigen64(in + (size_t)s * 3 * H, H, k, tb.is64[k], tb.ss64[k], a);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const size_t o = ((size_t)s * 3 + q) * K1 + k;
    const cf hi = cvt<float>(a[q]);
    U[o] = hi;
    ULO[o] = cvt<float>(a[q] - cvt<double>(hi));
    XS[o] = hi;
  }
}

__global__ void dft_fine_store_kernel(cd* __restrict__ out, int S_, int H, int K, FineTabs<float> tb,
                                      const cf* U, const cf* ULO) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S_ * H) return;
  const int k = (int)(t % H), s = (int)(t / H);
  cd* dst = out + (size_t)s * 3 * H;
  if (k >= K1) {
#pragma unroll
    for (int f = 0; f < 3; ++f) dst[f * H + k] = {0.0, 0.0};
    return;
  }
  cd a[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const size_t o = ((size_t)s * 3 + q) * K1 + k;
    a[q] = cvt<double>(U[o]) + cvt<double>(ULO[o]);
  }
  store_phys64(dst, H, k, tb.is64[k], tb.ss64[k], a);
}

unsigned blocks_for(long long n, int tb) { return (unsigned)((n + tb - 1) / tb); }

arp_status blas_check(arp_ctx* c, cublasStatus_t st, const char* what) {
  if (st == CUBLAS_STATUS_SUCCESS) return ARP_OK;
  return fail(c, st == CUBLAS_STATUS_ALLOC_FAILED ? ARP_ENOMEM : ARP_ECUDA,
              std::string(what) + ": cuBLAS status " + std::to_string((int)st));
}

// C (m x n, FP32) = A B with A (m x k) and B (k x n) given as hi/lo parts:
// A_hi B_hi + A_hi B_lo + A_lo B_hi, column-major.
template <class S>
arp_status gemm3(arp_ctx* c, cublasHandle_t h, int m, int n, int k, void* const A[2], int lda, void* const B[2],
                 int ldb, float* C, int ldc) {
  const float one = 1.0f, zero = 0.0f;
  const void* ops[3][2] = {{A[0], B[0]}, {A[0], B[1]}, {A[1], B[0]}};
  for (int i = 0; i < 3; ++i) {
    const cublasStatus_t st =
        cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, ops[i][0], S::kType, lda, ops[i][1], S::kType, ldb,
                     i == 0 ? &zero : &one, C, CUDA_R_32F, ldc, S::kCompute, CUBLAS_GEMM_DEFAULT);
    arp_status r = blas_check(c, st, "dft gemm");
    if (r != ARP_OK) return r;
  }
  return ARP_OK;
}

template <class S>
size_t elem_bytes() {
  return sizeof(typename S::E);
}

// The workspace for `cols` columns (4 per column group) and `fine` slices.
template <class S>
arp_status ensure_work(arp_ctx* c, size_t cols, int fine, cudaStream_t s) {
  DftWork*& d = c->dft;
  if (!d) {
    d = new (std::nothrow) DftWork();
    if (!d) return fail(c, ARP_ENOMEM, "dft: host allocation");
    if (cublasCreate(&d->blas) != CUBLAS_STATUS_SUCCESS) {
      d->blas = nullptr;
      return fail(c, ARP_ECUDA, "dft: cuBLAS handle");
    }
    d->R = (2 * c->K + 1 + 7) / 8 * 8;
  }
  const int N = c->N, R = d->R;
  const size_t eb = elem_bytes<S>();
  auto grow = [&](void*& p, size_t bytes) -> arp_status {
    if (p) cudaFree(p);
    p = nullptr;
    const cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(c, ARP_ENOMEM, "dft: workspace allocation");
    }
    return ARP_OK;
  };
  arp_status r;
  if (d->tables_prec != c->precision) {
    for (int i = 0; i < 2; ++i) {
      if ((r = grow(d->Winv[i], (size_t)N * R * eb)) != ARP_OK) return r;
      if ((r = grow(d->Wfwd[i], (size_t)N * R * eb)) != ARP_OK) return r;
    }
    using E = typename S::E;
    dft_tables_kernel<S><<<blocks_for((long long)N * R, 256), 256, 0, s>>>(
        N, c->K, R, (E*)d->Winv[0], (E*)d->Winv[1], (E*)d->Wfwd[0], (E*)d->Wfwd[1]);
    if ((r = check_cuda(c, cudaGetLastError(), "dft: tables")) != ARP_OK) return r;
    d->tables_prec = c->precision;
    d->cols = 0;  // the element type of the operands changed
  }
  if (cols > d->cols) {
    for (int i = 0; i < 2; ++i) {
      if ((r = grow(d->A[i], cols * R * eb)) != ARP_OK) return r;
      // the padding rows of A are never written: zero (a zero bit pattern in both types)
      if ((r = check_cuda(c, cudaMemsetAsync(d->A[i], 0, cols * R * eb, s), "dft: workspace")) != ARP_OK) return r;
      if ((r = grow(d->P[i], cols / 4 * 3 * N * eb)) != ARP_OK) return r;
    }
    void* x = d->X;
    if ((r = grow(x, cols * N * sizeof(float))) != ARP_OK) return r;
    d->X = (float*)x;
    void* q = d->Q;
    if ((r = grow(q, cols / 4 * 3 * R * sizeof(float))) != ARP_OK) return r;
    d->Q = (float*)q;
    d->cols = cols;
  }
  if (fine > d->fine_cap) {
    cf** arrs[6] = {&d->U, &d->ULO, &d->NU, &d->A1, &d->ACC, &d->XS};
    for (cf** a : arrs) {
      void* p = *a;
      if ((r = grow(p, (size_t)fine * 3 * c->K1 * sizeof(cf))) != ARP_OK) return r;
      *a = (cf*)p;
    }
    d->fine_cap = fine;
  }
  if (cublasSetStream(d->blas, s) != CUBLAS_STATUS_SUCCESS) return fail(c, ARP_ECUDA, "dft: cuBLAS stream");
  return ARP_OK;
}

// X = Winv A for `groups` column groups, then P = products, then Q = Wfwd P.
template <class S>
arp_status dft_transforms(arp_ctx* c, long long groups, cudaStream_t s) {
  DftWork* d = c->dft;
  const int N = c->N, R = d->R;
  arp_status r;
  if ((r = gemm3<S>(c, d->blas, N, (int)(4 * groups), R, d->Winv, N, d->A, R, d->X, N)) != ARP_OK) return r;
  using E = typename S::E;
  dft_products_kernel<S><<<blocks_for(groups * N, 256), 256, 0, s>>>(d->X, N, groups, (E*)d->P[0], (E*)d->P[1]);
  if ((r = check_cuda(c, cudaGetLastError(), "dft: products")) != ARP_OK) return r;
  return gemm3<S>(c, d->blas, R, (int)(3 * groups), N, d->Wfwd, R, d->P, N, d->Q, R);
}

template <class S>
arp_status dft_nbar_t(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  const int M = c->M, K1 = c->K1;
  // states per pass: at most 8192 (state, node) groups
  const int per = M >= 8192 ? 1 : 8192 / M;
  arp_status r = ensure_work<S>(c, (size_t)4 * (per < batch ? per : batch) * M, 0, s);
  if (r != ARP_OK) return r;
  using E = typename S::E;
  DftWork* d = c->dft;
  for (int s0 = 0; s0 < batch; s0 += per) {
    const int nb = batch - s0 < per ? batch - s0 : per;
    const long long groups = (long long)nb * M;
    dft_pack_avg_kernel<S><<<blocks_for(groups * K1, 128), 128, 0, s>>>(
        W + (size_t)s0 * 3 * K1, nb, M, c->K, d->R, c->phase32, c->inv_sig32, c->sk_sig32, (E*)d->A[0],
        (E*)d->A[1]);
    if ((r = check_cuda(c, cudaGetLastError(), "dft: pack")) != ARP_OK) return r;
    if ((r = dft_transforms<S>(c, groups, s)) != ARP_OK) return r;
    dft_unpack_avg_kernel<<<dim3((K1 + 31) / 32, nb), dim3(32, kAvgChunks), 0, s>>>(
        d->Q, nb, M, c->K, d->R, c->phase32, c->weight32, c->inv_sig32, c->sk_sig32, partial + (size_t)s0 * 3 * K1);
    if ((r = check_cuda(c, cudaGetLastError(), "dft: unpack")) != ARP_OK) return r;
  }
  return ARP_OK;
}

template <class S>
arp_status dft_fine_t(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  arp_status r = ensure_work<S>(c, (size_t)4 * batch, batch, s);
  if (r != ARP_OK) return r;
  using E = typename S::E;
  DftWork* d = c->dft;
  const FineTabs<float> tb = fine_tabs<float>(c);
  const long long n = (long long)batch * c->K1;
  dft_fine_load_kernel<<<blocks_for(n, 128), 128, 0, s>>>(in, batch, c->H, c->K, tb, d->U, d->ULO, d->XS);
  if ((r = check_cuda(c, cudaGetLastError(), "dft fine: load")) != ARP_OK) return r;
  for (int step = 0; step < c->steps; ++step) {
    for (int stage = 0; stage < 4; ++stage) {
      dft_pack_fine_kernel<S><<<blocks_for(n, 128), 128, 0, s>>>(d->XS, batch, c->K, d->R, c->inv_sig32,
                                                                  c->sk_sig32, (E*)d->A[0], (E*)d->A[1]);
      if ((r = check_cuda(c, cudaGetLastError(), "dft fine: pack")) != ARP_OK) return r;
      if ((r = dft_transforms<S>(c, batch, s)) != ARP_OK) return r;
      dft_fine_stage_kernel<<<blocks_for(n, 128), 128, 0, s>>>(d->Q, batch, c->K, d->R, stage, tb, d->U, d->ULO,
                                                                d->NU, d->A1, d->ACC, d->XS);
      if ((r = check_cuda(c, cudaGetLastError(), "dft fine: stage")) != ARP_OK) return r;
    }
  }
  dft_fine_store_kernel<<<blocks_for((long long)batch * c->H, 128), 128, 0, s>>>(out, batch, c->H, c->K, tb, d->U,
                                                                                  d->ULO);
  return check_cuda(c, cudaGetLastError(), "dft fine: store");
}

}  // namespace

bool dft_mode(const arp_ctx* c) { return c->precision == ARP_TF32X3 || c->precision == ARP_BF16X2; }

arp_status dft_nbar(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  return c->precision == ARP_BF16X2 ? dft_nbar_t<SplitBF16>(c, W, partial, batch, s)
                                    : dft_nbar_t<SplitTF32>(c, W, partial, batch, s);
}

arp_status dft_fine(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  return c->precision == ARP_BF16X2 ? dft_fine_t<SplitBF16>(c, in, out, batch, s)
                                    : dft_fine_t<SplitTF32>(c, in, out, batch, s);
}

void dft_release(arp_ctx* c) {
  DftWork* d = c->dft;
  if (!d) return;
  void* ptrs[] = {d->Winv[0], d->Winv[1], d->Wfwd[0], d->Wfwd[1], d->A[0], d->A[1], d->X, d->P[0], d->P[1], d->Q,
                  d->U, d->ULO, d->NU, d->A1, d->ACC, d->XS};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (d->blas) cublasDestroy(d->blas);
  delete d;
  c->dft = nullptr;
}

}  // namespace arp
