// dftgemm.cu -- the real DFTs of the nonlinearity as dense GEMMs on the tensor
// cores (precisions ARP_TF32X3, ARP_BF16X2 and ARP_BF16X3): the evaluation of N
// for a batch of states, used by the batched time average (one column group per
// (state, quadrature node)) and by a fine sweep that steps all slices in lock
// step (one column group per slice and ETDRK4 stage).
//
// Each field f is a column of real coefficients c = (Re f_0, Re f_1..K, Im f_1..K)
// (R = 2K + 1 rows), and with x_j = 2 pi j / N
//     f(x_j) = sum_r Winv[j][r] c_r,  Winv = [1, 2 cos(k x_j), -2 sin(k x_j)]       (N x R)
//     c_r(p) = sum_j Wfwd[r][j] p(x_j), Wfwd = [cos(k x_j); -sin(k x_j)] / N          (R x N)
// so the four inverse real transforms of a state (v1, h, v1_x, v2_x) are four
// columns of X = Winv A and the three forward ones (the products) three columns
// of Q = Wfwd P.  Both are split-precision products: every operand is split
// into two or three parts of the input type (TF32-rounded FP32, or BF16) and
//     Winv A ~ sum over the precision's products of Winv_part A_part,
// accumulated in FP32 in tensor memory by the library's own tcgen05 kernel
// (tc_gemm.cuh): the inverse GEMM's epilogue forms the products -v1 v1_x,
// -v1 v2_x, -h v1 at every grid point from the accumulator and splits them
// into the forward GEMM's operand, so X never reaches memory.  Packing, node
// sums and the ETDRK4 combination run in the kernels below.  Both GEMMs keep
// their operands K-major: Winv as [N][Rp], the coefficient columns as
// [columns][Rp], Wfwd as [Rp][Nk], the products as [columns][Nk]; the
// coefficient dimension is padded with zeros to Rp, a multiple of 128 (the
// tile), and the grid dimension to Nk, a multiple of 64, so every TMA box lies
// on a 16-byte boundary.  The dense DFT costs 2 N R flops per column against
// the FFT's ~2.5 N log2 N: this path exists for the precision study and the
// tensor-core measurement, not as the default.
#include <cuda.h>

#include <string>

#include "context.h"
#include "fine_impl.cuh"
#include "tc_gemm.cuh"

namespace arp {

struct DftWork {
  int R = 0;               // padded coefficient rows: 2K + 1 rounded up to a multiple of 128
  int Mi = 0;              // padded rows of Winv: N rounded up to a multiple of 128
  int Nk = 0;              // padded grid dimension of Wfwd and P: N rounded up to a multiple of 64
  size_t cols = 0;         // column capacity of A (4 per column group)
  void* Winv = nullptr;    // [parts][Mi][R]
  void* Wfwd = nullptr;    // [parts][R][Nk]
  void* A = nullptr;       // [parts][cols][R]
  void* P = nullptr;       // [parts][3 cols / 4][Nk]
  float* Q = nullptr;      // [3 cols / 4][R]
  unsigned* status = nullptr;       // device: bit 0 set by a bounded wait that gave up
  unsigned* status_host = nullptr;  // pinned copy read after each call
  int tables_prec = -1;    // precision the DFT matrices were split for
  // fine sweep state, [slices][3][K1] each
  int fine_cap = 0;
  cf *U = nullptr, *ULO = nullptr, *NU = nullptr, *A1 = nullptr, *ACC = nullptr, *XS = nullptr;
};

namespace {

using tc::SplitBF16x2;
using tc::SplitBF16x3;
using tc::SplitTF32x3;

template <class S>
__global__ void dft_tables_kernel(int N, int K, int R, int Mi, int Nk, typename S::E* winv, typename S::E* wfwd) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ni = (long long)Mi * R, nf = (long long)R * Nk;
  if (t >= ni + nf) return;
  int j, r;
  typename S::E* dst;
  size_t stride;
  bool fwd = t >= ni;
  if (!fwd) {
    j = (int)(t / R);
    r = (int)(t % R);
    dst = winv + t;
    stride = (size_t)ni;
  } else {
    r = (int)((t - ni) / Nk);
    j = (int)((t - ni) % Nk);
    dst = wfwd + (t - ni);
    stride = (size_t)nf;
  }
  double v = 0.0;
  if (j < N && r <= 2 * K) {
    const int k = r <= K ? r : r - K;
    const long long m = ((long long)k * j) % N;  // exact argument reduction of k x_j
    double sn, cs;
    sincospi(2.0 * (double)m / (double)N, &sn, &cs);
    v = fwd ? (r == 0 ? 1.0 : (r <= K ? cs : -sn)) / (double)N : (r == 0 ? 1.0 : (r <= K ? 2.0 * cs : -2.0 * sn));
  }
  S::split_d(v, dst, stride);
}

// The four field columns of one state from its eigen amplitudes x (FP32) at k,
// split into the parts of A ([parts][cols][R], parts `ps` elements apart).
template <class S>
__device__ __forceinline__ void pack_columns(const cf x[3], int k, int K, int R, float is, float ss, size_t g,
                                             typename S::E* A, size_t ps) {
  cf u[3];
  eigen_to_phys<float>(x, is, ss, u);
  const float kk = (float)k;
  const cf F[4] = {u[0], u[2], kk * mul_i(u[0]), kk * mul_i(u[1])};  // v1, h, v1_x, v2_x
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const size_t col = (4 * g + f) * (size_t)R;
    S::split(F[f].x, A + col + k, ps);
    if (k > 0) S::split(F[f].y, A + col + K + k, ps);
  }
}

// Column groups (state s, node m): x = e^{-i omega s_m} W_s.
template <class S>
__global__ void dft_pack_avg_kernel(const cd* __restrict__ W, int nb, int M, int K, int R, const cf* __restrict__ ph,
                                    const float* __restrict__ is, const float* __restrict__ ss,
                                    typename S::E* A, size_t ps) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nb * M * K1) return;
  const int k = (int)(t % K1);
  const size_t g = (size_t)(t / K1);
  const int s = (int)(g / M), m = (int)(g % M);
  cf x[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) x[b] = ph[((size_t)m * 3 + b) * K1 + k] * cvt<float>(W[((size_t)s * 3 + b) * K1 + k]);
  pack_columns<S>(x, k, K, R, is[k], ss[k], g, A, ps);
}

// Column groups (slice s): the fine sweep's stage inputs.
template <class S>
__global__ void dft_pack_fine_kernel(const cf* __restrict__ X, int S_, int K, int R, const float* __restrict__ is,
                                     const float* __restrict__ ss, typename S::E* A, size_t ps) {
  const int K1 = K + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S_ * K1) return;
  const int k = (int)(t % K1);
  const size_t g = (size_t)(t / K1);
  cf x[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) x[b] = X[(g * 3 + b) * K1 + k];
  pack_columns<S>(x, k, K, R, is[k], ss[k], g, A, ps);
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

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// does not link the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of a K-major operand [parts][rows_alloc][kdim] of which the first
// `rows` rows are read, with 128 x (128-byte) boxes, 128-byte swizzle, zero
// fill beyond `rows`.
template <class S>
arp_status make_map(arp_ctx* c, CUtensorMap* map, void* base, int kdim, long long rows, long long rows_alloc) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(c, ARP_ECUDA, "dft: cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t es = sizeof(typename S::E);
  const cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)S::kParts};
  const cuuint64_t strides[2] = {(cuuint64_t)kdim * es, (cuuint64_t)kdim * es * (cuuint64_t)rows_alloc};
  const cuuint32_t box[3] = {(cuuint32_t)(tc::kRowBytes / es), (cuuint32_t)tc::kBM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, S::kMapType, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, ARP_ECUDA, "dft: tensor map (CUresult " + std::to_string((int)r) + ")");
  return ARP_OK;
}

// One split-precision GEMM on the tensor cores: tiles of 128 x 128 over
// (m_rows, ncols), blockIdx.x over row tiles so the CTAs that share a column
// tile of B run together.
template <class S, int EPI>
arp_status tc_gemm(arp_ctx* c, void* A, int m_rows, void* B, long long ncols, long long b_rows_alloc, int kdim,
                   const tc::Epilogue& ep, cudaStream_t s) {
  CUtensorMap ma, mb;
  arp_status r;
  if ((r = make_map<S>(c, &ma, A, kdim, m_rows, m_rows)) != ARP_OK) return r;
  if ((r = make_map<S>(c, &mb, B, kdim, ncols, b_rows_alloc)) != ARP_OK) return r;
  const void* kern = (const void*)tc::split_gemm_kernel<S, EPI>;
  const size_t smem = tc::smem_bytes<S>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "dft gemm: shared-memory attribute");
  const long long ntiles = (ncols + tc::kBN - 1) / tc::kBN;
  if (ntiles > 65535) return fail(c, ARP_EINVAL, "dft gemm: too many column tiles in one pass");
  const int kblocks = kdim / (tc::kRowBytes / (int)sizeof(typename S::E));
  tc::Epilogue epc = ep;
  void* args[] = {(void*)&ma, (void*)&mb, (void*)&kblocks, (void*)&epc};
  e = cudaLaunchKernel(kern, dim3(m_rows / tc::kBM, (unsigned)ntiles), dim3(tc::kThreads), args, smem, s);
  return check_cuda(c, e, "dft gemm: launch");
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
    d->R = (2 * c->K + 1 + 127) / 128 * 128;
    d->Mi = (c->N + 127) / 128 * 128;
    d->Nk = (c->N + 63) / 64 * 64;
    if (cudaMalloc(&d->status, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&d->status_host, sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, ARP_ENOMEM, "dft: status word");
    }
    if (cudaMemsetAsync(d->status, 0, sizeof(unsigned), s) != cudaSuccess)
      return check_cuda(c, cudaGetLastError(), "dft: status word");
  }
  const int R = d->R, Mi = d->Mi, Nk = d->Nk;
  const size_t eb = elem_bytes<S>(), parts = S::kParts;
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
    if ((r = grow(d->Winv, parts * Mi * R * eb)) != ARP_OK) return r;
    if ((r = grow(d->Wfwd, parts * R * Nk * eb)) != ARP_OK) return r;
    using E = typename S::E;
    dft_tables_kernel<S><<<blocks_for((long long)Mi * R + (long long)R * Nk, 256), 256, 0, s>>>(
        c->N, c->K, R, Mi, Nk, (E*)d->Winv, (E*)d->Wfwd);
    if ((r = check_cuda(c, cudaGetLastError(), "dft: tables")) != ARP_OK) return r;
    d->tables_prec = c->precision;
    d->cols = 0;  // the element type of the operands changed
  }
  if (cols > d->cols) {
    // padding rows of A and padding points of P are never written: zero (a zero
    // bit pattern in both input types)
    if ((r = grow(d->A, parts * cols * R * eb)) != ARP_OK) return r;
    if ((r = check_cuda(c, cudaMemsetAsync(d->A, 0, parts * cols * R * eb, s), "dft: workspace")) != ARP_OK) return r;
    if ((r = grow(d->P, parts * (cols / 4 * 3) * Nk * eb)) != ARP_OK) return r;
    if ((r = check_cuda(c, cudaMemsetAsync(d->P, 0, parts * (cols / 4 * 3) * Nk * eb, s), "dft: workspace")) !=
        ARP_OK)
      return r;
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
  return ARP_OK;
}

// The inverse GEMM X = Winv A for `groups` column groups with the products
// formed in its epilogue (P), then Q = Wfwd P.
template <class S>
arp_status dft_transforms(arp_ctx* c, long long groups, cudaStream_t s) {
  DftWork* d = c->dft;
  const int N = c->N, R = d->R;
  const long long cols = 4 * groups, cols3 = 3 * groups;
  tc::Epilogue ei{nullptr, d->P, cols, 0, d->Nk, (long long)(d->cols / 4 * 3) * d->Nk, N, d->status};
  arp_status r = tc_gemm<S, tc::kEpiProducts>(c, d->Winv, d->Mi, d->A, cols, (long long)d->cols, R, ei, s);
  if (r != ARP_OK) return r;
  tc::Epilogue ef{d->Q, nullptr, cols3, R, 0, 0, R, d->status};
  return tc_gemm<S, tc::kEpiStore>(c, d->Wfwd, R, d->P, cols3, (long long)(d->cols / 4 * 3), d->Nk, ef, s);
}

// After the last GEMM of a call: the bounded waits' status word, read back
// (the call's stream is synchronised) and cleared.
arp_status dft_status(arp_ctx* c, cudaStream_t s) {
  DftWork* d = c->dft;
  arp_status r;
  if ((r = check_cuda(c, cudaMemcpyAsync(d->status_host, d->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                      "dft: status read")) != ARP_OK ||
      (r = check_cuda(c, cudaStreamSynchronize(s), "dft: synchronise")) != ARP_OK)
    return r;
  if (*d->status_host != 0u) {
    cudaMemsetAsync(d->status, 0, sizeof(unsigned), s);
    return fail(c, ARP_ETIMEOUT, "dft gemm: a bounded wait of the tensor-core kernel gave up");
  }
  return ARP_OK;
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
        W + (size_t)s0 * 3 * K1, nb, M, c->K, d->R, c->phase32, c->inv_sig32, c->sk_sig32, (E*)d->A,
        d->cols * (size_t)d->R);
    if ((r = check_cuda(c, cudaGetLastError(), "dft: pack")) != ARP_OK) return r;
    if ((r = dft_transforms<S>(c, groups, s)) != ARP_OK) return r;
    dft_unpack_avg_kernel<<<dim3((K1 + 31) / 32, nb), dim3(32, kAvgChunks), 0, s>>>(
        d->Q, nb, M, c->K, d->R, c->phase32, c->weight32, c->inv_sig32, c->sk_sig32, partial + (size_t)s0 * 3 * K1);
    if ((r = check_cuda(c, cudaGetLastError(), "dft: unpack")) != ARP_OK) return r;
  }
  return dft_status(c, s);
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
                                                                  c->sk_sig32, (E*)d->A, d->cols * (size_t)d->R);
      if ((r = check_cuda(c, cudaGetLastError(), "dft fine: pack")) != ARP_OK) return r;
      if ((r = dft_transforms<S>(c, batch, s)) != ARP_OK) return r;
      dft_fine_stage_kernel<<<blocks_for(n, 128), 128, 0, s>>>(d->Q, batch, c->K, d->R, stage, tb, d->U, d->ULO,
                                                                d->NU, d->A1, d->ACC, d->XS);
      if ((r = check_cuda(c, cudaGetLastError(), "dft fine: stage")) != ARP_OK) return r;
    }
  }
  dft_fine_store_kernel<<<blocks_for((long long)batch * c->H, 128), 128, 0, s>>>(out, batch, c->H, c->K, tb, d->U,
                                                                                  d->ULO);
  if ((r = check_cuda(c, cudaGetLastError(), "dft fine: store")) != ARP_OK) return r;
  return dft_status(c, s);
}

template <class S>
__global__ void split_rows_kernel(const float* __restrict__ X, long long rows, int cols, int ld,
                                  typename S::E* out, size_t part_stride) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * ld) return;
  const long long r = t / ld;
  const int k = (int)(t % ld);
  S::split(k < cols ? X[r * cols + k] : 0.0f, out + t, part_stride);
}

// C (n x m, row-major FP32), C[j][i] = sum_k A[i][k] B[j][k], with A (m x k)
// and B (n x k) row-major FP32, through the split-precision tensor-core kernel
// (operands split and padded in temporary device buffers).
template <class S>
arp_status gemm_check_t(arp_ctx* c, int m, int n, int k, const float* A, const float* B, float* C, cudaStream_t s) {
  const int mp = (m + tc::kBM - 1) / tc::kBM * tc::kBM;
  const int ke = tc::kRowBytes / (int)sizeof(typename S::E);
  const int kp = (k + ke - 1) / ke * ke;
  const size_t eb = sizeof(typename S::E);
  void *a = nullptr, *b = nullptr;
  unsigned* st = nullptr;
  float* ct = nullptr;
  arp_status r = ARP_OK;
  if (cudaMalloc(&a, (size_t)S::kParts * mp * kp * eb) != cudaSuccess ||
      cudaMalloc(&b, (size_t)S::kParts * n * kp * eb) != cudaSuccess ||
      cudaMalloc(&ct, (size_t)n * mp * sizeof(float)) != cudaSuccess || cudaMalloc(&st, sizeof(unsigned)) != cudaSuccess)
    r = fail(c, ARP_ENOMEM, "gemm check: allocation");
  if (r == ARP_OK) r = check_cuda(c, cudaMemsetAsync(a, 0, (size_t)S::kParts * mp * kp * eb, s), "gemm check");
  if (r == ARP_OK) r = check_cuda(c, cudaMemsetAsync(st, 0, sizeof(unsigned), s), "gemm check");
  if (r == ARP_OK) {
    split_rows_kernel<S><<<blocks_for((long long)m * kp, 256), 256, 0, s>>>(A, m, k, kp, (typename S::E*)a,
                                                                             (size_t)mp * kp);
    split_rows_kernel<S><<<blocks_for((long long)n * kp, 256), 256, 0, s>>>(B, n, k, kp, (typename S::E*)b,
                                                                             (size_t)n * kp);
    r = check_cuda(c, cudaGetLastError(), "gemm check: split");
  }
  // the kernel stores C^T column-major: ct[col * mp + row] = C[row][col]
  if (r == ARP_OK) r = tc_gemm<S, tc::kEpiStore>(c, a, mp, b, n, n, kp,
                                                tc::Epilogue{ct, nullptr, n, mp, 0, 0, m, st}, s);
  if (r == ARP_OK)
    r = check_cuda(c, cudaMemcpy2DAsync(C, (size_t)m * sizeof(float), ct, (size_t)mp * sizeof(float),
                                        (size_t)m * sizeof(float), (size_t)n, cudaMemcpyDeviceToDevice, s),
                   "gemm check: copy");
  unsigned hs = 0;
  if (r == ARP_OK) r = check_cuda(c, cudaMemcpyAsync(&hs, st, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "gemm check");
  if (r == ARP_OK) r = check_cuda(c, cudaStreamSynchronize(s), "gemm check: synchronise");
  if (r == ARP_OK && hs) r = fail(c, ARP_ETIMEOUT, "gemm check: a bounded wait gave up");
  cudaFree(a);
  cudaFree(b);
  cudaFree(ct);
  cudaFree(st);
  return r;
}

}  // namespace

bool dft_mode(const arp_ctx* c) {
  return c->precision == ARP_TF32X3 || c->precision == ARP_BF16X2 || c->precision == ARP_BF16X3;
}

arp_status dft_nbar(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  switch (c->precision) {
    case ARP_BF16X2: return dft_nbar_t<SplitBF16x2>(c, W, partial, batch, s);
    case ARP_BF16X3: return dft_nbar_t<SplitBF16x3>(c, W, partial, batch, s);
    default: return dft_nbar_t<SplitTF32x3>(c, W, partial, batch, s);
  }
}

arp_status dft_fine(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  switch (c->precision) {
    case ARP_BF16X2: return dft_fine_t<SplitBF16x2>(c, in, out, batch, s);
    case ARP_BF16X3: return dft_fine_t<SplitBF16x3>(c, in, out, batch, s);
    default: return dft_fine_t<SplitTF32x3>(c, in, out, batch, s);
  }
}

void dft_release(arp_ctx* c) {
  DftWork* d = c->dft;
  if (!d) return;
  void* ptrs[] = {d->Winv, d->Wfwd, d->A, d->P, d->Q, d->U, d->ULO, d->NU, d->A1, d->ACC, d->XS, d->status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (d->status_host) cudaFreeHost(d->status_host);
  delete d;
  c->dft = nullptr;
}

}  // namespace arp

extern "C" arp_status arp_gemm_check(int precision, int m, int n, int k, const float* A, const float* B, float* C,
                                     void* stream) {
  using namespace arp;
  if (m < 1 || n < 1 || k < 1 || m > (1 << 16) || n > (1 << 22) || k > (1 << 16) || !A || !B || !C) return ARP_EINVAL;
  if ((long long)(n + tc::kBN - 1) / tc::kBN > 65535) return ARP_EINVAL;
  arp_ctx c;  // host-side error record only
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (precision) {
    case ARP_TF32X3: return gemm_check_t<SplitTF32x3>(&c, m, n, k, A, B, C, s);
    case ARP_BF16X2: return gemm_check_t<SplitBF16x2>(&c, m, n, k, A, B, C, s);
    case ARP_BF16X3: return gemm_check_t<SplitBF16x3>(&c, m, n, k, A, B, C, s);
    default: return ARP_EINVAL;
  }
}
