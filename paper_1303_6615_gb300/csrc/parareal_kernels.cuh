// parareal_kernels.cuh -- FP64 streaming kernels of the parareal correction
// and of the stopping quantity, shared by the single-problem driver and by
// batches (the same reduction order in both, so results do not depend on the
// batch).
#pragma once

#include <cmath>

#include "spectral.cuh"

namespace arp {

// Tables the correction and finish bodies read: the eigen constants and
// e^{dT/2 D} per wavenumber k < K1.
struct BasisTabs {
  const double* is64;
  const double* ss64;
  const double* dhalf;
};

// Slice n of the correction: V_n = F_n - G_n (all H bins, three fields) and,
// for k < K1v, VT_n = e^{dT/2 D} R^H V_n (three branches, row stride K1v), the
// form in which the cluster chain adds V_n to its eigen-basis state (K1v < K1
// when the chain runs on a coarser grid: only its modes are needed).
__device__ __forceinline__ void corr_body(const cd* __restrict__ F, const cd* __restrict__ G, cd* __restrict__ V,
                                          cd* __restrict__ VT, int n, int H, int K1v, const BasisTabs& tb) {
  const size_t o = (size_t)n * 3 * H;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    cd v[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      v[f] = F[o + (size_t)f * H + k] - G[o + (size_t)f * H + k];
      V[o + (size_t)f * H + k] = v[f];
    }
    if (k < K1v) {
      cd e[3];
      phys_to_eigen<double>(v, tb.is64[k], tb.ss64[k], e);
#pragma unroll
      for (int b = 0; b < 3; ++b) VT[((size_t)n * 3 + b) * K1v + k] = tb.dhalf[k] * e[b];
    }
  }
}

// Slice n after the cluster chain: the G cache G_n = R g_n (the imaginary
// part of the k = 0 mode dropped, a real field's mean) and U_{n+1} = G_n + V_n
// (V = null: the predictor), zero above the kept modes K1.  g_n has K1g modes
// (row stride K1g); a chain on a coarser grid leaves G_n = 0 for K1g <= k < K1,
// where U_{n+1} = V_n.
__device__ __forceinline__ void finish_body(const cd* __restrict__ Ge, const cd* __restrict__ V, cd* __restrict__ U,
                                            cd* __restrict__ Gc, int n, int H, int K1, int K1g, const BasisTabs& tb) {
  const size_t o = (size_t)n * 3 * H, o1 = (size_t)(n + 1) * 3 * H;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    cd u[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    if (k < K1g) {
      cd g[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) g[b] = Ge[((size_t)n * 3 + b) * K1g + k];
      eigen_to_phys<double>(g, tb.is64[k], tb.ss64[k], u);
      if (k == 0)
#pragma unroll
        for (int f = 0; f < 3; ++f) u[f].y = 0.0;
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      Gc[o + (size_t)f * H + k] = u[f];
      U[o1 + (size_t)f * H + k] = (V && k < K1) ? u[f] + V[o + (size_t)f * H + k] : u[f];
    }
  }
}

// One block per slice: corr_body.
__global__ void correction_kernel(const cd* __restrict__ F, const cd* __restrict__ G, cd* __restrict__ V,
                                  cd* __restrict__ VT, int H, int K1v, BasisTabs tb);
// One block per slice: finish_body.
__global__ void finish_kernel(const cd* __restrict__ Ge, const cd* __restrict__ V, cd* __restrict__ U,
                              cd* __restrict__ Gc, int H, int K1, int K1g, BasisTabs tb);

// ||U_n - Uold_n||^2 and ||U_n||^2 (Parseval weights 1 at k = 0, 2 above) of the
// state at `base`, reduced by a 256-thread block in a fixed tree; thread 0
// returns ||U_n - Uold_n|| / ||U_n|| (0 if both vanish, inf if only ||U_n|| does).
__device__ __forceinline__ double slice_change_body(const cd* __restrict__ U, const cd* __restrict__ Uold, int H) {
  __shared__ double sd[256], sn[256];
  double d = 0.0, nn = 0.0;
  for (int i = threadIdx.x; i < 3 * H; i += 256) {
    const int k = i % H;
    const double w = (k == 0) ? 1.0 : 2.0;
    const cd a = U[i], b = Uold[i];
    const double dx = a.x - b.x, dy = a.y - b.y;
    d += w * (dx * dx + dy * dy);
    nn += w * (a.x * a.x + a.y * a.y);
  }
  sd[threadIdx.x] = d;
  sn[threadIdx.x] = nn;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sd[threadIdx.x] += sd[threadIdx.x + w];
      sn[threadIdx.x] += sn[threadIdx.x + w];
    }
    __syncthreads();
  }
  const double dd = sd[0], ns = sn[0];
  if (ns > 0.0) return sqrt(dd) / sqrt(ns);
  return (dd > 0.0) ? INFINITY : 0.0;
}

// max of rel[1..S] by a 256-thread block; NaN if any entry is NaN.
__device__ __forceinline__ double max_change_body(const double* __restrict__ rel, int S) {
  __shared__ double sm[256];
  __shared__ int bad[256];
  double m = 0.0;
  int nan = 0;
  for (int n = 1 + threadIdx.x; n <= S; n += 256) {
    const double r = rel[n];
    if (r != r) nan = 1;
    else m = fmax(m, r);
  }
  sm[threadIdx.x] = m;
  bad[threadIdx.x] = nan;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
      bad[threadIdx.x] |= bad[threadIdx.x + w];
    }
    __syncthreads();
  }
  return bad[0] ? NAN : sm[0];
}

// One 256-thread block per slice n: finish_body, then, if Uold is not null,
// rel[n+1] = ||U_{n+1} - Uold_{n+1}|| / ||U_{n+1}|| of the state it just wrote
// (slice_change_body, the same tree as slice_change_kernel: the same bits).
__global__ void finish_change_kernel(const cd* __restrict__ Ge, const cd* __restrict__ V, cd* __restrict__ U,
                                     cd* __restrict__ Gc, const cd* __restrict__ Uold, double* __restrict__ rel, int H,
                                     int K1, int K1g, BasisTabs tb);
// One 256-thread block per slice n = 1..S: rel[n] = ||U_n - Uold_n|| / ||U_n||.
__global__ void slice_change_kernel(const cd* __restrict__ U, const cd* __restrict__ Uold, double* __restrict__ rel,
                                    int H);
// One 256-thread block: out[0] = max_n rel[n].
__global__ void max_kernel(const double* __restrict__ rel, int S, double* __restrict__ out);

}  // namespace arp
