// static_avg.cu -- the time average of the nonlinearity (the computation of
// arp_coarse_avg) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns a fixed
// device-memory budget and forbids allocation once it has started, or a
// latency-critical loop where cudaMalloc's implicit synchronisation is not
// acceptable.  They cannot create a context either, because arp_create
// allocates its tables and workspaces.  This entry point needs no context: it
// keeps its tables and workspaces in one file-scope device array of
// kStaticScratchBytes, which every GPU that loads the library holds until the
// process exits, and runs the same table, time-average and reduction kernels
// as arp_coarse_avg on it.  It never calls cudaMalloc, cudaFree or any other
// allocating routine.  With lazy module loading (the CUDA default) the array
// is placed on a device by the first call there (the symbol lookup loads this
// module), so callers make one call per device at start-up, before their
// memory budget is fixed and before any stream capture; if the device has no
// room left at that point the call returns ARP_ENOMEM.
#include <cmath>
#include <mutex>

#include "context.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" arp_status arp_coarse_avg_static(int N, double eps, double dT, int M, const double* U_in, double* Nbar_out,
                                            int batch, void* stream) {
  using namespace arp;
  if (N < 8 || N > 2048 || (N & (N - 1)) != 0) return ARP_EINVAL;
  if (!(eps > 0.0) || !(dT > 0.0) || std::isinf(dT) || M < 2 || M > (1 << 16) || batch < 0) return ARP_EINVAL;
  if (batch == 0) return ARP_OK;
  if (!U_in || !Nbar_out) return ARP_EINVAL;

  arp_ctx c;  // host-side description only; every device pointer points into the static array
  c.N = N;
  c.logN = 0;
  while ((1 << c.logN) < N) ++c.logN;
  c.H = N / 2 + 1;
  c.K = (N - 1) / 3;
  c.K1 = c.K + 1;
  c.M = M;
  c.qc = (M + kMaxNodeBlocks - 1) / kMaxNodeBlocks;
  c.P = (M + c.qc - 1) / c.qc;
  c.eps = eps;
  c.nu = 0.0;
  c.dT = dT;
  c.dt = dT;
  c.steps = 1;
  c.h = dT;
  c.precision = ARP_FP64;
  if (cudaGetDevice(&c.device) != cudaSuccess || c.device < 0 || c.device >= kMaxDevices) return ARP_ECUDA;

  const size_t K1 = c.K1, Ns = N, Ms = M, P = c.P;
  // tables, in the order below; then per-state workspace: W [3][K1] and partials [P][3][K1]
  const size_t sizes[] = {K1 * 8,  K1 * 8,          K1 * 4,          K1 * 4,      18 * K1 * 16, 18 * K1 * 8, 3 * K1 * 8,
                          Ns * 16, Ns * 8,          Ms * 3 * K1 * 16, Ms * 3 * K1 * 8, Ms * 8,     Ms * 4,      K1 * 8,
                          3 * K1 * 16, 3 * K1 * 16};
  size_t tables = 0;
  for (size_t z : sizes) tables += align256(z);
  const size_t per_state = 3 * K1 * 16 * (1 + P);
  if (tables + per_state + 512 > kStaticScratchBytes) return ARP_EINVAL;  // sizes beyond the array
  const int chunk = (int)((kStaticScratchBytes - tables - 512) / per_state);

  unsigned char* base = nullptr;
  const cudaError_t se = scratch_address(c.device, &base);
  if (se != cudaSuccess) {
    cudaGetLastError();
    // the array is placed on the device when this module loads, which under
    // lazy module loading is this first lookup: no room left means ARP_ENOMEM
    return se == cudaErrorMemoryAllocation ? ARP_ENOMEM : ARP_ECUDA;
  }
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += align256(bytes);
    return p;
  };
  c.inv_sig64 = reinterpret_cast<double*>(carve(sizes[0]));
  c.sk_sig64 = reinterpret_cast<double*>(carve(sizes[1]));
  c.inv_sig32 = reinterpret_cast<float*>(carve(sizes[2]));
  c.sk_sig32 = reinterpret_cast<float*>(carve(sizes[3]));
  c.etd64 = reinterpret_cast<cd*>(carve(sizes[4]));
  c.etd32 = reinterpret_cast<cf*>(carve(sizes[5]));
  c.E_lo32 = reinterpret_cast<cf*>(carve(sizes[6]));
  c.tw64 = reinterpret_cast<cd*>(carve(sizes[7]));
  c.tw32 = reinterpret_cast<cf*>(carve(sizes[8]));
  c.phase64 = reinterpret_cast<cd*>(carve(sizes[9]));
  c.phase32 = reinterpret_cast<cf*>(carve(sizes[10]));
  c.weight64 = reinterpret_cast<double*>(carve(sizes[11]));
  c.weight32 = reinterpret_cast<float*>(carve(sizes[12]));
  c.dhalf = reinterpret_cast<double*>(carve(sizes[13]));
  c.gphase = reinterpret_cast<cd*>(carve(sizes[14]));
  c.strang_h64 = reinterpret_cast<cd*>(carve(sizes[15]));
  c.W = reinterpret_cast<cd*>(carve((size_t)chunk * 3 * K1 * 16));
  c.partial = reinterpret_cast<cd*>(carve((size_t)chunk * P * 3 * K1 * 16));
  c.slices = chunk;
  c.cchunk = chunk;  // states per pass through the workspace

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  arp_status r = build_tables(&c, s);
  if (r != ARP_OK) return r;
  return coarse_avg(&c, reinterpret_cast<const cd*>(U_in), reinterpret_cast<cd*>(Nbar_out), batch, s);
}
