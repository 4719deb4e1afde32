// pipeline.cu -- arp_parareal_solve as a pipeline across iterations.
//
// The parareal recursion (Eq. 3.1, Algorithm 4) only orders
//   link n of the chain of iteration k   after  F(U_n^{k-1})   (V_n needs it),
//   F(U_n^k)                              after  link n-1 of iteration k,
// so the fine sweeps of iteration k can start on the first slices while the
// chain of iteration k is still running on later ones.  This driver splits
// the S links into chunks; per chunk j of level L it enqueues, on one chain
// stream, the correction V = F - G, the cluster chain over the chunk's links
// (its eigen-basis state carried to the next chunk exactly), and the finish
// (U_{n+1}, G cache) with the per-slice change of the states it writes in the
// same launch; a fine stream per chunk runs F
// on the slices whose start states that chunk produced, as soon as it is done.
// Every kernel computes per slice or per link exactly what the level-by-level
// iteration computes, so the result is the same bit for bit; only the order in
// time differs.  The host reads each level's change before it enqueues the
// next level, so the stopping rule is the level-by-level one too.
//
// The cluster chain needs 16 whole SMs; fine blocks placed on them would stall
// it for a whole fine sweep.  So the SMs are split into two green contexts (an
// execution-resource partition of the device; memory stays shared): a group
// on which one cluster of the chain fits, and the rest for the fine sweeps.
// The driver entry points are resolved at run time through the runtime, so the
// library does not link the driver library.
#include <cuda.h>

#include <cmath>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "context.h"
#include "parareal_kernels.cuh"

namespace arp {

// The device's SM partition, made once per process and shared by every
// context: green context 0 holds the chain's cluster, 1 the rest for the fine
// sweeps.  A green context may be current on one thread at a time, so pushing
// either one holds `mu`.
struct Partition {
  bool ok = false;
  std::string why;
  CUgreenCtx g[2] = {nullptr, nullptr};
  CUcontext x[2] = {nullptr, nullptr};
  int sms[2] = {0, 0};
  std::mutex mu;
};

struct Pipe {
  bool built = false, ok = false;
  bool refused = false;               // a call on the partitions failed once; the context solves level by level
  std::string why;                    // why the pipeline is unavailable
  Partition* part = nullptr;          // the shared partition (not owned)
  CUgreenCtx g[2] = {nullptr, nullptr};  // its green contexts: 0 chain, 1 fine
  CUcontext x[2] = {nullptr, nullptr};
  int sms[2] = {0, 0};
  int cluster = 0;                    // chain cluster size that fits the chain partition
  CUstream sc = nullptr;              // chain stream
  std::vector<CUstream> sf;           // one fine stream per chunk
  std::vector<CUevent> ec, ef;        // per chunk: chain part done (chain ctx), fine part done (fine ctx)
  CUevent start = nullptr;            // user stream's work before the solve (primary context)
  CUevent done = nullptr;             // a level's chain part and change read back (chain ctx)
  cd* Fb2 = nullptr;                  // second fine-result buffer
  cd* Wc = nullptr;                   // [3][K1] chain state carried between chunks
  double* hchg = nullptr;             // pinned: the last level's change, then the chain's status word
  int chunk = 0, nchunks = 0;
};

void pipeline_release(arp_ctx* c);

namespace {

struct Driver {
  bool ok = false;
  decltype(&cuDeviceGetDevResource) getDevResource = nullptr;
  decltype(&cuDevSmResourceSplitByCount) split = nullptr;
  decltype(&cuDevResourceGenerateDesc) genDesc = nullptr;
  decltype(&cuGreenCtxCreate) greenCreate = nullptr;
  decltype(&cuGreenCtxDestroy) greenDestroy = nullptr;
  decltype(&cuCtxFromGreenCtx) fromGreen = nullptr;
  decltype(&cuGreenCtxStreamCreate) greenStream = nullptr;
  decltype(&cuCtxPushCurrent) push = nullptr;
  decltype(&cuCtxPopCurrent) pop = nullptr;
  decltype(&cuStreamDestroy) streamDestroy = nullptr;
  decltype(&cuEventCreate) eventCreate = nullptr;
  decltype(&cuEventDestroy) eventDestroy = nullptr;
  decltype(&cuEventRecord) eventRecord = nullptr;
  decltype(&cuEventSynchronize) eventSync = nullptr;
  decltype(&cuStreamWaitEvent) waitEvent = nullptr;
};

template <typename F>
bool entry(const char* name, F* fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion(name, &p, CUDA_VERSION, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *fn = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    d.ok = entry("cuDeviceGetDevResource", &d.getDevResource) && entry("cuDevSmResourceSplitByCount", &d.split) &&
           entry("cuDevResourceGenerateDesc", &d.genDesc) && entry("cuGreenCtxCreate", &d.greenCreate) &&
           entry("cuGreenCtxDestroy", &d.greenDestroy) && entry("cuCtxFromGreenCtx", &d.fromGreen) &&
           entry("cuGreenCtxStreamCreate", &d.greenStream) && entry("cuCtxPushCurrent", &d.push) &&
           entry("cuCtxPopCurrent", &d.pop) && entry("cuStreamDestroy", &d.streamDestroy) &&
           entry("cuEventCreate", &d.eventCreate) && entry("cuEventDestroy", &d.eventDestroy) &&
           entry("cuEventRecord", &d.eventRecord) && entry("cuEventSynchronize", &d.eventSync) &&
           entry("cuStreamWaitEvent", &d.waitEvent);
  });
  return d;
}

// Makes a partition's context current for the enclosed runtime calls (the
// partition's lock held meanwhile).
struct Current {
  const Driver& d;
  std::lock_guard<std::mutex> lock;
  bool pushed;
  Current(const Driver& drv, Partition* part, CUcontext x)
      : d(drv), lock(part->mu), pushed(drv.push(x) == CUDA_SUCCESS) {}
  ~Current() {
    CUcontext prev;
    if (pushed) d.pop(&prev);
  }
};

arp_status drv_check(arp_ctx* c, CUresult e, const char* what) {
  if (e == CUDA_SUCCESS) return ARP_OK;
  return fail(c, ARP_ECUDA, std::string("pipeline: ") + what + " failed (CUresult " + std::to_string((int)e) + ")");
}

// The per-context streams and events (the shared partition stays).
void destroy_streams(Pipe& p) {
  const Driver& d = driver();
  if (!d.ok) return;
  for (CUevent& e : p.ec) if (e) d.eventDestroy(e);
  for (CUevent& e : p.ef) if (e) d.eventDestroy(e);
  for (CUstream& s : p.sf) if (s) d.streamDestroy(s);
  p.ec.clear();
  p.ef.clear();
  p.sf.clear();
  if (p.done) d.eventDestroy(p.done);
  if (p.start) d.eventDestroy(p.start);
  if (p.sc) d.streamDestroy(p.sc);
  p.done = p.start = nullptr;
  p.sc = nullptr;
}

// Splits the device's SMs into a group of at least 16 SMs, grouped so that
// large clusters fit (the chain's), and the rest.  part.ok false, with
// part.why set, if the split or the contexts cannot be made.
void make_partition(Partition& part, int device) {
  const Driver& d = driver();
  CUdevResource all{}, grp{}, rest{};
  if (!d.ok) {
    part.why = "the driver has no green-context entry points";
    return;
  }
  if (d.getDevResource((CUdevice)device, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) {
    part.why = "the device's SM resource cannot be read";
    return;
  }
  unsigned nb = 1;
  if (d.split(&grp, &nb, &all, &rest, CU_DEV_SM_RESOURCE_SPLIT_MAX_POTENTIAL_CLUSTER_SIZE, 16) != CUDA_SUCCESS ||
      nb < 1 || rest.sm.smCount < 1) {
    part.why = "the SMs cannot be split into a chain group and a fine group";
    return;
  }
  CUdevResource* parts[2] = {&grp, &rest};
  for (int i = 0; i < 2; ++i) {
    CUdevResourceDesc desc;
    if (d.genDesc(&desc, parts[i], 1) != CUDA_SUCCESS ||
        d.greenCreate(&part.g[i], desc, (CUdevice)device, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS ||
        d.fromGreen(&part.x[i], part.g[i]) != CUDA_SUCCESS) {
      part.why = "a green context cannot be created";
      for (int j = 0; j <= i; ++j)
        if (part.g[j]) d.greenDestroy(part.g[j]);
      part.g[0] = part.g[1] = nullptr;
      part.x[0] = part.x[1] = nullptr;
      return;
    }
    part.sms[i] = (int)parts[i]->sm.smCount;
  }
  part.ok = true;
}

// The partition of `device`, made on the first request of the process; it
// lives as long as the process.
Partition* shared_partition(int device) {
  static std::mutex mu;
  static std::map<int, std::unique_ptr<Partition>> parts;
  std::lock_guard<std::mutex> lock(mu);
  std::unique_ptr<Partition>& part = parts[device];
  if (!part) {
    part.reset(new Partition);
    make_partition(*part, device);
  }
  return part.get();
}

// Per-chunk streams (fine partition) and events for chunks of `chunk` links.
arp_status make_chunks(arp_ctx* c, Pipe& p, int chunk) {
  const Driver& d = driver();
  for (CUevent& e : p.ec) d.eventDestroy(e);
  for (CUevent& e : p.ef) d.eventDestroy(e);
  for (CUstream& s : p.sf) d.streamDestroy(s);
  p.ec.clear();
  p.ef.clear();
  p.sf.clear();
  p.chunk = chunk;
  p.nchunks = (c->slices + chunk - 1) / chunk;
  // the chain takes the fine results chunk by chunk, so earlier chunks' sweeps
  // get the higher stream priority (block dispatch prefers them)
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  arp_status r;
  for (int j = 0; j < p.nchunks; ++j) {
    const int prio = p.nchunks > 1 ? greatest + (least - greatest) * j / (p.nchunks - 1) : greatest;
    CUevent e0 = nullptr, e1 = nullptr;
    CUstream s1 = nullptr;
    {
      Current cur(d, p.part, p.x[0]);
      if ((r = drv_check(c, d.eventCreate(&e0, CU_EVENT_DISABLE_TIMING), "event")) != ARP_OK) return r;
    }
    p.ec.push_back(e0);
    Current cur(d, p.part, p.x[1]);
    if ((r = drv_check(c, d.greenStream(&s1, p.g[1], CU_STREAM_NON_BLOCKING, prio), "fine stream")) != ARP_OK)
      return r;
    p.sf.push_back(s1);
    if ((r = drv_check(c, d.eventCreate(&e1, CU_EVENT_DISABLE_TIMING), "event")) != ARP_OK) return r;
    p.ef.push_back(e1);
  }
  return ARP_OK;
}

// c's streams, events and buffers on the shared partition, after checking
// that c's chain cluster (16 CTAs, else 8) fits the chain partition.  ARP_OK
// with nothing made (p.why set) where the partition is unavailable or the
// cluster does not fit.
arp_status make_pipe(arp_ctx* c, Pipe& p) {
  const Driver& d = driver();
  // A profiler attaches through an injection library (announced in the
  // environment); Nsight Compute fails to prepare the chain's cluster kernel
  // launched on a green-context stream ("Failed to prepare kernel for
  // profiling") and then ends the application, so with one attached the solve
  // runs level by level (the same kernels per slice and per link).
  for (const char* var : {"CUDA_INJECTION64_PATH", "NV_NSIGHT_INJECTION_TRANSPORT_TYPE",
                          "NV_COMPUTE_PROFILER_PERFWORKS_DIR"}) {
    const char* v = std::getenv(var);
    if (v && *v) {
      p.why = "a profiler is attached; green-context launches cannot be profiled";
      return ARP_OK;
    }
  }
  Partition* part = shared_partition(c->device);
  if (!part->ok) {
    p.why = part->why;
    return ARP_OK;
  }
  p.part = part;
  for (int i = 0; i < 2; ++i) {
    p.g[i] = part->g[i];
    p.x[i] = part->x[i];
    p.sms[i] = part->sms[i];
  }
  for (int want : {16, 8}) {
    Current cur(d, p.part, p.x[0]);
    ChainRange probe;
    probe.check_only = true;
    probe.cluster = want;
    if (launch_cluster_chain(c, c->U, c->Ge, nullptr, nullptr, &probe) == ARP_OK) {
      p.cluster = want;
      break;
    }
  }
  c->err.clear();
  if (!p.cluster) {
    p.why = "no chain cluster fits the chain partition";
    p.part = nullptr;
    return ARP_OK;
  }
  arp_status r;
  if ((r = check_cuda(c, cudaMalloc(&p.Fb2, (size_t)c->slices * 3 * c->H * sizeof(cd)), "pipeline: fine buffer")) !=
          ARP_OK ||
      (r = check_cuda(c, cudaMalloc(&p.Wc, (size_t)3 * c->K1 * sizeof(cd)), "pipeline: carried state")) != ARP_OK ||
      (r = check_cuda(c, cudaMallocHost(&p.hchg, 2 * sizeof(double)), "pipeline: change read-back")) != ARP_OK ||
      (r = drv_check(c, d.eventCreate(&p.start, CU_EVENT_DISABLE_TIMING), "event")) != ARP_OK)
    return r;
  Current cur(d, p.part, p.x[0]);
  if ((r = drv_check(c, d.greenStream(&p.sc, p.g[0], CU_STREAM_NON_BLOCKING, 0), "chain stream")) != ARP_OK ||
      (r = drv_check(c, d.eventCreate(&p.done, CU_EVENT_DISABLE_TIMING), "event")) != ARP_OK)
    return r;
  return ARP_OK;
}

// c's pipeline, made on first use; p.ok false (and the level-by-level solve
// used) where it cannot be made.  A failure while making it releases what was
// made and is returned.
arp_status ensure_pipe(arp_ctx* c) {
  if (!c->pipe) c->pipe = new Pipe;
  Pipe& p = *c->pipe;
  const int S = c->slices;
  const int chunk = c->pipeline >= 2 ? std::min(c->pipeline, S) : std::min(16, std::max(4, (S + 15) / 16));
  if (p.refused) return ARP_OK;
  arp_status r = ARP_OK;
  if (!p.built) {
    p.built = true;
    r = make_pipe(c, p);
  }
  if (r == ARP_OK && p.sc && (!p.ok || p.chunk != chunk)) {
    p.ok = false;
    r = make_chunks(c, p, chunk);
    p.ok = (r == ARP_OK);
  }
  if (r != ARP_OK) {
    const std::string why = c->err;
    pipeline_release(c);
    c->pipe = new Pipe;
    c->pipe->built = true;
    c->pipe->why = why;
  }
  return r;
}

BasisTabs tabs_of(const arp_ctx* c) { return BasisTabs{c->inv_sig64, c->sk_sig64, c->dhalf}; }

struct Level {
  cd* buf[2];  // U of levels Lb, Lb+2, ... and Lb+1, Lb+3, ...
  cd* fb[2];   // F(U^L) of the same parity
  int Lb;
  cd* U(int L) const { return buf[(L - Lb) & 1]; }
  cd* F(int L) const { return fb[(L - Lb) & 1]; }
};

// Chunk j of level L on the chain stream (L = 0: the predictor, no
// correction and no change): V = F(U^{L-1}) - G(U^{L-1}) for its links once
// the fine sweeps it needs are done, the chain over its links, U^L and the G
// cache of its links, the change of the slices it produced.
arp_status chain_chunk(arp_ctx* c, Pipe& p, const Level& lv, int L, int j) {
  const Driver& d = driver();
  const int S = c->slices, H = c->H, K1 = c->K1;
  const size_t st = (size_t)3 * H, se = (size_t)3 * K1;
  const int a = j * p.chunk, nl = std::min(p.chunk, S - a);
  cudaStream_t s = (cudaStream_t)p.sc;
  cd* U = lv.U(L);
  arp_status r;
  if (L >= 1) {
    if ((r = drv_check(c, d.waitEvent(p.sc, p.ef[j], 0), "wait")) != ARP_OK) return r;
    correction_kernel<<<nl, 256, 0, s>>>(lv.F(L - 1) + a * st, c->Gc + a * st, c->V + a * st, c->VT + a * se, H, K1,
                                         tabs_of(c));
  }
  ChainRange rg;
  rg.n0 = a;
  rg.nl = nl;
  rg.Win = j > 0 ? p.Wc : nullptr;
  rg.Wout = j + 1 < p.nchunks ? p.Wc : nullptr;
  rg.cluster = p.cluster;
  if ((r = launch_cluster_chain(c, U, c->Ge, L >= 1 ? c->VT : nullptr, s, &rg)) != ARP_OK) return r;
  // U and the G cache of the chunk's links, and at iterations the per-slice change, in one launch
  finish_change_kernel<<<nl, 256, 0, s>>>(c->Ge + a * se, L >= 1 ? c->V + a * st : nullptr, U + a * st,
                                          c->Gc + a * st, L >= 1 ? lv.U(L - 1) + a * st : nullptr, c->rel + a, H, K1,
                                          K1, tabs_of(c));
  if ((r = check_cuda(c, cudaGetLastError(), "pipeline: chain chunk")) != ARP_OK) return r;
  return drv_check(c, d.eventRecord(p.ec[j], p.sc), "record");
}

// Chunk j of level L's fine sweeps: F(U_n^L) for the slices chunk j of the
// chain produced (chunk 0 also takes slice 0, whose state u0 never changes),
// after that chunk of the chain when `after_chain`.
arp_status fine_chunk(arp_ctx* c, Pipe& p, const Level& lv, int L, int j, bool after_chain) {
  const Driver& d = driver();
  const int S = c->slices;
  const size_t st = (size_t)3 * c->H;
  const int a = j * p.chunk, b = std::min(S, a + p.chunk);
  const int f0 = j == 0 ? 0 : a + 1, f1 = std::min(b + 1, S);
  arp_status r;
  if (after_chain && (r = drv_check(c, d.waitEvent(p.sf[j], p.ec[j], 0), "wait")) != ARP_OK) return r;
  if (f1 > f0 && (r = launch_fine(c, lv.U(L) + f0 * st, lv.F(L) + f0 * st, f1 - f0, (cudaStream_t)p.sf[j])) != ARP_OK)
    return r;
  return drv_check(c, d.eventRecord(p.ef[j], p.sf[j]), "record");
}

// Level L: its chain (if `chain`) and its fine sweeps (if `fine`), enqueued
// chunk by chunk so that each chunk's fine sweeps are queued right behind it;
// then, for L >= 1, the change, read back into pinned memory.
arp_status level(arp_ctx* c, Pipe& p, const Level& lv, int L, bool chain, bool fine) {
  const Driver& d = driver();
  arp_status r;
  for (int j = 0; j < p.nchunks; ++j) {
    if (chain) {
      Current cur(d, p.part, p.x[0]);
      if ((r = chain_chunk(c, p, lv, L, j)) != ARP_OK) return r;
    }
    if (fine) {
      Current cur(d, p.part, p.x[1]);
      if ((r = fine_chunk(c, p, lv, L, j, chain)) != ARP_OK) return r;
    }
  }
  if (!chain) return ARP_OK;
  Current cur(d, p.part, p.x[0]);
  if (L >= 1) {
    max_kernel<<<1, 256, 0, (cudaStream_t)p.sc>>>(c->rel, c->slices, c->scalar);
    if ((r = check_cuda(c, cudaGetLastError(), "pipeline: norm")) != ARP_OK) return r;
    if ((r = check_cuda(c, cudaMemcpyAsync(p.hchg, c->scalar, sizeof(double), cudaMemcpyDeviceToHost,
                                           (cudaStream_t)p.sc), "pipeline: change read")) != ARP_OK)
      return r;
  }
  // the chain's status word (sticky over the solve's levels)
  if ((r = check_cuda(c, cudaMemcpyAsync(p.hchg + 1, c->sync + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                         (cudaStream_t)p.sc), "pipeline: status read")) != ARP_OK)
    return r;
  return drv_check(c, d.eventRecord(p.done, p.sc), "record");
}

}  // namespace

bool pipeline_eligible(const arp_ctx* c) {
  if (c->pipeline == 0 || c->coarse_scheme != 0 || c->coarse_grid || dft_mode(c) || c->skip_arrival) return false;
  if (c->chain_mode == 3) return true;
  return c->chain_mode == 0 && !fp64_grid_first(c);
}

arp_status parareal_solve_pipelined(arp_ctx* c, cudaStream_t user, bool* ran, int* k_done, double* change) {
  *ran = false;
  arp_status r;
  if ((r = ensure_pipe(c)) != ARP_OK) return r;
  Pipe& p = *c->pipe;
  c->last_pipelined = 0;
  if (!p.ok) return ARP_OK;
  *ran = true;
  c->last_pipelined = 1;
  const Driver& d = driver();
  const int L0 = c->level, kmax = c->kmax;
  double ch = INFINITY;
  int L = L0;
  const Level lv{{c->U, c->Uold}, {c->Fb, p.Fb2}, std::max(L0, 0)};
  const size_t st = (size_t)3 * c->H;

  // order after the caller's stream; u0 into both buffers
  if ((r = drv_check(c, d.eventRecord(p.start, (CUstream)user), "record")) != ARP_OK) return r;
  {
    Current cur(d, p.part, p.x[0]);
    if ((r = drv_check(c, d.waitEvent(p.sc, p.start, 0), "wait")) != ARP_OK) return r;
    if ((r = check_cuda(c, cudaMemcpyAsync(c->Uold, c->U, st * sizeof(cd), cudaMemcpyDeviceToDevice,
                                           (cudaStream_t)p.sc), "pipeline: copy u0")) != ARP_OK ||
        (r = check_cuda(c, cudaMemsetAsync(c->sync, 0, 4 * sizeof(unsigned), (cudaStream_t)p.sc),
                        "pipeline: status reset")) != ARP_OK)
      return r;
  }
  const unsigned* hstatus = reinterpret_cast<const unsigned*>(p.hchg + 1);
  bool unchecked = false;  // a chain level whose status word has not been read yet
  {
    Current cur(d, p.part, p.x[1]);
    for (CUstream s : p.sf)
      if ((r = drv_check(c, d.waitEvent(s, p.start, 0), "wait")) != ARP_OK) return r;
  }

  // the caller's stream waits for everything enqueued on the partitions
  auto join = [&]() {
    arp_status q;
    {
      Current cur(d, p.part, p.x[0]);
      q = drv_check(c, d.eventRecord(p.done, p.sc), "record");
    }
    if (q == ARP_OK) q = drv_check(c, d.waitEvent((CUstream)user, p.done, 0), "wait");
    for (CUevent e : p.ef)
      if (q == ARP_OK) q = drv_check(c, d.waitEvent((CUstream)user, e, 0), "wait");
    return q;
  };
  auto finish = [&](arp_status status) {
    if (status == ARP_OK && unchecked) {
      status = drv_check(c, d.eventSync(p.done), "synchronise");
      if (status == ARP_OK && *hstatus != 0u) status = chain_status(c, *hstatus);
    }
    const arp_status q = join();
    if (L > L0) {
      if ((L - lv.Lb) & 1) std::swap(c->U, c->Uold);
      c->level = L;
    }
    if (k_done) *k_done = L;
    if (change) *change = ch;
    return status != ARP_OK ? status : q;
  };

  if (L < 0) {
    if ((r = level(c, p, lv, 0, true, kmax > 0)) != ARP_OK) return finish(r);
    unchecked = true;
    L = 0;
  } else if (L < kmax) {
    if ((r = level(c, p, lv, L, false, true)) != ARP_OK) return finish(r);
  }
  while (L < kmax && !(L >= 1 && ch <= c->tol)) {
    if ((r = level(c, p, lv, L + 1, true, L + 1 < kmax)) != ARP_OK) return finish(r);
    if ((r = drv_check(c, d.eventSync(p.done), "synchronise")) != ARP_OK) return finish(r);
    unchecked = false;
    if (*hstatus != 0u) return finish(chain_status(c, *hstatus));
    ch = *p.hchg;
    L += 1;
    if (!std::isfinite(ch)) return finish(fail(c, ARP_ENONFINITE, "parareal: relative change is not finite"));
  }
  return finish(ARP_OK);
}

bool pipeline_recover(arp_ctx* c) {
  Pipe* p = c->pipe;
  if (!p || !p->ok) return false;
  const std::string cause = c->err;
  cudaGetLastError();  // a refused launch leaves a non-sticky error behind
  bool usable = true;
  if (p->sc && cudaStreamSynchronize((cudaStream_t)p->sc) != cudaSuccess) usable = false;
  for (CUstream s : p->sf)
    if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess) usable = false;
  if (cudaDeviceSynchronize() != cudaSuccess) usable = false;
  cudaGetLastError();
  if (!usable) return false;  // a fault: the context is lost, nothing to fall back to
  p->ok = false;
  p->refused = true;
  p->why = "a call on the SM partitions failed (" + cause + "); this context solves level by level";
  c->last_pipelined = 0;
  c->err.clear();
  return true;
}

arp_status pipeline_info(const arp_ctx* c, int* out) {
  const Pipe* p = c->pipe;
  out[0] = c->last_pipelined;
  out[1] = p && p->ok ? p->sms[0] : 0;
  out[2] = p && p->ok ? p->sms[1] : 0;
  out[3] = p && p->ok ? p->chunk : 0;
  out[4] = p && p->ok ? p->cluster : 0;
  out[5] = p && p->refused ? 1 : 0;
  return ARP_OK;
}

void pipeline_release(arp_ctx* c) {
  if (!c->pipe) return;
  Pipe& p = *c->pipe;
  if (p.sc) cudaStreamSynchronize((cudaStream_t)p.sc);
  for (CUstream s : p.sf) cudaStreamSynchronize((cudaStream_t)s);
  destroy_streams(p);
  if (p.Fb2) cudaFree(p.Fb2);
  if (p.Wc) cudaFree(p.Wc);
  if (p.hchg) cudaFreeHost(p.hchg);
  delete c->pipe;
  c->pipe = nullptr;
}

}  // namespace arp
