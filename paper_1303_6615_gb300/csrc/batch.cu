// batch.cu -- one parareal iteration (Eq. 3.1, Algorithm 4) of many independent
// problems at once: each context advances exactly as arp_parareal_iterate would
// advance it, but the work of all contexts with the same grid size and
// precision runs in fused launches -- one fine sweep over every (problem,
// slice), one correction, one launch of one thread-block cluster per problem
// for the serial chains, and one norm over every problem's slices.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "batch_impl.cuh"
#include "parareal_kernels.cuh"

namespace arp {

arp_status launch_fine_batch_f64(arp_ctx*, arp_ctx*, int, const void*, const int*, int, int, cudaStream_t);
arp_status launch_fine_batch_f32(arp_ctx*, arp_ctx*, int, const void*, const int*, int, int, cudaStream_t);
arp_status plan_chain_batch_f64(int, const int*, const int*, int, int*, ClusterPlan*, size_t*);
arp_status plan_chain_batch_f32(int, const int*, const int*, int, int*, ClusterPlan*, size_t*);
arp_status launch_chain_batch_f64(arp_ctx*, int, const void*, int, int, size_t, cudaStream_t);
arp_status launch_chain_batch_f32(arp_ctx*, int, const void*, int, int, size_t, cudaStream_t);

namespace {

struct CorrJob {
  const cd* F;
  const cd* G;
  cd* V;
  cd* VT;
  const cd* Uold0;
  cd* U0;
  int H, K1;
  BasisTabs tb;
};

struct FinishJob {
  const cd* Ge;
  const cd* V;  // null: predictor
  cd* U;
  cd* Gc;
  int H, K1;
  BasisTabs tb;
};

BasisTabs basis_tabs(const arp_ctx* c) { return BasisTabs{c->inv_sig64, c->sk_sig64, c->dhalf}; }

struct NormJob {
  const cd* U;
  const cd* Uold;
  double* rel;
  int H, S;
};

// Blocks per (problem, slice n < S): corr_body; slice 0 also copies u0 into the new iterate.
__global__ void corr_batch_kernel(const CorrJob* __restrict__ jobs, const int* __restrict__ first, int njobs) {
  const int i = find_job(first, njobs, blockIdx.x);
  const CorrJob j = jobs[i];
  const int n = blockIdx.x - first[i];
  corr_body(j.F, j.G, j.V, j.VT, n, j.H, j.K1, j.tb);
  if (n == 0)
    for (int t = threadIdx.x; t < 3 * j.H; t += blockDim.x) j.U0[t] = j.Uold0[t];
}

// Blocks per (problem, slice n < S) of the problems whose chain ran in a cluster: finish_body.
__global__ void finish_batch_kernel(const FinishJob* __restrict__ jobs, const int* __restrict__ first, int njobs) {
  const int i = find_job(first, njobs, blockIdx.x);
  const FinishJob j = jobs[i];
  finish_body(j.Ge, j.V, j.U, j.Gc, blockIdx.x - first[i], j.H, j.K1, j.K1, j.tb);
}

// 256-thread blocks per (problem, slice n = 1..S): the relative change of the slice.
__global__ void norm_batch_kernel(const NormJob* __restrict__ jobs, const int* __restrict__ first, int njobs) {
  const int i = find_job(first, njobs, blockIdx.x);
  const NormJob j = jobs[i];
  const int n = blockIdx.x - first[i] + 1;
  const double r = slice_change_body(j.U + (size_t)n * 3 * j.H, j.Uold + (size_t)n * 3 * j.H, j.H);
  if (threadIdx.x == 0) j.rel[n] = r;
}

// One 256-thread block per problem: out[i] = max_n rel[n].
__global__ void max_batch_kernel(const NormJob* __restrict__ jobs, double* __restrict__ out) {
  const NormJob j = jobs[blockIdx.x];
  const double m = max_change_body(j.rel, j.S);
  if (threadIdx.x == 0) out[blockIdx.x] = m;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace
}  // namespace arp

using namespace arp;

struct arp_batch {
  std::vector<arp_ctx*> ctx;
  int capacity = 0;                // members the device buffers are sized for
  int device = 0;
  unsigned char* dmem = nullptr;   // device: job arrays, prefix arrays, results
  size_t dbytes = 0;
  std::vector<unsigned char> host; // staging copy of the same layout
  std::vector<double> out;
  std::string err;
  // one stream per group of the iteration (forked from the caller's stream after
  // the job upload, joined back before the norms) and their events
  std::vector<cudaStream_t> gs;
  std::vector<cudaEvent_t> ge;
  cudaEvent_t ready = nullptr;
};

namespace {

struct Layout {
  size_t fine, chain, corr, fin, norm, first, out, status, total;
};

Layout layout_for(int n) {
  Layout L;
  size_t off = 0;
  L.fine = off;
  off += align256((size_t)n * std::max(sizeof(FineJob<double>), sizeof(FineJob<float>)));
  L.chain = off;
  off += align256((size_t)n * std::max(sizeof(ChainJob<double>), sizeof(ChainJob<float>)));
  L.corr = off;
  off += align256((size_t)n * sizeof(CorrJob));
  L.fin = off;
  off += align256((size_t)n * sizeof(FinishJob));
  L.norm = off;
  off += align256((size_t)n * sizeof(NormJob));
  L.first = off;
  off += align256((size_t)4 * (n + 1) * sizeof(int) * 2);
  L.out = off;
  off += align256((size_t)n * sizeof(double));
  L.status = off;  // per problem: the batched chain's status word, zero in the uploaded block
  off += align256((size_t)n * sizeof(unsigned));
  L.total = off;
  return L;
}

arp_status bfail(arp_batch* b, arp_status s, const std::string& m) {
  b->err = m;
  return s;
}

}  // namespace

extern "C" {

arp_status arp_batch_create(arp_batch** out, arp_ctx* const* ctxs, int count) {
  if (!out) return ARP_EINVAL;
  *out = nullptr;
  if (count < 1) return ARP_EINVAL;
  arp_batch* b = new (std::nothrow) arp_batch();
  if (!b) return ARP_ENOMEM;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ARP_ECUDA;
  }
  for (int i = 0; ctxs && i < count; ++i) {
    if (!ctxs[i] || ctxs[i]->device != b->device) {
      delete b;
      return ARP_EINVAL;
    }
    b->ctx.push_back(ctxs[i]);
  }
  b->capacity = count;
  const Layout L = layout_for(count);
  b->dbytes = L.total;
  if (cudaMalloc((void**)&b->dmem, b->dbytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ARP_ENOMEM;
  }
  b->host.assign(b->dbytes, 0);
  b->out.assign(count, 0.0);  // ctxs == NULL: an empty batch with room for `count` members
  *out = b;
  return ARP_OK;
}

arp_status arp_batch_reset(arp_batch* b, arp_ctx* const* ctxs, int count) {
  if (!b) return ARP_EINVAL;
  if (count < 0 || count > b->capacity || (count > 0 && !ctxs)) return bfail(b, ARP_EINVAL, "batch: bad member list");
  for (int i = 0; i < count; ++i)
    if (!ctxs[i] || ctxs[i]->device != b->device) return bfail(b, ARP_EINVAL, "batch: bad member");
  b->ctx.assign(ctxs, ctxs + count);
  b->out.assign(count > 0 ? count : 1, 0.0);
  return ARP_OK;
}

arp_status arp_batch_destroy(arp_batch* b) {
  if (!b) return ARP_OK;
  for (cudaStream_t g : b->gs) {
    cudaStreamSynchronize(g);
    cudaStreamDestroy(g);
  }
  for (cudaEvent_t e : b->ge) cudaEventDestroy(e);
  if (b->ready) cudaEventDestroy(b->ready);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
  return ARP_OK;
}

const char* arp_batch_last_error(const arp_batch* b) { return b ? b->err.c_str() : ""; }

arp_status arp_batch_iterate(arp_batch* b, void* stream, int* levels, double* changes) {
  if (!b) return ARP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = (int)b->ctx.size();
  if (n == 0) return ARP_OK;
  const Layout L = layout_for(b->capacity);
  unsigned char* H = b->host.data();
  arp_status r;
  std::vector<int> act, iter;  // indices: contexts with an initial state; those past their predictor
  for (int i = 0; i < n; ++i)
    if (b->ctx[i]->fine_scheme != 0 || b->ctx[i]->coarse_scheme != 0 || b->ctx[i]->coarse_grid != 0 ||
        dft_mode(b->ctx[i]))
      return bfail(b, ARP_EINVAL, "batch: members must use the default schemes and grid, FP64 or FP32");
  for (int i = 0; i < n; ++i) {
    arp_ctx* c = b->ctx[i];
    if (!c->have_initial) continue;
    if ((r = ensure_tables(c, s)) != ARP_OK) return bfail(b, r, c->err);
    act.push_back(i);
    if (c->level >= 0) iter.push_back(i);
  }
  for (int i : iter) std::swap(b->ctx[i]->U, b->ctx[i]->Uold);
  auto unswap = [&]() {
    for (int i : iter) std::swap(b->ctx[i]->U, b->ctx[i]->Uold);
  };

  // groups by (log2 N, precision, ARP_OPT_FINE_BLOCK): members of a group share
  // fused launches, so each gets the block size it would get on its own
  std::map<std::tuple<int, int, int>, std::vector<int>> groups;
  for (int i : act) groups[{b->ctx[i]->logN, b->ctx[i]->precision, b->ctx[i]->fine_block}].push_back(i);
  // within a group the problems with the most fine steps per slice come first, so
  // their (longest) blocks are dispatched first and do not form the launch's tail
  for (auto& g : groups)
    std::stable_sort(g.second.begin(), g.second.end(),
                     [&](int x, int y) { return b->ctx[x]->steps > b->ctx[y]->steps; });

  int* first = reinterpret_cast<int*>(H + L.first);
  int nfirst = 0;  // ints used in the prefix region
  struct Launch {
    int logN, prec;
    size_t fine_off, first_fine, corr_off, first_corr, chain_off, fin_off, first_fin;
    int nfine, fine_blocks, ncorr, corr_blocks, nchain, C, fin_blocks;
    size_t smem;
    arp_ctx* tune;              // first member with a fine sweep: sets the FP32 block size
    std::vector<int> fallback;  // contexts whose chain runs on its own
  };
  std::vector<Launch> launches;
  size_t fine_bytes = 0, chain_bytes = 0, corr_count = 0, fin_count = 0;
  for (auto& g : groups) {
    Launch l{};
    l.logN = std::get<0>(g.first);
    l.prec = std::get<1>(g.first);
    const bool f32 = (l.prec == ARP_FP32);
    // fine sweeps and corrections of the contexts past their predictor
    l.fine_off = L.fine + fine_bytes;
    l.first_fine = nfirst;
    l.corr_off = L.corr + corr_count * sizeof(CorrJob);
    for (int i : g.second) {
      arp_ctx* c = b->ctx[i];
      if (c->level < 0) continue;
      if (!l.tune) l.tune = c;
      first[nfirst + l.nfine] = l.fine_blocks;
      if (f32) {
        FineJob<float> j{c->Uold, c->Fb, c->steps, fine_tabs<float>(c)};
        memcpy(H + l.fine_off + (size_t)l.nfine * sizeof(j), &j, sizeof(j));
      } else {
        FineJob<double> j{c->Uold, c->Fb, c->steps, fine_tabs<double>(c)};
        memcpy(H + l.fine_off + (size_t)l.nfine * sizeof(j), &j, sizeof(j));
      }
      CorrJob cj{c->Fb, c->Gc, c->V, c->VT, c->Uold, c->U, c->H, c->K1, basis_tabs(c)};  // K1 = VT's modes
      memcpy(H + l.corr_off + (size_t)l.ncorr * sizeof(CorrJob), &cj, sizeof(cj));
      l.fine_blocks += c->slices;
      ++l.nfine;
      ++l.ncorr;
    }
    l.corr_blocks = l.fine_blocks;
    first[nfirst + l.nfine] = l.fine_blocks;
    l.first_corr = l.first_fine;  // same per-problem slice counts
    nfirst += l.nfine + 1;
    fine_bytes += (size_t)l.nfine * (f32 ? sizeof(FineJob<float>) : sizeof(FineJob<double>));
    corr_count += l.ncorr;
    // chains of every context in the group, in one cluster launch if all fit
    std::vector<int> M, K1;
    for (int i : g.second) {
      M.push_back(b->ctx[i]->M);
      K1.push_back(b->ctx[i]->K1);
    }
    std::vector<ClusterPlan> plans(g.second.size());
    arp_status pr = ARP_EINVAL;
    bool forced = false;
    // a member whose chain might not run the batched cluster on its own runs it on its own
    // here too (FP64 in automatic mode takes the cooperative grid above 16 nodes, and runs
    // its own chain choice in any case), so batched = solo bit for bit
    for (int i : g.second) {
      const arp_ctx* c = b->ctx[i];
      forced |= (c->chain_mode == 1 || c->chain_mode == 2 || c->skip_arrival ||
                 (c->chain_mode == 0 && c->precision == ARP_FP64));
    }
    if (!forced)
      pr = f32 ? plan_chain_batch_f32(l.logN, M.data(), K1.data(), (int)M.size(), &l.C, plans.data(), &l.smem)
               : plan_chain_batch_f64(l.logN, M.data(), K1.data(), (int)M.size(), &l.C, plans.data(), &l.smem);
    l.chain_off = L.chain + chain_bytes;
    l.fin_off = L.fin + fin_count * sizeof(FinishJob);
    l.first_fin = nfirst;
    if (pr == ARP_OK) {
      for (size_t t = 0; t < g.second.size(); ++t) {
        arp_ctx* c = b->ctx[g.second[t]];
        const ClusterPlan& p = plans[t];
        ClusterChainArgs a{c->level >= 0 ? c->VT : nullptr, c->U, c->Ge, c->slices, c->M, p.q, p.own, p.ph_smem,
                           p.tmp_smem, c->dT, c->inv_sig64, c->sk_sig64, c->dhalf, c->gphase};
        a.status = reinterpret_cast<unsigned*>(b->dmem + L.status) + g.second[t];
        FinishJob fj{c->Ge, c->level >= 0 ? c->V : nullptr, c->U, c->Gc, c->H, c->K1, basis_tabs(c)};
        memcpy(H + l.fin_off + t * sizeof(FinishJob), &fj, sizeof(fj));
        first[nfirst + t] = l.fin_blocks;
        l.fin_blocks += c->slices;
        if (f32) {
          ChainJob<float> j{a, nbar_tabs<float>(c)};
          memcpy(H + l.chain_off + t * sizeof(j), &j, sizeof(j));
        } else {
          ChainJob<double> j{a, nbar_tabs<double>(c)};
          memcpy(H + l.chain_off + t * sizeof(j), &j, sizeof(j));
        }
      }
      l.nchain = (int)g.second.size();
      first[nfirst + l.nchain] = l.fin_blocks;
      nfirst += l.nchain + 1;
      fin_count += l.nchain;
      chain_bytes += (size_t)l.nchain * (f32 ? sizeof(ChainJob<float>) : sizeof(ChainJob<double>));
    } else {
      l.fallback = g.second;
    }
    launches.push_back(std::move(l));
  }
  // norms of every context past its predictor (any group)
  NormJob* nj = reinterpret_cast<NormJob*>(H + L.norm);
  const int first_norm = nfirst;
  int norm_blocks = 0;
  for (size_t t = 0; t < iter.size(); ++t) {
    arp_ctx* c = b->ctx[iter[t]];
    nj[t] = NormJob{c->U, c->Uold, c->rel, c->H, c->slices};
    first[nfirst + t] = norm_blocks;
    norm_blocks += c->slices;
  }
  first[nfirst + iter.size()] = norm_blocks;
  nfirst += (int)iter.size() + 1;

  if ((r = check_cuda(b->ctx[0], cudaMemcpyAsync(b->dmem, H, L.total, cudaMemcpyHostToDevice, s), "batch: jobs")) !=
      ARP_OK) {
    unswap();
    return bfail(b, r, b->ctx[0]->err);
  }
  int* dfirst = reinterpret_cast<int*>(b->dmem + L.first);
  arp_ctx* ec = b->ctx[0];  // carries launch error messages
  // each group on a stream of its own after the upload (groups are independent
  // problems), the one with the most fine work first
  std::vector<size_t> order(launches.size());
  std::vector<double> work(launches.size(), 0.0);
  for (size_t li = 0; li < launches.size(); ++li) {
    order[li] = li;
    work[li] = (double)launches[li].fine_blocks * (1 << launches[li].logN) * launches[li].logN;
  }
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work[x] > work[y]; });
  while (b->gs.size() < launches.size()) {
    cudaStream_t g = nullptr;
    cudaEvent_t e = nullptr;
    if ((r = check_cuda(ec, cudaStreamCreateWithFlags(&g, cudaStreamNonBlocking), "batch: stream")) != ARP_OK ||
        (r = check_cuda(ec, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch: event")) != ARP_OK) {
      if (g) cudaStreamDestroy(g);
      unswap();
      return bfail(b, r, ec->err);
    }
    b->gs.push_back(g);
    b->ge.push_back(e);
  }
  if (!b->ready && (r = check_cuda(ec, cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming), "batch: event")) !=
                       ARP_OK) {
    unswap();
    return bfail(b, r, ec->err);
  }
  if ((r = check_cuda(ec, cudaEventRecord(b->ready, s), "batch: fork")) != ARP_OK) {
    unswap();
    return bfail(b, r, ec->err);
  }
  size_t forked = 0;
  for (size_t oi = 0; oi < order.size(); ++oi) {
    auto& l = launches[order[oi]];
    const bool f32 = (l.prec == ARP_FP32);
    const cudaStream_t gstream = b->gs[oi];
    if ((r = check_cuda(ec, cudaStreamWaitEvent(gstream, b->ready, 0), "batch: fork")) != ARP_OK) break;
    forked = oi + 1;
    cudaStream_t s = gstream;  // this group's work goes on its own stream
    if (l.nfine > 0) {
      r = f32 ? launch_fine_batch_f32(ec, l.tune, l.logN, b->dmem + l.fine_off, dfirst + l.first_fine, l.nfine, l.fine_blocks, s)
              : launch_fine_batch_f64(ec, l.tune, l.logN, b->dmem + l.fine_off, dfirst + l.first_fine, l.nfine, l.fine_blocks, s);
      if (r != ARP_OK) break;
      corr_batch_kernel<<<l.corr_blocks, 256, 0, s>>>(reinterpret_cast<const CorrJob*>(b->dmem + l.corr_off),
                                                      dfirst + l.first_corr, l.ncorr);
      if ((r = check_cuda(ec, cudaGetLastError(), "batch: correction")) != ARP_OK) break;
    }
    if (l.nchain > 0) {
      r = f32 ? launch_chain_batch_f32(ec, l.logN, b->dmem + l.chain_off, l.nchain, l.C, l.smem, s)
              : launch_chain_batch_f64(ec, l.logN, b->dmem + l.chain_off, l.nchain, l.C, l.smem, s);
      if (r != ARP_OK) break;
      finish_batch_kernel<<<l.fin_blocks, 256, 0, s>>>(reinterpret_cast<const FinishJob*>(b->dmem + l.fin_off),
                                                       dfirst + l.first_fin, l.nchain);
      if ((r = check_cuda(ec, cudaGetLastError(), "batch: finish")) != ARP_OK) break;
    }
    for (int i : l.fallback) {
      arp_ctx* c = b->ctx[i];
      if ((r = run_chain(c, c->level >= 0 ? c->V : nullptr, s)) != ARP_OK) break;
    }
    if (r != ARP_OK) break;
  }
  // join: the caller's stream waits for every group that was forked
  for (size_t oi = 0; oi < forked; ++oi) {
    const arp_status q = check_cuda(ec, cudaEventRecord(b->ge[oi], b->gs[oi]), "batch: join");
    const arp_status q2 = q == ARP_OK ? check_cuda(ec, cudaStreamWaitEvent(s, b->ge[oi], 0), "batch: join") : q;
    if (r == ARP_OK) r = q2;
  }
  if (r == ARP_OK && !iter.empty()) {
    norm_batch_kernel<<<norm_blocks, 256, 0, s>>>(reinterpret_cast<const NormJob*>(b->dmem + L.norm),
                                                  dfirst + first_norm, (int)iter.size());
    max_batch_kernel<<<(int)iter.size(), 256, 0, s>>>(reinterpret_cast<const NormJob*>(b->dmem + L.norm),
                                                      reinterpret_cast<double*>(b->dmem + L.out));
    r = check_cuda(ec, cudaGetLastError(), "batch: norm");
  }
  if (r == ARP_OK && !iter.empty())
    r = check_cuda(ec, cudaMemcpyAsync(b->out.data(), b->dmem + L.out, iter.size() * sizeof(double),
                                       cudaMemcpyDeviceToHost, s), "batch: norm read");
  // status words: of the batched chains (bounded waits), and of contexts whose chain ran on its own
  std::vector<unsigned> status(n, 0u);
  if (r == ARP_OK)
    r = check_cuda(ec, cudaMemcpyAsync(status.data(), b->dmem + L.status, n * sizeof(unsigned),
                                       cudaMemcpyDeviceToHost, s), "batch: status read");
  if (r == ARP_OK)
    for (auto& l : launches)
      for (int i : l.fallback)
        if (r == ARP_OK)
          r = check_cuda(ec, cudaMemcpyAsync(&status[i], b->ctx[i]->sync + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                             s), "batch: status read");
  if (r == ARP_OK) r = check_cuda(ec, cudaStreamSynchronize(s), "batch: synchronise");
  if (r != ARP_OK) {
    unswap();
    return bfail(b, r, ec->err);
  }
  arp_status first_err = ARP_OK;
  std::vector<char> is_iter(n, 0);
  for (int i : iter) is_iter[i] = 1;
  size_t t_iter = 0;
  for (int i = 0; i < n; ++i) {
    arp_ctx* c = b->ctx[i];
    double ch = NAN;
    if (!c->have_initial) {
      if (levels) levels[i] = c->level;
      if (changes) changes[i] = ch;
      continue;
    }
    if (status[i] != 0u) {
      if (is_iter[i]) std::swap(c->U, c->Uold);
      if (is_iter[i]) ++t_iter;
      c->err = "chain: a bounded wait timed out (a block's arrival or data never came)";
      if (first_err == ARP_OK) first_err = ARP_ETIMEOUT;
    } else if (is_iter[i]) {
      ch = b->out[t_iter++];
      c->level += 1;
      if (!std::isfinite(ch) && first_err == ARP_OK) first_err = ARP_ENONFINITE;
    } else {
      c->level = 0;
      ch = INFINITY;
    }
    if (levels) levels[i] = c->level;
    if (changes) changes[i] = ch;
  }
  if (first_err != ARP_OK) b->err = "a problem of the batch failed (see its context's last error)";
  return first_err;
}

}  // extern "C"
