// batch.cu -- sea_apply_vxx_batch: several independent configurations in
// one pass (Sec. II B applied to each; pairs of different configurations
// never interact, so their Poisson problems share one persistent launch).
//
// Per call: every configuration's plan (boxes, pairs, entries) is built on
// the shared stream; one readback sizes the per-pair buffers; then the
// post-plan phase -- pair moments and boundary values of every
// configuration, one persistent CG launch over all pairs of all
// configurations, far field and accumulation of every configuration -- is
// captured once into a CUDA graph and replayed on later calls whose plan
// sizes and buffers are unchanged (a changed plan re-captures).
//
// Autotuner: the persistent CG launch has two free choices that leave every
// pair's arithmetic unchanged (so the results stay bit-identical to one call
// per configuration): the order in which the pairs of all configurations
// are dealt to the CTAs, and the persistent grid (CTAs per SM, up to the
// occupancy limit).  The first call for a workload (the configurations'
// pair counts, unknowns, grids and forms) times every order with every grid
// size on the batch itself, one CG launch each after a warm-up launch, and
// keeps the fastest in a process-wide table; later calls for the same
// workload -- and the graph captured for it -- use that choice.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "sea_internal.cuh"

namespace {

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> sig;
  long long launches = 0;
  int device = -1;
};

// One cache per (first context) -- kept in the first context's slot table.
GraphCache* cache_of(sea_ctx* c0) {
  if (!c0->batch_cache) c0->batch_cache = new GraphCache();
  return (GraphCache*)c0->batch_cache;
}

void push_buf(std::vector<long long>& v, const SeaBuf& b) {
  v.push_back((long long)(uintptr_t)b.p);
  v.push_back((long long)b.bytes);
}

// Orders of the batched CG's work items (configuration, rank), rank r being
// a configuration's r-th longest pair: 0 ranks dealt round-robin over the
// configurations; 1 all pairs by box size, longest first (ties: rank, then
// configuration); 2 configuration after configuration.
constexpr int N_ORDERS = 3;

struct Tuned {
  int order = 0, per_sm_mixed = 0, per_sm_fp64 = 0;
  double ms = 0.0;  // the chosen candidate's CG time
};
std::mutex g_tune_mutex;
std::map<std::vector<long long>, Tuned> g_tuned;

// Work items in `order`, the mixed-form items first, then the FP64 ones.
// size[k][r]: box size of configuration k's rank-r pair (order 1 only).
void build_items(int order, sea_ctx* const* ctxs, int n, int maxP,
                 const std::vector<std::vector<int>>& size, std::vector<int2>& items) {
  items.clear();
  for (int mixed = 1; mixed >= 0; --mixed) {
    auto form = [&](int k) { return (ctxs[k]->prm.precision == 1) == (mixed == 1); };
    const size_t first = items.size();
    if (order == 2) {
      for (int k = 0; k < n; ++k)
        if (form(k))
          for (int r = 0; r < ctxs[k]->P; ++r) items.push_back(make_int2(k, r));
    } else {
      for (int r = 0; r < maxP; ++r)
        for (int k = 0; k < n; ++k)
          if (r < ctxs[k]->P && form(k)) items.push_back(make_int2(k, r));
      if (order == 1)
        std::stable_sort(items.begin() + first, items.end(), [&](const int2& a, const int2& b) {
          return size[a.x][a.y] > size[b.x][b.y];
        });
    }
  }
}

}  // namespace

void sea_batch_cache_free(sea_ctx* c) {
  GraphCache* g = (GraphCache*)c->batch_cache;
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  c->batch_cache = nullptr;
}

#define SEA_BCK(call, msg)                                                      \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      char b_[256];                                                             \
      snprintf(b_, sizeof(b_), "%s: %s", msg, cudaGetErrorString(e_));         \
      for (int k_ = 0; k_ < n; ++k_) sea_fail(ctxs[k_], SEA_ERR_CUDA, b_);      \
      return SEA_ERR_CUDA;                                                      \
    }                                                                           \
  } while (0)

extern "C" sea_status sea_apply_vxx_batch(sea_ctx* const* ctxs, int n, double* const* outs,
                                          int on_device, double* exx) {
  if (!ctxs || n < 1 || !outs) return SEA_ERR_ARG;
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k] || !outs[k]) return SEA_ERR_ARG;
    if (ctxs[k]->poisoned) return sea_fail(ctxs[k], SEA_ERR_STATE, "context poisoned");
    if (!ctxs[k]->have_phi) return sea_fail(ctxs[k], SEA_ERR_STATE, "sea_set_orbitals first");
    if (ctxs[k]->stream != ctxs[0]->stream || ctxs[k]->device != ctxs[0]->device)
      return sea_fail(ctxs[k], SEA_ERR_ARG, "batched contexts must share device and stream");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return sea_fail(ctxs[k], SEA_ERR_ARG, "a context appears twice");
  }
  sea_ctx* c0 = ctxs[0];
  cudaStream_t st = c0->stream;
  sea::Trace tr("sea_apply_vxx_batch");
  tr.stage("plans");
  // plans
  for (int k = 0; k < n; ++k) {
    sea_ctx* c = ctxs[k];
    c->have_vxx = c->have_ace = false;
    c->far_side = false;  // the accumulation forms every contribution itself
    SEA_BCK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), st), "memset");
    SEA_BCK(sea::launch_plan_boxes(c), "domain boxes");
    SEA_BCK(sea::launch_plan_pairs(c), "pair selection");
    SEA_BCK(sea::launch_entries(c), "accumulation entries");
  }
  std::vector<int> hc((size_t)n * 16);
  for (int k = 0; k < n; ++k)
    SEA_BCK(cudaMemcpyAsync(&hc[(size_t)k * 16], ctxs[k]->counts.p, 16 * sizeof(int),
                            cudaMemcpyDeviceToHost, st),
            "counts");
  SEA_BCK(cudaStreamSynchronize(st), "plan");
  long long total = 0;
  int maxP = 0;
  for (int k = 0; k < n; ++k) {
    sea_ctx* c = ctxs[k];
    const int* h = &hc[(size_t)k * 16];
    c->Pproto = h[0];
    c->P = h[1];
    c->E = h[2];
    memcpy(&c->U, h + 4, sizeof(long long));
    memcpy(&c->WC, h + 6, sizeof(long long));
    memcpy(&c->max_window, h + 8, sizeof(long long));
    c->cg_pad_max = h[10];
    const size_t U = (size_t)(c->U > 1 ? c->U : 1);
    const size_t P = (size_t)(c->P > 1 ? c->P : 1);
    if (!sea_ensure(c, c->vbuf, U * sizeof(double)) || !sea_ensure(c, c->bbuf, U * sizeof(double)) ||
        !sea_ensure(c, c->rbuf, U * sizeof(double)) || !sea_ensure(c, c->pbuf, U * sizeof(double)) ||
        !sea_ensure(c, c->qbuf, U * sizeof(double)) ||
        !sea_ensure(c, c->cbuf, (size_t)(c->WC > 1 ? c->WC : 1) * sizeof(double)) ||
        !sea_ensure(c, c->Q, P * SEA_QSTRIDE * sizeof(double)) ||
        !sea_ensure(c, c->gbuf, 36 * U * sizeof(double)) ||
        !sea_ensure(c, c->epair, P * sizeof(double)) || !sea_ensure(c, c->iters, P * sizeof(int)))
      return sea_fail(c, SEA_ERR_OOM, "device allocation failed: batch buffers");
    total += c->P;
    maxP = c->P > maxP ? c->P : maxP;
  }
  // descriptors and items (longest-first ranks dealt round-robin)
  const size_t db = sea::batch_desc_bytes();
  std::vector<unsigned char> hdesc((size_t)n * db);
  int pad_cap = 0;
  for (int k = 0; k < n; ++k) {
    pad_cap = std::max(pad_cap, sea::cg_pad_cap(ctxs[k]));
    ctxs[k]->cg_warm = false;  // the batched form solves from zero
    sea::make_batch_desc(ctxs[k], &hdesc[(size_t)k * db]);
  }
  // the workload's tuned choice (absent: tune below, before the capture)
  std::vector<long long> wsig;
  wsig.push_back(n);
  for (int k = 0; k < n; ++k) {
    const sea_ctx* c = ctxs[k];
    wsig.push_back(c->P);
    wsig.push_back(c->U);
    wsig.push_back(c->cg_pad_max);
    wsig.push_back(c->prm.precision);
    for (int a = 0; a < 3; ++a) wsig.push_back(c->N[a]);
  }
  Tuned tuned;
  bool have_tuned = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(wsig);
    if (it != g_tuned.end()) {
      tuned = it->second;
      have_tuned = true;
    }
  }
  // box sizes per rank (the pairs' ranks are longest first in each
  // configuration): needed by order 1 and by the tuning
  std::vector<std::vector<int>> rsize((size_t)n);
  if (!have_tuned || tuned.order == 1) {
    std::vector<std::vector<int>> ord((size_t)n), psz((size_t)n);
    for (int k = 0; k < n; ++k) {
      sea_ctx* c = ctxs[k];
      ord[k].resize((size_t)c->P);
      psz[k].resize((size_t)c->P);
      if (c->P) {
        SEA_BCK(cudaMemcpyAsync(ord[k].data(), c->order.p, (size_t)c->P * sizeof(int),
                                cudaMemcpyDeviceToHost, st),
                "pair order");
        SEA_BCK(cudaMemcpyAsync(psz[k].data(), c->psize.p, (size_t)c->P * sizeof(int),
                                cudaMemcpyDeviceToHost, st),
                "pair sizes");
      }
    }
    SEA_BCK(cudaStreamSynchronize(st), "pair sizes");
    for (int k = 0; k < n; ++k) {
      rsize[k].resize(ord[k].size());
      for (size_t r = 0; r < ord[k].size(); ++r) rsize[k][r] = psz[k][(size_t)ord[k][r]];
    }
  }
  std::vector<int2> hitems;
  hitems.reserve((size_t)total);
  build_items(have_tuned ? tuned.order : 0, ctxs, n, maxP, rsize, hitems);
  long long total_mixed = 0;
  for (int k = 0; k < n; ++k)
    if (ctxs[k]->prm.precision == 1) total_mixed += ctxs[k]->P;
  if (!sea_ensure(c0, c0->bdesc, (size_t)n * db) ||
      !sea_ensure(c0, c0->bitems, (size_t)(total > 1 ? total : 1) * sizeof(int2)))
    return sea_fail(c0, SEA_ERR_OOM, "device allocation failed: batch descriptors");
  SEA_BCK(cudaMemcpyAsync(c0->bdesc.p, hdesc.data(), hdesc.size(), cudaMemcpyHostToDevice, st),
          "descriptors");
  if (total)
    SEA_BCK(cudaMemcpyAsync(c0->bitems.p, hitems.data(), hitems.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, st),
            "items");

  // signature of everything the captured launches depend on
  std::vector<long long> sig;
  sig.push_back(n);
  sig.push_back(on_device);
  sig.push_back(total);
  push_buf(sig, c0->bdesc);
  push_buf(sig, c0->bitems);
  for (int k = 0; k < n; ++k) {
    sea_ctx* c = ctxs[k];
    sig.push_back((long long)(uintptr_t)c);
    sig.push_back(c->P);
    sig.push_back(c->E);
    sig.push_back(c->U);
    sig.push_back(c->WC);
    sig.push_back(c->max_window);
    sig.push_back(c->cg_pad_max);
    sig.push_back(c->prm.precision);
    sig.push_back((long long)(uintptr_t)outs[k]);
    const SeaBuf* bufs[] = {&c->phi, &c->vxx_dev, &c->pinfo, &c->voff, &c->order, &c->Q,
                            &c->epair, &c->iters, &c->vbuf, &c->bbuf, &c->rbuf, &c->pbuf,
                            &c->qbuf, &c->eptr, &c->ewin, &c->coff, &c->cbuf, &c->status,
                            &c->exx_dev, &c->queue, &c->counts};
    for (const SeaBuf* b : bufs) push_buf(sig, *b);
  }
  GraphCache* gc = cache_of(c0);
  const bool can_graph = st != nullptr;  // the legacy stream cannot be captured
  auto post_plan = [&]() -> cudaError_t {
    long long l0 = 0;
    for (int k = 0; k < n; ++k) l0 += ctxs[k]->launches;
    for (int k = 0; k < n; ++k) {
      cudaError_t e = sea::launch_pair_setup(ctxs[k]);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = sea::launch_cg_batch(st, c0->device, c0->bdesc.p, (const int2*)c0->bitems.p,
                                         (int)total_mixed, (int*)c0->queue.p, pad_cap, true,
                                         tuned.per_sm_mixed);
    if (e != cudaSuccess) return e;
    e = sea::launch_cg_batch(st, c0->device, c0->bdesc.p,
                             (const int2*)c0->bitems.p + total_mixed, (int)(total - total_mixed),
                             (int*)c0->queue.p, 0, false, tuned.per_sm_fp64);
    if (e != cudaSuccess) return e;
    c0->launches += (total_mixed > 0) + (total > total_mixed);
    for (int k = 0; k < n; ++k) {
      e = sea::launch_accumulate(ctxs[k], (double*)ctxs[k]->vxx_dev.p,
                                 on_device ? outs[k] : nullptr);
      if (e != cudaSuccess) return e;
    }
    long long l1 = 0;
    for (int k = 0; k < n; ++k) l1 += ctxs[k]->launches;
    gc->launches = l1 - l0;
    return cudaSuccess;
  };
  c0->stats.batch_tune_ms = 0.0;
  if (!have_tuned && total > 0) {
    tr.stage("autotuning");
    // every order x every grid size, one timed CG launch each (after one
    // warm-up launch), on the batch's own pairs; the pair setup runs once
    float t_tune = 0.f;
    cudaEvent_t ev[3];
    for (int q = 0; q < 3; ++q) SEA_BCK(cudaEventCreate(&ev[q]), "event");
    SEA_BCK(cudaEventRecord(ev[2], st), "event");
    for (int k = 0; k < n; ++k) SEA_BCK(sea::launch_pair_setup(ctxs[k]), "pair setup (tuning)");
    const int occ_m = sea::cg_batch_max_ctas_per_sm(c0->device, pad_cap, true);
    const int occ_f = sea::cg_batch_max_ctas_per_sm(c0->device, 0, false);
    double best = 1e300;
    std::vector<int2> items;
    for (int o = 0; o < N_ORDERS; ++o) {
      build_items(o, ctxs, n, maxP, rsize, items);
      SEA_BCK(cudaMemcpyAsync(c0->bitems.p, items.data(), items.size() * sizeof(int2),
                              cudaMemcpyHostToDevice, st),
              "items");
      double best_m = 1e300, best_f = 1e300;
      int pm = 1, pf = 1;
      for (int form = 0; form < 2; ++form) {
        const bool mixed = form == 0;
        const long long cnt = mixed ? total_mixed : total - total_mixed;
        if (cnt == 0) continue;
        const int2* it0 = (const int2*)c0->bitems.p + (mixed ? 0 : total_mixed);
        const int occ = mixed ? occ_m : occ_f;
        for (int j = (o == 0 ? 0 : 1); j <= occ; ++j) {  // j = 0: the warm-up launch
          SEA_BCK(cudaEventRecord(ev[0], st), "event");
          SEA_BCK(sea::launch_cg_batch(st, c0->device, c0->bdesc.p, it0, (int)cnt,
                                       (int*)c0->queue.p, mixed ? pad_cap : 0, mixed, j < 1 ? 1 : j),
                  "batched CG (tuning)");
          SEA_BCK(cudaEventRecord(ev[1], st), "event");
          SEA_BCK(cudaEventSynchronize(ev[1]), "tuning");
          float ms = 0.f;
          cudaEventElapsedTime(&ms, ev[0], ev[1]);
          if (j == 0) continue;
          if (mixed && ms < best_m) best_m = ms, pm = j;
          if (!mixed && ms < best_f) best_f = ms, pf = j;
        }
      }
      const double tot = (best_m < 1e300 ? best_m : 0.0) + (best_f < 1e300 ? best_f : 0.0);
      if (tot < best) {
        best = tot;
        tuned.order = o;
        tuned.per_sm_mixed = pm;
        tuned.per_sm_fp64 = pf;
        tuned.ms = tot;
      }
    }
    SEA_BCK(cudaEventRecord(ev[1], st), "event");
    SEA_BCK(cudaEventSynchronize(ev[1]), "tuning");
    cudaEventElapsedTime(&t_tune, ev[2], ev[1]);
    for (int q = 0; q < 3; ++q) cudaEventDestroy(ev[q]);
    c0->stats.batch_tune_ms = t_tune;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tuned[wsig] = tuned;
    }
    // the chosen order's items for the launches below
    build_items(tuned.order, ctxs, n, maxP, rsize, hitems);
    SEA_BCK(cudaMemcpyAsync(c0->bitems.p, hitems.data(), hitems.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, st),
            "items");
  }
  tr.stage("post-plan phase");
  c0->stats.batch_order = tuned.order;
  c0->stats.batch_ctas_per_sm = tuned.per_sm_mixed;
  c0->stats.batch_ctas_per_sm_fp64 = tuned.per_sm_fp64;
  if (!can_graph) {
    SEA_BCK(post_plan(), "batched post-plan phase");
    c0->stats.batch_graph = 0;
  } else if (gc->exec && gc->sig == sig && gc->device == c0->device) {
    SEA_BCK(cudaGraphLaunch(gc->exec, st), "graph launch");
    c0->launches += gc->launches;
    c0->stats.batch_graph = 2;  // replayed
  } else {
    if (gc->exec) {
      cudaGraphExecDestroy(gc->exec);
      gc->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    SEA_BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = post_plan();
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    SEA_BCK(e, "batched post-plan phase (capture)");
    SEA_BCK(e2, "end capture");
    e = cudaGraphInstantiate(&gc->exec, g, 0);
    cudaGraphDestroy(g);
    SEA_BCK(e, "graph instantiate");
    gc->sig = sig;
    gc->device = c0->device;
    SEA_BCK(cudaGraphLaunch(gc->exec, st), "graph launch");
    c0->stats.batch_graph = 1;  // captured
  }
  struct R {
    double res[5];
    unsigned st;
  };
  std::vector<R> r((size_t)n);
  for (int k = 0; k < n; ++k) {
    sea_ctx* c = ctxs[k];
    if (!on_device)
      SEA_BCK(cudaMemcpyAsync(outs[k], c->vxx_dev.p, (size_t)c->n_orb * c->ng * sizeof(double),
                              cudaMemcpyDeviceToHost, st),
              "copy V_xx phi");
    SEA_BCK(cudaMemcpyAsync(r[k].res, c->exx_dev.p, sizeof(r[k].res), cudaMemcpyDeviceToHost, st),
            "exx");
    SEA_BCK(cudaMemcpyAsync(&r[k].st, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
            "status");
  }
  SEA_BCK(cudaStreamSynchronize(st), "apply_vxx_batch");
  sea_status rs = SEA_OK;
  for (int k = 0; k < n; ++k) {
    sea_ctx* c = ctxs[k];
    c->stats.n_pairs = c->P;
    c->stats.n_proto_pairs = c->Pproto;
    c->stats.n_unknowns = c->U;
    c->stats.n_window_points = c->WC;
    c->stats.exx = r[k].res[0];
    c->stats.cg_unknown_iters = (long long)r[k].res[1];
    c->stats.cg_iters_min = (int)r[k].res[2];
    c->stats.cg_iters_max = (int)r[k].res[3];
    c->stats.cg_iters_mean = r[k].res[4];
    if (exx) exx[k] = r[k].res[0];
    c->w_dense = false;
    c->have_vxx = true;
    c->lists_ready = false;  // the batch forms no ACE tile lists
    if (r[k].st & SEA_FLAG_CG_CAP) {
      sea_fail(c, SEA_ERR_CG_NOT_CONVERGED, "a pair's CG reached cg_max_iter");
      rs = SEA_ERR_CG_NOT_CONVERGED;
    }
  }
  return rs;
}
