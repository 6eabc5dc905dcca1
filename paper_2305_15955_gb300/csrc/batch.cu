// Batched CD-WAC over many systems of uneven size (the C ABI's cdwac_batch_run).
//
// Systems are assigned to lanes, largest first (longest-processing-time rule on an N_aux^2 N_ov + N_aux^3 cost
// estimate); a lane is a stream with its own context (own scratch, own LDL^T side stream) sharing the parent's
// device status word.  The caller's stream forks to the lanes through one event and joins them back, so the
// whole batch is one stream-ordered unit that can be captured into a CUDA graph: with CDWAC_BATCH_GRAPH the first
// call runs eagerly (sizing every lane's scratch), captures the same sequence, and later calls with identical
// items replay the graph.  The autotuner times, per size bucket, lane counts and the lookahead switch, then the tile
// configuration of the tensor-core kernels: the Pi output tile width (128 x 128 or 128 x 256), its tile-group size
// (the rasterisation of the output tiles over the waves) and the number of CTA waves the real trailing update's
// row strips are cut into (the number of 128 x 32 tiles each CTA streams against its resident W digits).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

struct Config {
  int lanes;
  int lookahead;
  int pi_group;    // Pi tile-group size (cdwac_ctx::pi_group)
  int pi_tile;     // Pi output tile width, 128 or 256 (cdwac_ctx::pi_tile)
  int upd_waves;   // real trailing update: CTA waves of row-strip chunks (cdwac_ctx::upd_waves)
};

double item_cost(const cdwac_batch_item& it, const cdwac_params* p) {
  const double n = it.sys.n_aux, nov = (double)it.sys.n_occ * (it.sys.n_basis - it.sys.n_occ);
  const double pts = p->n_imag + 2.0 * p->n_real;
  return pts * (n * n * nov / 500.0 + n * n * n);   // tensor-core contraction (fast) + FP64 factorisation
}

cdwac_status make_lane(cdwac_ctx* parent, cdwac_ctx** out) {
  cdwac_ctx* l = new cdwac_ctx();
  l->is_lane = true;
  l->device = parent->device;
  l->num_sms = parent->num_sms;
  l->d_status = parent->d_status;
  l->h_status = parent->h_status;
  l->lookahead = parent->lookahead;
  if (!create_factor_streams(l)) {
    cdwac_destroy(l);
    return set_error(parent, CDWAC_ERR_CUDA, "lane creation failed");
  }
  l->freq_lanes = 1;
  *out = l;
  return CDWAC_OK;
}

}  // namespace

cdwac_status ensure_lanes(cdwac_ctx* ctx, int n) {
  if (!ctx->ev_fork) CDWAC_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  while ((int)ctx->lanes.size() < n) {
    cdwac_ctx* l = nullptr;
    cdwac_status rc = make_lane(ctx, &l);
    if (rc) return rc;
    cudaStream_t s;
    cudaEvent_t e;
    CDWAC_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    CDWAC_CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->lanes.push_back(l);
    ctx->lane_streams.push_back(s);
    ctx->lane_events.push_back(e);
  }
  return CDWAC_OK;
}

namespace {

cdwac_status run_item(cdwac_ctx* lane, const cdwac_batch_item& it, const cdwac_params* prm, double tol, int max_iter,
                      cudaStream_t s) {
  cdwac_status rc;
  if ((rc = cdwac_build_W_imag(lane, &it.sys, prm, it.xi, it.wxi, it.W_imag, s))) return rc;
  if ((rc = cdwac_fit_pade(lane, &it.sys, prm, it.xi, it.W_imag, it.z_real, it.W_real, &it.pade, s))) return rc;
  if (it.n_omega > 0 && it.omega && it.sigma &&
      (rc = cdwac_sigma(lane, &it.sys, prm, it.xi, it.wxi, it.W_imag, &it.pade, it.omega, it.n_omega, it.sigma, s)))
    return rc;
  if (it.qp_grid && it.n_grid >= 2 && it.e_qp)
    rc = cdwac_qp_solve(lane, &it.sys, prm, it.xi, it.wxi, it.W_imag, &it.pade, it.shift, it.qp_grid, it.n_grid, tol,
                        max_iter, it.e_qp, it.Z, it.iters, it.qp_status, s);
  return rc;
}

// Enqueue the batch on `stream` with the given configuration (fork to lanes, run, join).
cdwac_status enqueue(cdwac_ctx* ctx, const cdwac_batch_item* items, int n_items, const cdwac_params* prm,
                     double tol, int max_iter, Config cfg, cudaStream_t stream) {
  cdwac_status rc = ensure_lanes(ctx, cfg.lanes);
  if (rc) return rc;
  std::vector<int> order(n_items);
  for (int i = 0; i < n_items; ++i) order[i] = i;
  std::vector<double> cost(n_items);
  for (int i = 0; i < n_items; ++i) cost[i] = item_cost(items[i], prm);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> lane_items(cfg.lanes);
  std::vector<double> load(cfg.lanes, 0.0);
  for (int i : order) {
    int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane_items[best].push_back(i);
    load[best] += cost[i];
  }
  CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, stream));
  for (int l = 0; l < cfg.lanes; ++l) {
    if (lane_items[l].empty()) continue;
    cdwac_ctx* lane = ctx->lanes[l];
    lane->side_stream = cfg.lookahead ? lane->own_side : nullptr;
    lane->pi_group = cfg.pi_group;
    lane->pi_tile = cfg.pi_tile;
    lane->upd_waves = cfg.upd_waves;
    lane->prof = 0;
    cudaStream_t s = ctx->lane_streams[l];
    CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->ev_fork, 0));
    for (int i : lane_items[l]) {
      rc = run_item(lane, items[i], prm, tol, max_iter, s);
      if (rc) return set_error(ctx, rc, "batch item %d: %s", i, lane->last_error.c_str());
    }
    CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->lane_events[l], s));
    CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(stream, ctx->lane_events[l], 0));
  }
  return CDWAC_OK;
}

std::string batch_key(cdwac_ctx* ctx, const cdwac_batch_item* items, int n_items, const cdwac_params* prm, double tol,
                      int max_iter, Config cfg) {
  std::string k;
  for (auto* l : ctx->lanes) k.append(reinterpret_cast<const char*>(&l->scratch_gen), sizeof(l->scratch_gen));
  k.append(reinterpret_cast<const char*>(items), sizeof(cdwac_batch_item) * (size_t)n_items);
  k.append(reinterpret_cast<const char*>(prm), sizeof(cdwac_params));
  k.append(reinterpret_cast<const char*>(&tol), sizeof(tol));
  k.append(reinterpret_cast<const char*>(&max_iter), sizeof(max_iter));
  k.append(reinterpret_cast<const char*>(&cfg), sizeof(cfg));
  return k;
}

std::string bucket_of(const cdwac_batch_item* items, int n_items, const cdwac_params* prm) {
  double total = 0;
  int nmax = 0;
  for (int i = 0; i < n_items; ++i) {
    total += item_cost(items[i], prm);
    nmax = std::max(nmax, items[i].sys.n_aux);
  }
  char buf[128];
  snprintf(buf, sizeof(buf), "t3_n%d_c%d_a%d_p%d", n_items, (int)std::floor(std::log2(total + 1.0)),
           (int)std::floor(std::log2((double)nmax + 1.0)), prm->precision);
  return buf;
}

bool cache_lookup(const std::string& bucket, int max_lanes, Config* cfg) {
  const char* path = getenv("CDWAC_TUNE_CACHE");
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char b[128];
  int lanes, la, pg, pt, uw;
  double ms;
  bool found = false;
  while (fscanf(f, "%127s %d %d %d %d %d %lf", b, &lanes, &la, &pg, &pt, &uw, &ms) == 7)
    if (bucket == b && lanes <= max_lanes && pg >= 1 && pg <= 64 && (pt == 128 || pt == 256) && uw >= 1 && uw <= 8) {
      *cfg = {lanes, la, pg, pt, uw};
      found = true;
    }
  fclose(f);
  return found;
}

void cache_store(const std::string& bucket, Config cfg, double ms) {
  const char* path = getenv("CDWAC_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d %.3f\n", bucket.c_str(), cfg.lanes, cfg.lookahead, cfg.pi_group, cfg.pi_tile,
          cfg.upd_waves, ms);
  fclose(f);
}

struct TuneMemo {
  std::string bucket;
  Config cfg;
};
std::vector<TuneMemo> g_memo;

}  // namespace

extern "C" cdwac_status cdwac_batch_run(cdwac_ctx* ctx, const cdwac_batch_item* items, int n_items,
                                        const cdwac_params* prm, double tol, int max_iter, int max_lanes,
                                        unsigned flags, int* chosen, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!items || n_items < 1 || !prm || max_lanes < 1 || max_lanes > 64)
    return set_error(ctx, CDWAC_ERR_ARG, "bad batch arguments");
  for (int i = 0; i < n_items; ++i)
    if (!items[i].xi || !items[i].wxi || !items[i].W_imag || !items[i].pade.a)
      return set_error(ctx, CDWAC_ERR_ARG, "batch item %d has a null output", i);
  if (prm->precision != CDWAC_PREC_FP64 && prm->precision != CDWAC_PREC_MIXED)
    return set_error(ctx, CDWAC_ERR_ARG, "bad precision");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;

  Config cfg{std::min(max_lanes, std::min(n_items, 4)), 1, ctx->pi_group, ctx->pi_tile, ctx->upd_waves};
  if (flags & CDWAC_BATCH_AUTOTUNE) {
    const std::string bucket = bucket_of(items, n_items, prm);
    bool have = false;
    for (auto& m : g_memo)
      if (m.bucket == bucket && m.cfg.lanes <= max_lanes) {
        cfg = m.cfg;
        have = true;
      }
    if (!have) have = cache_lookup(bucket, max_lanes, &cfg);
    if (!have) {
      cudaEvent_t t0, t1;
      CDWAC_CUDA_TRY(ctx, cudaEventCreate(&t0));
      CDWAC_CUDA_TRY(ctx, cudaEventCreate(&t1));
      double best = 1e300;
      Config best_cfg = cfg;
      // one warm run (sizes scratch), one timed run; keeps the fastest
      auto trial = [&](Config c) -> cdwac_status {
        cdwac_status rc = enqueue(ctx, items, n_items, prm, tol, max_iter, c, st);
        if (rc) return rc;
        CDWAC_CUDA_TRY(ctx, cudaEventRecord(t0, st));
        rc = enqueue(ctx, items, n_items, prm, tol, max_iter, c, st);
        if (rc) return rc;
        CDWAC_CUDA_TRY(ctx, cudaEventRecord(t1, st));
        CDWAC_CUDA_TRY(ctx, cudaEventSynchronize(t1));
        float ms = 0.f;
        CDWAC_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, t0, t1));
        if (ms < best) {
          best = ms;
          best_cfg = c;
        }
        return CDWAC_OK;
      };
      // stage 1: lanes x lookahead at the current tile configuration
      for (int lanes : {1, 2, 4, 8}) {
        if (lanes > max_lanes || lanes > n_items) continue;
        for (int la = 0; la < 2; ++la) {
          cdwac_status rc = trial(Config{lanes, la, cfg.pi_group, cfg.pi_tile, cfg.upd_waves});
          if (rc) return rc;
        }
      }
      // stage 2: Pi tile width; stage 3: Pi tile-group size; stage 4: row-strip waves of the real trailing update
      // (each from the best so far)
      {
        Config c = best_cfg;
        c.pi_tile = c.pi_tile == 128 ? 256 : 128;
        cdwac_status rc = trial(c);
        if (rc) return rc;
      }
      for (int g : {4, 8, 12, 16}) {
        Config c = best_cfg;
        if (g == c.pi_group) continue;
        c.pi_group = g;
        cdwac_status rc = trial(c);
        if (rc) return rc;
      }
      for (int w : {1, 2, 3}) {
        Config c = best_cfg;
        if (w == c.upd_waves) continue;
        c.upd_waves = w;
        cdwac_status rc = trial(c);
        if (rc) return rc;
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      cfg = best_cfg;
      cache_store(bucket, cfg, best);
    }
    g_memo.push_back({bucket, cfg});
  }
  if (chosen) {
    chosen[0] = cfg.lanes;
    chosen[1] = cfg.lookahead;
    chosen[2] = cfg.pi_group;
    chosen[3] = cfg.pi_tile;
    chosen[4] = cfg.upd_waves;
  }

  if (!(flags & CDWAC_BATCH_GRAPH)) return enqueue(ctx, items, n_items, prm, tol, max_iter, cfg, st);

  const std::string key = batch_key(ctx, items, n_items, prm, tol, max_iter, cfg);
  if (!(ctx->graph_exec && ctx->graph_key == key)) {
    // eager run sizes every lane's scratch, so that nothing is allocated while the stream is being captured
    cdwac_status rc = enqueue(ctx, items, n_items, prm, tol, max_iter, cfg, st);
    if (rc) return rc;
    CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (ctx->graph_exec) {
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    cudaStream_t cap = nullptr;
    CDWAC_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    CDWAC_CUDA_TRY(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    rc = enqueue(ctx, items, n_items, prm, tol, max_iter, cfg, cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return set_error(ctx, CDWAC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ctx->graph_exec = nullptr;
      return set_error(ctx, CDWAC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    ctx->graph_key = batch_key(ctx, items, n_items, prm, tol, max_iter, cfg);   // lanes may have grown above
    return CDWAC_OK;   // the eager run above already produced this call's results
  }
  CDWAC_CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph_exec, st));
  return CDWAC_OK;
}
