// evr_batch.cu -- many independent event streams solved together.
//
// Every stream keeps the state layout of a single stream (evr_internal.cuh); the
// device holds an array of their plane descriptors.  A step takes one packet per
// stream (streams without events in the step are left alone): one launch validates
// and scatters all packets (one CTA per stream), then a CUDA graph runs the packet
// prologue over every stream's pixel blocks and the tiled iteration passes over a
// work list of (stream, tile) pairs.  The tiled kernel is the same instantiation the
// single-stream solver uses, so each stream's result is bit-identical to solving it
// alone with the same solver configuration.
//
// The streams can be cut into groups whose pass working set fits L2: the graph then runs
// each group's prologue and all its passes before the next group (optionally two groups
// at a time on two graph branches), so that a group's (u, p) and constants stay in L2
// across its passes instead of every pass sweeping the whole batch through HBM.
//
// The other schedule runs a whole step -- every stream's push, prologue and passes -- as
// one persistent launch working through an ordered list of (stream, item) pairs with
// per-stream dependency counts (evr_persist.cu), captured as a one-node CUDA graph whose
// arguments take each step's packets.  The autotuner times both schedules after choosing
// the tile configuration and keeps the faster one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/evr.h"
#include "evr_internal.cuh"
#include "evr_persist.cuh"

namespace evr {
int check_params(const evr_params* p);
}

using namespace evr;

struct evr_batch {
  int n = 0;
  evr_params prm{};
  std::vector<Planes> planes;  // host copies of the descriptors
  char* dev = nullptr;         // all device memory of the batch
  Planes* d_descs = nullptr;
  int* d_curs = nullptr;
  int* d_active = nullptr;
  int2* d_work_pro = nullptr;
  int n_work_pro = 0;
  int2* d_work_tile = nullptr;
  int n_work_tile = 0;
  std::vector<int> pro_off, tile_off;  // per stream: first work item (n + 1 entries)
  int cfg = -1;
  bool tuned = false;
  // L2 grouping of a step's work: pass working set per group (0: one group of all
  // streams), graph branches running groups side by side; auto: chosen by the autotuner
  long long group_budget = 0;
  int branches = 1;
  bool group_auto = true, group_tuned = false;
  struct Group {
    int tile0, ntile, pro0, npro;
  };
  std::vector<Group> groups;
  cudaStream_t stream = nullptr, own_stream = nullptr, cap_stream = nullptr;
  static constexpr int kMaxBranches = 4;
  cudaStream_t side[kMaxBranches - 1] = {};  // the other branches (capture and tuning)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::map<int, cudaGraphExec_t> graphs;  // by iteration count
  // persistent schedule (one launch per step): requested (-1 auto, 0 graph of launches,
  // 1 persistent), chosen, its window budget (pass bytes of the streams whose passes are
  // interleaved; 0: one window) and per iteration count its work list and graph
  int sched_req = EVR_BATCH_SCHEDULE_AUTO;
  bool persistent = false, sched_tuned = false;
  long long win_budget = 0;
  int pgrid = 0;
  int* d_ctrl = nullptr;    // control words (evr_persist.cuh)
  int* d_totals = nullptr;  // per stream: work items of a step
  struct Plan {
    int4* d_items = nullptr;
    int n_items = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    cudaGraph_t graph = nullptr;
  };
  std::map<int, Plan> plans;  // by iteration count
  // host-pointer steps: packed pinned staging (two slots) and device staging
  size_t stage_cap = 0;
  char* d_stage = nullptr;
  char* h_stage[2] = {nullptr, nullptr};
  size_t h_stage_cap[2] = {0, 0};
  cudaEvent_t h_stage_done[2] = {nullptr, nullptr};
  int next_stage = 0;
  // image readback: every stream's image gathered into one buffer, then one copy
  long long* d_img_off = nullptr;  // per stream, offset in floats
  float* d_img = nullptr;          // px_total floats (synchronous readback, staging 0)
  float* d_img2 = nullptr;         // staging 1 of the asynchronous readbacks
  cudaEvent_t img_ev[16] = {};     // recorded on copy_stream after each readback
  cudaEvent_t stage_ready[2] = {};
  cudaStream_t copy_stream = nullptr;  // the host copies of asynchronous readbacks
  unsigned long long img_ticket = 0;
  long long* d_offsets = nullptr;
  DevScalars* h_sc = nullptr;  // pinned, one per stream
  int* h_curs = nullptr;       // pinned
  // kernel timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
  std::vector<int> ev_launches;
  std::vector<long long> ev_pixiters;
  double t_ms = 0.0;
  long long t_launches = 0, t_pixiters = 0;
  long long px_total = 0;
  char name[96] = {0};
};

// Every stream's current image into one buffer: stream s at out + off[s], W*H floats,
// row-major without padding.  One CTA per stream, a warp per row.
__global__ void __launch_bounds__(256) k_batch_gather(const Planes* __restrict__ descs,
                                                     const int* __restrict__ curs,
                                                     const long long* __restrict__ off,
                                                     float* __restrict__ out) {
  __shared__ Planes P;
  const int s = blockIdx.x;
  if (threadIdx.x == 0) P = descs[s];
  __syncthreads();
  const float* u = P.u[curs[s]];
  float* o = out + off[s];
  for (int y = threadIdx.x / 32; y < P.H; y += blockDim.x / 32)
    for (int x = threadIdx.x % 32; x < P.W; x += 32)
      o[(size_t)y * P.W + x] = u[(size_t)y * P.pitch + x];
}

namespace {

// NVTX range for the duration of a C ABI call (a no-op when no tool is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

SolveConsts consts(const evr_batch* b) {
  return SolveConsts{b->prm.tau, b->prm.sigma, b->prm.lambda, b->prm.u_min, b->prm.u_max,
                     b->prm.data_term};
}

PrologueConsts pconsts(const evr_batch* b) {
  return PrologueConsts{b->prm.time_scale, b->prm.delta_pos, b->prm.delta_neg,
                        (long long)b->prm.t_max_us, b->prm.manifold, b->prm.data_mode, nullptr};
}

BatchRef bref(const evr_batch* b, bool tiles, int first = 0) {
  return BatchRef{b->d_descs, (tiles ? b->d_work_tile : b->d_work_pro) + first, b->d_curs,
                  b->d_active};
}

// Bytes one pass reads and writes of stream s: (u, p) of both buffers and the five
// constant planes (tx, ty, 1/G, sqrt G, f).
long long pass_bytes(const evr_batch* b, int s) {
  const long long ps = b->prm.storage ? 2 : 4;
  return (long long)b->planes[s].pitch * b->planes[s].H * (2 * (4 + 3 * ps) + 5 * 4);
}

// Cut the streams, in index order, into groups whose pass bytes stay within
// group_budget (a stream larger than the budget is a group of its own); budget 0: one
// group.  Needs the work offsets of the current tile work list.
void build_groups(evr_batch* b) {
  b->groups.clear();
  int s0 = 0;
  long long acc = 0;
  for (int s = 0; s <= b->n; ++s) {
    const long long sb = s < b->n ? pass_bytes(b, s) : 0;
    const bool cut = s == b->n || (b->group_budget > 0 && s > s0 && acc + sb > b->group_budget);
    if (cut) {
      b->groups.push_back(evr_batch::Group{b->tile_off[s0], b->tile_off[s] - b->tile_off[s0],
                                           b->pro_off[s0], b->pro_off[s] - b->pro_off[s0]});
      s0 = s;
      acc = 0;
    }
    acc += sb;
  }
}

// (stream, tile) work items of configuration ci for every stream.
int build_tile_work(evr_batch* b, int ci) {
  const SolverCfg& c = kSolverCfgs[ci];
  const TileShape& t = kTileShapes[c.shape];
  const int OW = t.EW - 2 * c.R, OH = t.EH - 2 * c.R;
  std::vector<int2> w;
  b->tile_off.assign(b->n + 1, 0);
  for (int s = 0; s < b->n; ++s) {
    const int tx = (b->planes[s].W + OW - 1) / OW, ty = (b->planes[s].H + OH - 1) / OH;
    b->tile_off[s] = (int)w.size();
    for (int k = 0; k < tx * ty; ++k) w.push_back(make_int2(s, k));
  }
  b->tile_off[b->n] = (int)w.size();
  build_groups(b);
  if (b->d_work_tile) cudaFree(b->d_work_tile);
  b->d_work_tile = nullptr;
  if (dev_alloc((void**)&b->d_work_tile, sizeof(int2) * w.size()) != cudaSuccess)
    return EVR_ERR_OOM;
  if (cudaMemcpy(b->d_work_tile, w.data(), sizeof(int2) * w.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return EVR_ERR_CUDA;
  b->n_work_tile = (int)w.size();
  return EVR_OK;
}

void drop_graphs(evr_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// ---- persistent schedule (evr_persist.cu)

void drop_plans(evr_batch* b) {
  if (!b->plans.empty()) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->plans) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    if (kv.second.d_items) cudaFree(kv.second.d_items);
  }
  b->plans.clear();
}

// Tiles of stream s under configuration ci.
int stream_tiles(const evr_batch* b, int s, int ci) {
  const SolverCfg& c = kSolverCfgs[ci];
  const TileShape& t = kTileShapes[c.shape];
  const int OW = t.EW - 2 * c.R, OH = t.EH - 2 * c.R;
  return ((b->planes[s].W + OW - 1) / OW) * ((b->planes[s].H + OH - 1) / OH);
}

// A step's work list for configuration ci with `passes` passes, window by window
// (streams in index order whose pass bytes stay within budget; 0: one window): the
// window's pushes and prologue bands, then pass after pass every stream's tiles, the
// next window's pushes and bands placed before the last pass, so that they run while
// this window drains.  Each item waits for the items of its stream listed before its own
// group (the push for a band; the push, the bands and the earlier passes for a pass).
// timing: passes only.  totals[s]: stream s's items.
void persist_items(const evr_batch* b, int ci, int passes, bool timing, long long budget,
                   std::vector<int4>* items, std::vector<int>* totals) {
  items->clear();
  totals->assign(b->n, 0);
  std::vector<std::pair<int, int>> win;
  int s0 = 0;
  long long acc = 0;
  for (int s = 0; s <= b->n; ++s) {
    const long long sb = s < b->n ? pass_bytes(b, s) : 0;
    const bool cut = s == b->n || (budget > 0 && s > s0 && acc + sb > budget);
    if (cut && s > s0) {
      win.emplace_back(s0, s);
      s0 = s;
      acc = 0;
    }
    acc += sb;
  }
  auto bands = [&](int q) { return (b->planes[q].H + kPersistProRows - 1) / kPersistProRows; };
  auto front = [&](size_t g) {
    if (timing || g >= win.size()) return;
    for (int q = win[g].first; q < win[g].second; ++q)
      items->push_back(make_int4(q, kItemPush, 0, 0));
    for (int q = win[g].first; q < win[g].second; ++q)
      for (int k = 0; k < bands(q); ++k) items->push_back(make_int4(q, kItemPrologue, k, 1));
  };
  auto pass = [&](size_t g, int j) {
    for (int q = win[g].first; q < win[g].second; ++q) {
      const int nt = stream_tiles(b, q, ci);
      const int need = (timing ? 0 : 1 + bands(q)) + j * nt;
      for (int k = 0; k < nt; ++k) items->push_back(make_int4(q, j, k, need));
    }
  };
  front(0);
  for (size_t g = 0; g < win.size(); ++g) {
    for (int j = 0; j + 1 < passes; ++j) pass(g, j);
    front(g + 1);
    if (passes > 0) pass(g, passes - 1);
    for (int q = win[g].first; q < win[g].second; ++q)
      (*totals)[q] = (timing ? 0 : 1 + bands(q)) + passes * stream_tiles(b, q, ci);
  }
}

// Work list and per-stream totals in one device buffer (items, then totals).
int upload_items(const std::vector<int4>& items, const std::vector<int>& totals, int4** out) {
  *out = nullptr;
  const size_t ib = sizeof(int4) * items.size(), tb = sizeof(int) * totals.size();
  if (dev_alloc((void**)out, ib + tb + 16) != cudaSuccess) {
    *out = nullptr;
    return EVR_ERR_OOM;
  }
  cudaError_t e = cudaMemcpy(*out, items.data(), ib, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy((char*)*out + ib, totals.data(), tb, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(*out);
    *out = nullptr;
    return EVR_ERR_CUDA;
  }
  return EVR_OK;
}

int ensure_ctrl(evr_batch* b) {
  if (b->d_ctrl) return EVR_OK;
  const size_t bytes = sizeof(int) * persist_ctrl_ints(b->n);
  if (dev_alloc((void**)&b->d_ctrl, bytes) != cudaSuccess) {
    b->d_ctrl = nullptr;
    return EVR_ERR_OOM;
  }
  if (cudaMemset(b->d_ctrl, 0, bytes) != cudaSuccess) return EVR_ERR_CUDA;
  return EVR_OK;
}

PersistArgs persist_args(const evr_batch* b, int ci, const int4* d_items, int n_items,
                         int iters, bool timing) {
  PersistArgs a{};
  a.descs = b->d_descs;
  a.curs = b->d_curs;
  a.active = b->d_active;
  a.items = d_items;
  a.totals = (const int*)(d_items + n_items);
  a.ctrl = b->d_ctrl;
  a.n_items = n_items;
  a.n_streams = b->n;
  a.R = kSolverCfgs[ci].R;
  a.iters = iters;
  a.timing = timing ? 1 : 0;
  a.c = consts(b);
  a.pc = pconsts(b);
  return a;
}

// Milliseconds of one persistent run of configuration ci's passes over the batch (timing
// items: each pass reads the live buffer and writes the other one), best of `reps` after
// one warm-up run, or -1.  need_bump > 0 (self-test): the first item waits for that
// many more completions than its stream will ever reach.
float time_persist(evr_batch* b, int ci, int iters, long long budget, int reps,
                   cudaEvent_t e0, cudaEvent_t e1, int need_bump = 0) {
  const SolverCfg& cfg = kSolverCfgs[ci];
  if (!persist_supported(cfg, b->prm.storage) || ensure_ctrl(b)) return -1.f;
  const int grid = persist_grid(cfg, b->prm.storage);
  if (grid <= 0) return -1.f;
  std::vector<int4> items;
  std::vector<int> totals;
  persist_items(b, ci, (iters + cfg.R - 1) / cfg.R, true, budget, &items, &totals);
  if (items.empty()) return -1.f;
  if (need_bump > 0) items[0].w += need_bump;
  int4* d_items = nullptr;
  if (upload_items(items, totals, &d_items)) return -1.f;
  const PersistArgs a = persist_args(b, ci, d_items, (int)items.size(), iters, true);
  float best = -1.f;
  bool ok = need_bump > 0 ||
            launch_batch_persist(cfg, b->prm.storage, a, grid, b->stream) == 0;
  for (int rep = 0; ok && rep < reps; ++rep) {
    cudaEventRecord(e0, b->stream);
    ok = launch_batch_persist(cfg, b->prm.storage, a, grid, b->stream) == 0;
    cudaEventRecord(e1, b->stream);
    float ms = 0.f;
    if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      ok = false;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.f || ms < best) best = ms;
  }
  cudaStreamSynchronize(b->stream);
  cudaFree(d_items);
  return ok ? best : -1.f;
}

float time_passes(evr_batch* b, int ci, int iters, int reps, cudaEvent_t e0, cudaEvent_t e1);

// The persistent schedule against the graph of launches, after the graph's configuration
// and grouping were chosen: window budgets for the chosen configuration (or the first
// persistent-capable one), then (configs) every persistent-capable configuration under
// the best budget.  Keeps the persistent schedule if it is faster (or requested).
void tune_schedule(evr_batch* b, int iters, bool configs, cudaEvent_t e0, cudaEvent_t e1) {
  const int storage = b->prm.storage;
  const bool forced = b->sched_req == EVR_BATCH_SCHEDULE_PERSISTENT;
  const float graph_ms = forced ? 1e30f : time_passes(b, b->cfg, iters, 2, e0, e1);
  int pc = -1;
  if (persist_supported(kSolverCfgs[b->cfg], storage)) {
    pc = b->cfg;
  } else if (configs) {
    for (int ci = 0; ci < kNumSolverCfgs && pc < 0; ++ci)
      if (persist_supported(kSolverCfgs[ci], storage)) pc = ci;
  }
  if (pc < 0) {
    b->persistent = false;
    b->sched_tuned = true;
    return;
  }
  static const long long kWindowsMB[] = {0, 128, 96, 64, 48, 32, 24, 16};
  long long best_budget = b->group_auto ? 0 : b->group_budget;
  float best = -1.f;
  if (b->group_auto) {
    for (long long mb : kWindowsMB) {
      const float t = time_persist(b, pc, iters, mb << 20, 2, e0, e1);
      if (t >= 0.f && (best < 0.f || t < best)) {
        best = t;
        best_budget = mb << 20;
      }
    }
  } else {
    best = time_persist(b, pc, iters, best_budget, 2, e0, e1);
  }
  if (configs) {
    for (int ci = 0; ci < kNumSolverCfgs; ++ci) {
      if (ci == pc || !persist_supported(kSolverCfgs[ci], storage)) continue;
      const float t = time_persist(b, ci, iters, best_budget, 2, e0, e1);
      if (t >= 0.f && (best < 0.f || t < best)) {
        best = t;
        pc = ci;
      }
    }
  }
  b->sched_tuned = true;
  if (best >= 0.f && (forced || best < graph_ms)) {
    b->persistent = true;
    b->win_budget = best_budget;
    b->pgrid = persist_grid(kSolverCfgs[pc], storage);
    if (pc != b->cfg) {
      b->cfg = pc;
      build_tile_work(b, b->cfg);
    }
  } else {
    b->persistent = false;
  }
}

// The persistent step of `iters` iterations with this call's packets: the plan's graph
// (one kernel node) is captured at the first use, later calls set the node's arguments.
int persist_step(evr_batch* b, const uint16_t* x, const uint16_t* y, const long long* t,
                 const int8_t* pol, const long long* offsets, int iters) {
  if (ensure_ctrl(b)) return EVR_ERR_OOM;
  const SolverCfg& cfg = kSolverCfgs[b->cfg];
  auto it = b->plans.find(iters);
  evr_batch::Plan* pl = nullptr;
  if (it == b->plans.end()) {
    evr_batch::Plan np;
    std::vector<int4> items;
    std::vector<int> totals;
    persist_items(b, b->cfg, (iters + cfg.R - 1) / cfg.R, false, b->win_budget, &items,
                  &totals);
    np.n_items = (int)items.size();
    int rc = upload_items(items, totals, &np.d_items);
    if (rc) return rc;
    PersistArgs a = persist_args(b, b->cfg, np.d_items, np.n_items, iters, false);
    a.x = x;
    a.y = y;
    a.t = t;
    a.pol = pol;
    a.offsets = offsets;
    bool bad = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) !=
               cudaSuccess;
    if (!bad) bad = launch_batch_persist(cfg, b->prm.storage, a, b->pgrid, b->cap_stream) != 0;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &np.graph);
    size_t roots = 1;
    if (!bad && e == cudaSuccess) e = cudaGraphGetRootNodes(np.graph, &np.node, &roots);
    if (!bad && e == cudaSuccess && roots == 1) e = cudaGraphInstantiate(&np.exec, np.graph, 0);
    if (bad || e != cudaSuccess || roots != 1 || !np.exec) {
      if (np.exec) cudaGraphExecDestroy(np.exec);
      if (np.graph) cudaGraphDestroy(np.graph);
      cudaFree(np.d_items);
      return EVR_ERR_CUDA;
    }
    pl = &(b->plans[iters] = np);
  } else {
    pl = &it->second;
    PersistArgs a = persist_args(b, b->cfg, pl->d_items, pl->n_items, iters, false);
    a.x = x;
    a.y = y;
    a.t = t;
    a.pol = pol;
    a.offsets = offsets;
    if (persist_node_set(pl->exec, pl->node, a)) return EVR_ERR_CUDA;
  }
  return cudaGraphLaunch(pl->exec, b->stream) == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

void set_name(evr_batch* b) {
  if (b->cfg < 0) {
    std::snprintf(b->name, sizeof(b->name), "batch: untuned");
    return;
  }
  const SolverCfg& c = kSolverCfgs[b->cfg];
  const TileShape& t = kTileShapes[c.shape];
  if (b->persistent) {
    const int n = std::snprintf(b->name, sizeof(b->name),
                                "batch of %d: persistent step, tiled %dx%d R%d (%d threads, "
                                "%d CTAs)",
                                b->n, t.EW, t.EH, c.R, 32 * t.NTY, b->pgrid);
    if (b->win_budget > 0 && n > 0 && n < (int)sizeof(b->name))
      std::snprintf(b->name + n, sizeof(b->name) - n, ", windows of <= %lld MB",
                    b->win_budget >> 20);
    return;
  }
  const int n = std::snprintf(b->name, sizeof(b->name),
                              "batch of %d: tiled %dx%d R%d (%d threads, %d CTAs)", b->n, t.EW,
                              t.EH, c.R, 32 * t.NTY, b->n_work_tile);
  if (b->groups.size() > 1 && n > 0 && n < (int)sizeof(b->name))
    std::snprintf(b->name + n, sizeof(b->name) - n, ", %d L2 groups of <= %lld MB x %d",
                  (int)b->groups.size(), b->group_budget >> 20, b->branches);
}

// A step's work for configuration ci, group by group: group g on branch g mod
// `branches`, branch 0 being q and the others the batch's side streams (fork and join
// through events, so the same code serves stream capture and direct launches).  step:
// each group's prologue, then its passes with their indices in the step; otherwise
// (timing) the passes only, all with index 0 (each reads the live buffer and writes the
// other one, which a step overwrites anyway).
int enqueue_groups(evr_batch* b, int ci, int iters, bool step, cudaStream_t q) {
  const SolverCfg& cfg = kSolverCfgs[ci];
  const SolveConsts c = consts(b);
  const int nb = std::min<int>(b->branches, (int)b->groups.size());
  int bad = 0;
  if (nb > 1) bad |= cudaEventRecord(b->ev_fork, q) != cudaSuccess;
  for (int k = 1; k < nb; ++k) bad |= cudaStreamWaitEvent(b->side[k - 1], b->ev_fork, 0) != cudaSuccess;
  for (size_t g = 0; g < b->groups.size(); ++g) {
    const evr_batch::Group& G = b->groups[g];
    cudaStream_t st = g % nb ? b->side[g % nb - 1] : q;
    if (step) bad |= launch_prologue_batch(bref(b, false, G.pro0), G.npro, pconsts(b), st);
    for (int done = 0, j = 0; done < iters; done += cfg.R, ++j) {
      const int k = iters - done < cfg.R ? iters - done : cfg.R;
      bad |= launch_tiled_pass_batch(bref(b, true, G.tile0), G.ntile, cfg, step ? j : 0, k, c,
                                     b->prm.storage, st);
    }
  }
  for (int k = 1; k < nb; ++k) {  // each wait takes the event's latest record
    bad |= cudaEventRecord(b->ev_join, b->side[k - 1]) != cudaSuccess;
    bad |= cudaStreamWaitEvent(q, b->ev_join, 0) != cudaSuccess;
  }
  return bad;
}

// Milliseconds of the passes of a step (best of `reps` after one warm-up), or -1.
float time_passes(evr_batch* b, int ci, int iters, int reps, cudaEvent_t e0, cudaEvent_t e1) {
  float best = -1.f;
  if (enqueue_groups(b, ci, iters, false, b->stream)) return -1.f;
  for (int rep = 0; rep < reps; ++rep) {
    cudaEventRecord(e0, b->stream);
    const int bad = enqueue_groups(b, ci, iters, false, b->stream);
    cudaEventRecord(e1, b->stream);
    float ms = 0.f;
    if (bad || cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      return -1.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.f || ms < best) best = ms;
  }
  return best;
}

// Fastest multi-launch configuration under the current grouping (every configuration
// timed on the whole batch with the packet's iteration count, best of two runs), or -1.
int screen_configs(evr_batch* b, int iters, cudaEvent_t e0, cudaEvent_t e1, float* best_ms) {
  float best = 1e30f;
  int best_cfg = -1;
  for (int ci = 0; ci < kNumSolverCfgs; ++ci) {
    if (kSolverCfgs[ci].kind != 1) continue;
    if (build_tile_work(b, ci)) continue;
    const float ms = time_passes(b, ci, iters, 2, e0, e1);
    if (ms >= 0.f && ms < best) {
      best = ms;
      best_cfg = ci;
    }
  }
  *best_ms = best;
  return best_cfg;
}

// The step's tiled configuration and L2 grouping.  configs: the configuration is
// screened with one group.  Unless the grouping was set: every budget from 64 MB down to
// 8 MB of pass working set per group with one to four branches is timed against one
// group for that configuration, and with configs the configurations are screened again
// under the best grouping.  The timing launches read the live buffer and write the other
// one, so the live state is untouched.
void autotune(evr_batch* b, int iters, bool configs) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const long long budget = b->group_budget;
  const int branches = b->branches;
  float ms = 0.f;
  if (configs) {
    b->group_budget = 0;
    b->branches = 1;
    const int ci = screen_configs(b, iters, e0, e1, &ms);
    b->cfg = ci < 0 ? 0 : ci;
    b->group_budget = budget;
    b->branches = branches;
  }
  if (b->group_auto) {
    static const long long kBudgetsMB[] = {64, 48, 32, 24, 16, 12, 8};
    long long best_budget = 0;
    int best_branches = 1;
    b->group_budget = 0;
    b->branches = 1;
    float best = build_tile_work(b, b->cfg) ? -1.f : time_passes(b, b->cfg, iters, 2, e0, e1);
    for (long long mb : kBudgetsMB)
      for (int br = 1; br <= evr_batch::kMaxBranches && best >= 0.f; ++br) {
        b->group_budget = mb << 20;
        b->branches = br;
        build_groups(b);
        if ((int)b->groups.size() < std::max(2, br)) continue;
        const float t = time_passes(b, b->cfg, iters, 2, e0, e1);
        if (t >= 0.f && t < best) {
          best = t;
          best_budget = b->group_budget;
          best_branches = br;
        }
      }
    b->group_budget = best_budget;
    b->branches = best_branches;
    b->group_tuned = true;
    if (configs && best_budget > 0) {
      const int ci = screen_configs(b, iters, e0, e1, &ms);
      if (ci >= 0 && ms < best) b->cfg = ci;
    }
  }
  build_tile_work(b, b->cfg);
  if (b->sched_req != EVR_BATCH_SCHEDULE_GRAPH) {
    tune_schedule(b, iters, configs, e0, e1);
  } else {
    b->persistent = false;
    b->sched_tuned = true;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

void resolve_timing(evr_batch* b) {
  for (size_t k = 0; k < b->ev_used.size(); ++k) {
    cudaEventSynchronize(b->ev_used[k].second);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev_used[k].first, b->ev_used[k].second);
    b->t_ms += ms;
    b->t_launches += b->ev_launches[k];
    b->t_pixiters += b->ev_pixiters[k];
    b->ev_free.push_back(b->ev_used[k]);
  }
  b->ev_used.clear();
  b->ev_launches.clear();
  b->ev_pixiters.clear();
}

// Graph of one step after the push: prologue over all streams, the passes, the flip.
int step_graph(evr_batch* b, int iters, cudaGraphExec_t* out) {
  auto it = b->graphs.find(iters);
  if (it != b->graphs.end()) {
    *out = it->second;
    return EVR_OK;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return EVR_ERR_CUDA;
  int bad = enqueue_groups(b, b->cfg, iters, true, b->cap_stream);
  if (iters > 0) {
    const int R = kSolverCfgs[b->cfg].R;
    bad |= launch_batch_flip(b->d_curs, b->d_active, b->n, (iters + R - 1) / R, b->cap_stream);
  }
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  if (bad || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return EVR_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  b->graphs[iters] = exec;
  *out = exec;
  return EVR_OK;
}

int read_back(evr_batch* b) {
  cudaError_t e = cudaMemcpyAsync(b->h_curs, b->d_curs, sizeof(int) * b->n,
                                  cudaMemcpyDeviceToHost, b->stream);
  for (int s = 0; s < b->n && e == cudaSuccess; ++s)
    e = cudaMemcpyAsync(&b->h_sc[s], b->planes[s].sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

}  // namespace

extern "C" {

int evr_batch_create(int n, const int* W, const int* H, const evr_params* params,
                     evr_batch** out) {
  if (!out) return EVR_ERR_INVALID_ARG;
  *out = nullptr;
  if (n <= 0 || !W || !H || !params || !check_params(params)) return EVR_ERR_INVALID_ARG;
  if (params->solver == EVR_SOLVER_UNFUSED || params->tvl1_iters > 0)
    return EVR_ERR_NOT_SUPPORTED;
  if (params->tile_config > 0 && kSolverCfgs[params->tile_config - 1].kind != 1)
    return EVR_ERR_NOT_SUPPORTED;
  for (int s = 0; s < n; ++s)
    if (W[s] <= 0 || H[s] <= 0 || W[s] > 65536 || H[s] > 65536) return EVR_ERR_INVALID_ARG;
  int rc = check_device();
  if (rc) return rc;
  evr_batch* b = new (std::nothrow) evr_batch();
  if (!b) return EVR_ERR_OOM;
  b->n = n;
  b->prm = *params;
  size_t total = 0;
  std::vector<size_t> off(n);
  for (int s = 0; s < n; ++s) {
    off[s] = total;
    total += state_bytes(W[s], H[s], false);
  }
  const size_t tail = total;
  total += sizeof(Planes) * n + 256 + 2 * sizeof(int) * n + 256;
  if (dev_alloc((void**)&b->dev, total) != cudaSuccess) {
    delete b;
    return EVR_ERR_OOM;
  }
  b->planes.resize(n);
  std::vector<int2> pro;
  b->pro_off.assign(n + 1, 0);
  for (int s = 0; s < n; ++s) {
    carve_state(b->dev + off[s], W[s], H[s], false, &b->planes[s]);
    b->planes[s].storage = params->storage;
    const int nb = ((W[s] + 31) / 32) * ((H[s] + 7) / 8);
    b->pro_off[s] = (int)pro.size();
    for (int k = 0; k < nb; ++k) pro.push_back(make_int2(s, k));
    b->px_total += (long long)W[s] * H[s];
  }
  b->pro_off[n] = (int)pro.size();
  b->d_descs = (Planes*)(b->dev + tail);
  b->d_curs = (int*)(b->dev + tail + (sizeof(Planes) * n + 255) / 256 * 256);
  b->d_active = b->d_curs + n;
  cudaError_t e = cudaMemcpy(b->d_descs, b->planes.data(), sizeof(Planes) * n,
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_curs, 0, 2 * sizeof(int) * n);
  if (e == cudaSuccess) e = dev_alloc((void**)&b->d_work_pro, sizeof(int2) * pro.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_work_pro, pro.data(), sizeof(int2) * pro.size(), cudaMemcpyHostToDevice);
  b->n_work_pro = (int)pro.size();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  for (auto& q : b->side)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = host_alloc((void**)&b->h_sc, sizeof(DevScalars) * n);
  if (e == cudaSuccess) e = host_alloc((void**)&b->h_curs, sizeof(int) * n);
  b->stream = b->own_stream;
  const bool first = params->t_init_us == EVR_T_INIT_FIRST;
  const long long t0 = first ? 0 : (long long)params->t_init_us;
  for (int s = 0; s < n && e == cudaSuccess; ++s)
    if (launch_init(b->planes[s], params->u_init, t0, t0, first ? 0 : 1, b->stream))
      e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    evr_batch_destroy(b);
    return EVR_ERR_CUDA;
  }
  if (params->tile_config > 0) {
    b->cfg = params->tile_config - 1;
    if (build_tile_work(b, b->cfg)) {
      evr_batch_destroy(b);
      return EVR_ERR_OOM;
    }
    b->tuned = true;
  }
  set_name(b);
  *out = b;
  return EVR_OK;
}

void evr_batch_destroy(evr_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  drop_plans(b);
  if (b->d_ctrl) cudaFree(b->d_ctrl);
  resolve_timing(b);
  for (auto& e : b->ev_free) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (b->d_work_pro) cudaFree(b->d_work_pro);
  if (b->d_work_tile) cudaFree(b->d_work_tile);
  if (b->d_stage) cudaFree(b->d_stage);
  for (int k = 0; k < 2; ++k) {
    if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
    if (b->h_stage_done[k]) cudaEventDestroy(b->h_stage_done[k]);
  }
  if (b->copy_stream) {
    cudaStreamSynchronize(b->copy_stream);
    cudaStreamDestroy(b->copy_stream);
  }
  if (b->d_img_off) cudaFree(b->d_img_off);
  if (b->d_img) cudaFree(b->d_img);
  if (b->d_img2) cudaFree(b->d_img2);
  for (auto& e : b->img_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : b->stage_ready)
    if (e) cudaEventDestroy(e);
  if (b->h_sc) cudaFreeHost(b->h_sc);
  if (b->h_curs) cudaFreeHost(b->h_curs);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (auto& q : b->side)
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

int evr_batch_set_grouping(evr_batch* b, long long budget_bytes, int branches) {
  if (!b || branches < 1 || branches > evr_batch::kMaxBranches) return EVR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return EVR_ERR_CUDA;
  b->group_auto = budget_bytes < 0;
  b->group_tuned = false;
  b->group_budget = budget_bytes > 0 ? budget_bytes : 0;
  b->branches = budget_bytes < 0 ? 1 : branches;
  if (b->cfg >= 0 && !b->tile_off.empty()) build_groups(b);
  drop_graphs(b);
  drop_plans(b);
  b->sched_tuned = false;  // the windows follow the grouping
  set_name(b);
  return EVR_OK;
}

int evr_batch_set_schedule(evr_batch* b, int schedule) {
  if (!b || schedule < EVR_BATCH_SCHEDULE_AUTO || schedule > EVR_BATCH_SCHEDULE_PERSISTENT)
    return EVR_ERR_INVALID_ARG;
  if (schedule == EVR_BATCH_SCHEDULE_PERSISTENT && b->prm.tile_config > 0 &&
      !persist_supported(kSolverCfgs[b->prm.tile_config - 1], b->prm.storage))
    return EVR_ERR_NOT_SUPPORTED;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return EVR_ERR_CUDA;
  b->sched_req = schedule;
  b->sched_tuned = false;
  b->persistent = false;
  drop_plans(b);
  set_name(b);
  return EVR_OK;
}

int evr_batch_get_schedule(evr_batch* b, int* schedule) {
  if (!b || !schedule) return EVR_ERR_INVALID_ARG;
  *schedule = b->persistent ? EVR_BATCH_SCHEDULE_PERSISTENT : EVR_BATCH_SCHEDULE_GRAPH;
  return EVR_OK;
}

int evr_batch_selftest_persist_timeout(evr_batch* b) {
  if (!b) return EVR_ERR_INVALID_ARG;
  int ci = b->cfg >= 0 && persist_supported(kSolverCfgs[b->cfg], b->prm.storage) ? b->cfg : -1;
  for (int k = 0; k < kNumSolverCfgs && ci < 0; ++k)
    if (persist_supported(kSolverCfgs[k], b->prm.storage)) ci = k;
  if (ci < 0) return EVR_ERR_NOT_SUPPORTED;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return EVR_ERR_CUDA;
  int rc = ensure_ctrl(b);
  if (rc) return rc;
  if (cudaMemset(b->d_ctrl + kCtrlStatus, 0, sizeof(int)) != cudaSuccess) return EVR_ERR_CUDA;
  // every stream taken as active: the timing items ignore the active flags
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  time_persist(b, ci, kSolverCfgs[ci].R, 0, 1, e0, e1, 1 << 30);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<int> ctrl(persist_ctrl_ints(b->n));
  if (cudaMemcpy(ctrl.data(), b->d_ctrl, sizeof(int) * ctrl.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return EVR_ERR_CUDA;
  const int status = ctrl[kCtrlStatus];
  bool clean = ctrl[kCtrlHead] == 0 && ctrl[kCtrlLeft] == 0 && ctrl[kCtrlAbort] == 0;
  for (int s = 0; s < b->n; ++s) clean = clean && ctrl[kCtrlCount + s * kCtrlStride] == 0;
  if (cudaMemset(b->d_ctrl + kCtrlStatus, 0, sizeof(int)) != cudaSuccess) return EVR_ERR_CUDA;
  if (!clean) return EVR_ERR_CUDA;
  return status;
}

int evr_batch_set_cuda_stream(evr_batch* b, void* cuda_stream) {
  if (!b) return EVR_ERR_INVALID_ARG;
  cudaStream_t ns = cuda_stream == EVR_OWN_STREAM ? b->own_stream : (cudaStream_t)cuda_stream;
  if (ns != b->stream) {
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return EVR_ERR_CUDA;
    b->stream = ns;
  }
  return EVR_OK;
}

int evr_batch_step_device(evr_batch* b, const uint16_t* x, const uint16_t* y,
                          const int64_t* t_us, const int8_t* pol, const int64_t* offsets,
                          int iters) {
  Range range("evr_batch_step_device");
  if (!b || !offsets || iters < 0) return EVR_ERR_INVALID_ARG;
  if (!x || !y || !t_us || !pol) return EVR_ERR_INVALID_ARG;
  cudaStream_t st = b->stream;
  const bool tuned = b->tuned && (!b->group_auto || b->group_tuned) && b->sched_tuned;
  if (iters > 0 && tuned && b->persistent) {  // the whole step in one launch
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (b->timing) {
      if (b->ev_free.empty()) {
        cudaEventCreate(&ev.first);
        cudaEventCreate(&ev.second);
      } else {
        ev = b->ev_free.back();
        b->ev_free.pop_back();
      }
      cudaEventRecord(ev.first, st);
    }
    const int rc = persist_step(b, x, y, (const long long*)t_us, pol, (const long long*)offsets,
                                iters);
    if (b->timing) {
      cudaEventRecord(ev.second, st);
      b->ev_used.push_back(ev);
      b->ev_launches.push_back(1);
      b->ev_pixiters.push_back(b->px_total * iters);  // upper bound: every stream active
    }
    return rc;
  }
  if (launch_push_batch(b->d_descs, b->n, x, y, (const long long*)t_us, pol,
                        (const long long*)offsets, b->d_active, st))
    return EVR_ERR_CUDA;
  if (iters > 0 && !tuned) {
    autotune(b, iters, !b->tuned);
    drop_graphs(b);  // the tile work list may have moved
    drop_plans(b);
    b->tuned = true;
    set_name(b);
  }
  if (b->cfg < 0) {  // iters == 0 before any tuning: prologue only
    b->cfg = 0;
    if (build_tile_work(b, 0)) return EVR_ERR_OOM;
  }
  cudaGraphExec_t exec = nullptr;
  int rc = step_graph(b, iters, &exec);
  if (rc) return rc;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (b->timing) {
    if (b->ev_free.empty()) {
      cudaEventCreate(&ev.first);
      cudaEventCreate(&ev.second);
    } else {
      ev = b->ev_free.back();
      b->ev_free.pop_back();
    }
    cudaEventRecord(ev.first, st);
  }
  if (cudaGraphLaunch(exec, st) != cudaSuccess) return EVR_ERR_CUDA;
  if (b->timing) {
    cudaEventRecord(ev.second, st);
    b->ev_used.push_back(ev);
    const int R = kSolverCfgs[b->cfg].R, groups = (int)b->groups.size();
    // every launch of the graph: per group the prologue and the passes; the flip
    b->ev_launches.push_back(iters > 0 ? groups * (1 + (iters + R - 1) / R) + 1 : groups);
    b->ev_pixiters.push_back(b->px_total * iters);  // upper bound: every stream active
  }
  return EVR_OK;
}

int evr_batch_step(evr_batch* b, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
                   const int8_t* pol, const int64_t* offsets, int iters) {
  Range range("evr_batch_step");
  if (!b || !offsets || iters < 0) return EVR_ERR_INVALID_ARG;
  const long long n_ev = offsets[b->n];
  for (int s = 0; s < b->n; ++s)
    if (offsets[s + 1] < offsets[s] || offsets[0] != 0) return EVR_ERR_INVALID_ARG;
  if (n_ev > 0 && (!x || !y || !t_us || !pol)) return EVR_ERR_INVALID_ARG;
  // packed layout, the same in the pinned slot and on the device:
  // offsets | t | x | y | pol, each part at a 256-byte boundary
  const size_t o_t = (sizeof(long long) * (b->n + 1) + 255) / 256 * 256;
  const size_t o_x = o_t + ((size_t)n_ev * 8 + 255) / 256 * 256;
  const size_t o_y = o_x + ((size_t)n_ev * 2 + 255) / 256 * 256;
  const size_t o_p = o_y + ((size_t)n_ev * 2 + 255) / 256 * 256;
  const size_t bytes = o_p + (size_t)n_ev;
  if (b->stage_cap < bytes) {
    if (b->d_stage) {
      cudaStreamSynchronize(b->stream);
      cudaFree(b->d_stage);
    }
    b->d_stage = nullptr;
    b->stage_cap = 0;
    if (dev_alloc((void**)&b->d_stage, bytes * 2) != cudaSuccess) return EVR_ERR_OOM;
    b->stage_cap = bytes * 2;
  }
  const int k = b->next_stage;
  b->next_stage ^= 1;
  if (b->h_stage_done[k] && cudaEventSynchronize(b->h_stage_done[k]) != cudaSuccess)
    return EVR_ERR_CUDA;  // the slot's previous copy has completed
  if (b->h_stage_cap[k] < bytes) {
    if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
    b->h_stage[k] = nullptr;
    b->h_stage_cap[k] = 0;
    if (host_alloc((void**)&b->h_stage[k], bytes * 2) != cudaSuccess) return EVR_ERR_OOM;
    b->h_stage_cap[k] = bytes * 2;
  }
  if (!b->h_stage_done[k] &&
      cudaEventCreateWithFlags(&b->h_stage_done[k], cudaEventDisableTiming) != cudaSuccess)
    return EVR_ERR_CUDA;
  char* h = b->h_stage[k];
  std::memcpy(h, offsets, sizeof(long long) * (b->n + 1));
  if (n_ev > 0) {
    std::memcpy(h + o_t, t_us, (size_t)n_ev * 8);
    std::memcpy(h + o_x, x, (size_t)n_ev * 2);
    std::memcpy(h + o_y, y, (size_t)n_ev * 2);
    std::memcpy(h + o_p, pol, (size_t)n_ev);
  }
  cudaStream_t st = b->stream;
  char* q = b->d_stage;
  cudaError_t e = cudaMemcpyAsync(q, h, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->h_stage_done[k], st);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  return evr_batch_step_device(b, (const uint16_t*)(q + o_x), (const uint16_t*)(q + o_y),
                               (const int64_t*)(q + o_t), (const int8_t*)(q + o_p),
                               (const int64_t*)q, iters);
}

int evr_batch_get_image(evr_batch* b, int s, float* out_host, size_t len) {
  if (!b || s < 0 || s >= b->n || !out_host) return EVR_ERR_INVALID_ARG;
  const Planes& P = b->planes[s];
  if (len < (size_t)P.W * P.H) return EVR_ERR_INVALID_ARG;
  if (read_back(b)) return EVR_ERR_CUDA;
  cudaError_t e = cudaMemcpy2DAsync(out_host, (size_t)P.W * 4, P.u[b->h_curs[s]],
                                    (size_t)P.pitch * 4, (size_t)P.W * 4, P.H,
                                    cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

// Queue the gather of all images and their copy to out_host on the batch's stream.
// The gather buffer and per-stream offsets (allocated at the first readback).
static int ensure_gather(evr_batch* b) {
  if (b->d_img) return EVR_OK;
  std::vector<long long> off(b->n);
  long long acc = 0;
  for (int s = 0; s < b->n; ++s) {
    off[s] = acc;
    acc += (long long)b->planes[s].W * b->planes[s].H;
  }
  if (dev_alloc((void**)&b->d_img_off, sizeof(long long) * b->n) != cudaSuccess)
    return EVR_ERR_OOM;
  if (dev_alloc((void**)&b->d_img, sizeof(float) * (size_t)b->px_total) != cudaSuccess) {
    cudaFree(b->d_img_off);
    b->d_img_off = nullptr;
    b->d_img = nullptr;
    return EVR_ERR_OOM;
  }
  if (cudaMemcpy(b->d_img_off, off.data(), sizeof(long long) * b->n, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return EVR_ERR_CUDA;
  return EVR_OK;
}

int evr_batch_get_images(evr_batch* b, float* out_host, size_t len) {
  Range range("evr_batch_get_images");
  if (!b || !out_host) return EVR_ERR_INVALID_ARG;
  if ((long long)len < b->px_total) return EVR_ERR_INVALID_ARG;
  int rc = ensure_gather(b);
  if (rc) return rc;
  k_batch_gather<<<b->n, 256, 0, b->stream>>>(b->d_descs, b->d_curs, b->d_img_off, b->d_img);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_host, b->d_img, sizeof(float) * (size_t)b->px_total,
                        cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

// Asynchronous: the gather into one of two staging buffers runs on the batch's stream in
// order with the steps; the host copy runs on copy_stream and overlaps the next steps.
int evr_batch_get_images_async(evr_batch* b, float* out_host, size_t len, uint64_t* ticket) {
  Range range("evr_batch_get_images_async");
  if (!b || !out_host || !ticket) return EVR_ERR_INVALID_ARG;
  if ((long long)len < b->px_total) return EVR_ERR_INVALID_ARG;
  int rc = ensure_gather(b);
  if (rc) return rc;
  if (!b->copy_stream) {
    if (dev_alloc((void**)&b->d_img2, sizeof(float) * (size_t)b->px_total) != cudaSuccess) {
      b->d_img2 = nullptr;
      return EVR_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return EVR_ERR_CUDA;
    for (auto& e : b->img_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return EVR_ERR_CUDA;
    for (auto& e : b->stage_ready)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return EVR_ERR_CUDA;
  }
  const unsigned long long t = b->img_ticket + 1;
  const int slot = (int)(t % 16), stage = (int)(t % 2);
  float* dst = stage ? b->d_img2 : b->d_img;
  if (cudaEventSynchronize(b->img_ev[slot]) != cudaSuccess) return EVR_ERR_CUDA;  // ring reuse
  cudaError_t e = cudaSuccess;
  // the staging buffer is reused once its previous host copy (ticket t - 2) is done
  if (t > 2) e = cudaStreamWaitEvent(b->stream, b->img_ev[(t - 2) % 16], 0);
  if (e == cudaSuccess) {
    k_batch_gather<<<b->n, 256, 0, b->stream>>>(b->d_descs, b->d_curs, b->d_img_off, dst);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->stage_ready[stage], b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_stream, b->stage_ready[stage], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_host, dst, sizeof(float) * (size_t)b->px_total,
                        cudaMemcpyDeviceToHost, b->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->img_ev[slot], b->copy_stream);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  b->img_ticket = t;
  *ticket = t;
  return EVR_OK;
}

int evr_batch_wait_images(evr_batch* b, uint64_t ticket) {
  if (!b || ticket == 0 || ticket > b->img_ticket) return EVR_ERR_INVALID_ARG;
  // a slot recorded again since belongs to a later readback, which completes later
  return cudaEventSynchronize(b->img_ev[ticket % 16]) == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

int evr_batch_get_state(evr_batch* b, int s, int which, void* out_host, size_t bytes) {
  if (!b || s < 0 || s >= b->n || !out_host) return EVR_ERR_INVALID_ARG;
  if (read_back(b)) return EVR_ERR_CUDA;
  const Planes& P = b->planes[s];
  const int cur = b->h_curs[s];
  if (which == EVR_STATE_CLOCK || which == EVR_STATE_TINIT) {
    if (bytes != 8) return EVR_ERR_INVALID_ARG;
    long long v = which == EVR_STATE_CLOCK ? b->h_sc[s].clock
                                           : (b->h_sc[s].t_init_set ? b->h_sc[s].t_init : 0);
    std::memcpy(out_host, &v, 8);
    return EVR_OK;
  }
  const void* src = nullptr;
  size_t elem = 4;
  switch (which) {
    case EVR_STATE_U: src = P.u[cur]; break;
    case EVR_STATE_P1: src = P.p1[cur]; break;
    case EVR_STATE_P2: src = P.p2[cur]; break;
    case EVR_STATE_P3: src = P.p3[cur]; break;
    case EVR_STATE_F: src = P.f; break;
    case EVR_STATE_SQRTG: src = P.sG; break;
    case EVR_STATE_TX: src = P.tx; break;
    case EVR_STATE_TY: src = P.ty; break;
    case EVR_STATE_NPOS: src = P.npos; break;
    case EVR_STATE_NNEG: src = P.nneg; break;
    case EVR_STATE_TLAST: src = P.t_last; elem = 8; break;
    default: return EVR_ERR_INVALID_ARG;
  }
  if (bytes != elem * P.W * P.H) return EVR_ERR_INVALID_ARG;
  if (P.storage != 0 && which >= EVR_STATE_P1 && which <= EVR_STATE_P3) {
    if (launch_p_convert(P, (void*)src, P.ubar, 1, b->stream)) return EVR_ERR_CUDA;
    src = P.ubar;
  }
  cudaError_t e = cudaMemcpy2DAsync(out_host, elem * P.W, src, elem * P.pitch, elem * P.W, P.H,
                                    cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  if (which == EVR_STATE_TLAST) {
    long long t_init = b->h_sc[s].t_init_set ? b->h_sc[s].t_init : b->h_sc[s].clock;
    long long* v = (long long*)out_host;
    for (size_t i = 0; i < (size_t)P.W * P.H; ++i)
      if (v[i] == kNeverFired) v[i] = t_init;
  }
  return EVR_OK;
}

int evr_batch_synchronize(evr_batch* b, int* stream_out) {
  if (!b) return EVR_ERR_INVALID_ARG;
  if (stream_out) *stream_out = -1;
  if (read_back(b)) return EVR_ERR_CUDA;
  int code = EVR_OK;
  for (int s = 0; s < b->n; ++s) {
    if (b->h_sc[s].status != 0) {
      if (code == EVR_OK) {
        code = b->h_sc[s].status;
        if (stream_out) *stream_out = s;
      }
      if (cudaMemsetAsync(&b->planes[s].sc->status, 0, sizeof(int), b->stream) != cudaSuccess)
        return EVR_ERR_CUDA;
    }
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return EVR_ERR_CUDA;
  return code;
}

int evr_batch_enable_kernel_timing(evr_batch* b, int enable) {
  if (!b) return EVR_ERR_INVALID_ARG;
  resolve_timing(b);
  b->t_ms = 0.0;
  b->t_launches = 0;
  b->t_pixiters = 0;
  b->timing = enable != 0;
  return EVR_OK;
}

int evr_batch_kernel_time(evr_batch* b, double* ms, int64_t* launches, int64_t* pixel_iters) {
  if (!b || !ms || !launches || !pixel_iters) return EVR_ERR_INVALID_ARG;
  resolve_timing(b);
  *ms = b->t_ms;
  *launches = b->t_launches;
  *pixel_iters = b->t_pixiters;
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

const char* evr_batch_solver_name(evr_batch* b) { return b ? b->name : ""; }

}  // extern "C"
