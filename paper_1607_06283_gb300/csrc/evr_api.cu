// evr_api.cu -- host runtime and C ABI (include/evr.h).
//
// The host side validates arguments, stages host events through pinned memory,
// owns the device state, picks the solver configuration by timing the candidates
// on the actual sensor (autotuner), captures the multi-launch tiled solver's
// launches into a CUDA graph (one per iteration count and buffer parity), and reads
// results back.  Every step of the reconstruction itself runs in the kernels of
// evr_kernels.cu and evr_solvers.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include <atomic>

#include "../../include/evr.h"
#include "evr_internal.cuh"

using namespace evr;

// ---------------------------------------------------------------- allocation hook
namespace {
std::atomic<int> g_fail_countdown{0};  // > 0: the allocation that takes it to 0 fails

bool alloc_fails() {
  int c = g_fail_countdown.load();
  while (c > 0)
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  return false;
}

// NVTX range for the duration of a C ABI call (visible to profilers and tracers; a no-op
// when none is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

namespace evr {
cudaError_t dev_alloc(void** p, size_t bytes) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
cudaError_t host_alloc(void** p, size_t bytes) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}
}  // namespace evr

namespace {

constexpr int kStageSlots = 4;  // pinned staging slots: packets whose copy may be in flight
constexpr int kMaxTimingPairs = 8192;

// A packet of n events is staged packed, x | y | t | pol (t at an 8-byte boundary), so
// one host-to-device copy moves it; the device buffer uses the same layout.
struct Packed {
  size_t off_y, off_t, off_p, bytes;
  explicit Packed(size_t n)
      : off_y(2 * n), off_t((4 * n + 7) / 8 * 8), off_p(off_t + 8 * n), bytes(off_p + n) {}
};

struct StageSlot {
  size_t cap = 0;            // events
  char* h = nullptr;         // pinned, 13 * cap bytes
  cudaEvent_t done = nullptr;  // recorded after the work that reads the slot
  bool pending = false;
  // evr_step: the slot's own device copy of the packet, filled on the handle's copy
  // stream ahead of the packet's graph (which waits for `copied`)
  size_t dcap = 0;           // events
  char* d = nullptr;         // device, 13 * dcap bytes
  cudaEvent_t copied = nullptr;
};

constexpr int kImgRing = 16;  // asynchronous image readbacks in flight per handle
constexpr int kImgStage = 3;  // device staging images of the asynchronous readbacks

struct GraphKey {
  int iters, cur, front;  // front: the graph starts with the (TV-L1 +) prologue launches
  int cfg;
  bool operator<(const GraphKey& o) const {
    if (iters != o.iters) return iters < o.iters;
    if (cur != o.cur) return cur < o.cur;
    return front != o.front ? front < o.front : cfg < o.cfg;
  }
};

constexpr int kScreenKeep = 6;   // configurations re-timed after the autotuner's screen
constexpr int kRefineCands = 3;  // configurations refined on real solves
constexpr int kRefineReps = 3;   // real solves per candidate

}  // namespace

struct evr_stream {
  int W = 0, H = 0, pitch = 0, device = 0;
  evr_params prm{};
  Planes P{};
  void* dev_base = nullptr;
  cudaStream_t stream = nullptr;      // where work is queued
  cudaStream_t own_stream = nullptr;  // the library's stream
  cudaStream_t cap_stream = nullptr;  // graph capture
  int cur = 0;                        // buffer holding the current (u, p)
  int cfg = -1;                       // index into kSolverCfgs, -1 = unfused
  bool tuned = false;
  // online refinement of the autotuner's choice: its closest candidates take turns on
  // the next real solves, timed with CUDA events around each solve; the fastest stays
  int cand[kRefineCands] = {0, 0, 0};
  int n_cand = 0;
  int refine_done = 0;  // real solves timed so far
  cudaEvent_t ref_ev[kRefineCands * kRefineReps][2] = {};
  int flag_base = 0;                  // persistent solver: progress-flag count
  // host-to-device event staging
  StageSlot slot[kStageSlots];
  cudaStream_t h2d_stream = nullptr;  // evr_step: packet copies ahead of their graphs
  int next_slot = 0;
  size_t dcap = 0;           // events
  char* dstage = nullptr;    // device, 13 * dcap bytes
  // asynchronous image readbacks: completion event and status copy per ticket
  cudaEvent_t img_ev[kImgRing] = {};  // recorded on copy_stream after each readback
  int* h_img_status = nullptr;  // pinned, kImgRing ints
  unsigned long long img_ticket = 0;
  // the device-to-host part of an asynchronous readback runs on copy_stream from one of
  // kImgStage staging images (W*H floats each), overlapping the next packets' kernels
  cudaStream_t copy_stream = nullptr;
  float* d_img_stage = nullptr;
  cudaEvent_t stage_ready[kImgStage] = {};
  // host mirror of the stream clock for immediate checks
  long long h_clock = 0;
  bool h_have_clock = false;
  bool h_clock_valid = true;
  // results
  double* d_gap = nullptr;   // 2 doubles on the device
  double* h_gap = nullptr;   // pinned
  DevScalars* h_sc = nullptr;  // pinned
  // graphs of the per-packet iteration launches
  std::map<GraphKey, cudaGraphExec_t> graphs;
  // push-and-solve graphs (evr_step_device): the executable, its graph and push node
  struct Fused {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t push = nullptr;
  };
  std::map<GraphKey, Fused> fused;
  // kernel timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free, ev_used;
  std::vector<int> ev_launches;
  std::vector<long long> ev_pixiters;
  double t_ms = 0.0;
  long long t_launches = 0, t_pixiters = 0;
  char name[64] = {0};
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? EVR_OK : EVR_ERR_CUDA; }

SolveConsts solve_consts(const evr_stream* s) {
  return SolveConsts{s->prm.tau, s->prm.sigma, s->prm.lambda, s->prm.u_min, s->prm.u_max,
                     s->prm.data_term};
}

PrologueConsts prologue_consts(const evr_stream* s) {
  return PrologueConsts{s->prm.time_scale, s->prm.delta_pos, s->prm.delta_neg,
                        (long long)s->prm.t_max_us, s->prm.manifold, s->prm.data_mode, nullptr};
}

int params_valid(const evr_params* p) {
  if (!(p->lambda > 0.f) || !(p->delta_pos > 0.f) || !(p->delta_neg > 0.f)) return 0;
  if (!(p->u_min > 0.f) || !(p->u_min < p->u_max)) return 0;
  if (!(p->u_init >= p->u_min && p->u_init <= p->u_max)) return 0;
  if (!(p->tau > 0.f) || !(p->sigma > 0.f)) return 0;
  double bound = (double)p->tau * (double)p->sigma * (8.0 + 4.0 * std::sqrt(2.0));
  if (bound > 1.0 + 1e-6) return 0;
  if (!(p->time_scale >= 0.f) || !std::isfinite(p->time_scale)) return 0;
  if (p->data_mode != 0 && p->data_mode != 1) return 0;
  if (p->manifold != 0 && p->manifold != 1) return 0;
  if (p->solver < 0 || p->solver > EVR_SOLVER_TILED) return 0;
  if (p->tile_config < 0 || p->tile_config > kNumSolverCfgs) return 0;
  if (p->storage < 0 || p->storage > 2) return 0;
  if (p->data_term != 0 && p->data_term != 1) return 0;
  if (p->tvl1_iters < 0 || p->tvl1_iters > 100000) return 0;
  if (p->tvl1_iters > 0 && !(p->tvl1_lambda > 0.f)) return 0;
  if (p->storage != 0) {
    if (p->solver == EVR_SOLVER_UNFUSED) return 0;
    if (p->tile_config > 0 && kSolverCfgs[p->tile_config - 1].kind != 1) return 0;
  }
  return 1;
}

void set_name(evr_stream* s) {
  if (s->cfg < 0) {
    std::snprintf(s->name, sizeof(s->name), "unfused");
  } else {
    const SolverCfg& c = kSolverCfgs[s->cfg];
    const TileShape& t = kTileShapes[c.shape];
    if (c.kind == 3)
      std::snprintf(s->name, sizeof(s->name), "cluster %dx%d of %dx%d R%d (%d threads, %d CTAs)",
                    c.cx, c.cy, t.EW, t.EH, c.R, 32 * t.NTY, solver_cfg_ctas(s->P, c));
    else if (c.kind == 4)
      std::snprintf(s->name, sizeof(s->name), "staged %dx%d R%d (%d threads, %d CTAs)", t.EW,
                    t.EH, c.R, 32 * t.NTY, solver_cfg_ctas(s->P, c));
    else
      std::snprintf(s->name, sizeof(s->name), "%s %dx%d R%d (%d threads, %d CTAs)",
                    c.kind == 2 ? "persistent" : c.kind == 5 ? "resident" : "tiled", t.EW,
                    t.EH, c.R, 32 * t.NTY,
                    solver_cfg_ctas(s->P, c));
  }
}

void free_stage(evr_stream* s) {
  if (s->h2d_stream) {
    cudaStreamSynchronize(s->h2d_stream);
    cudaStreamDestroy(s->h2d_stream);
    s->h2d_stream = nullptr;
  }
  for (auto& sl : s->slot) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.copied) cudaEventDestroy(sl.copied);
    if (sl.h) cudaFreeHost(sl.h);
    if (sl.d) cudaFree(sl.d);
    sl = StageSlot{};
  }
  if (s->dstage) cudaFree(s->dstage);
  s->dstage = nullptr;
  s->dcap = 0;
  if (s->copy_stream) {
    cudaStreamSynchronize(s->copy_stream);
    cudaStreamDestroy(s->copy_stream);
    s->copy_stream = nullptr;
  }
  for (auto& e : s->img_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  for (auto& e : s->stage_ready) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (s->d_img_stage) cudaFree(s->d_img_stage);
  s->d_img_stage = nullptr;
  if (s->h_img_status) cudaFreeHost(s->h_img_status);
  s->h_img_status = nullptr;
}

// Grow the pinned slot to hold n events.
int ensure_stage(StageSlot& sl, size_t n) {
  if (sl.cap < n) {
    if (sl.done) cudaEventSynchronize(sl.done);
    if (sl.h) cudaFreeHost(sl.h);
    // cap > n, so 13 cap bytes hold Packed(n).bytes <= 13 n + 7
    size_t cap = ((n < 4096 ? 4096 : n + n / 2) + 63) / 64 * 64;
    if (host_alloc((void**)&sl.h, cap * 13) != cudaSuccess) {
      sl.h = nullptr;
      sl.cap = 0;
      return EVR_ERR_OOM;
    }
    sl.cap = cap;
    if (!sl.done && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      return EVR_ERR_CUDA;
  }
  return EVR_OK;
}

// evr_push_events: grow the handle's device staging buffer (read by the push on the
// handle's stream) to hold n events.
int ensure_dstage(evr_stream* s, size_t n) {
  if (s->dcap < n) {
    if (s->dstage) {
      cudaStreamSynchronize(s->stream);
      cudaFree(s->dstage);
    }
    size_t cap = ((n < 4096 ? 4096 : n + n / 2) + 63) / 64 * 64;
    if (dev_alloc((void**)&s->dstage, cap * 13) != cudaSuccess) {
      s->dstage = nullptr;
      s->dcap = 0;
      return EVR_ERR_OOM;
    }
    s->dcap = cap;
  }
  return EVR_OK;
}

// evr_step: the slot's device copy of n events, its copy event and the handle's copy
// stream.  The caller has waited for the slot's previous packet (stage_host), so the old
// device buffer is no longer read.
int ensure_slot_device(evr_stream* s, StageSlot& sl, size_t n) {
  if (!s->h2d_stream &&
      cudaStreamCreateWithFlags(&s->h2d_stream, cudaStreamNonBlocking) != cudaSuccess) {
    s->h2d_stream = nullptr;
    return EVR_ERR_CUDA;
  }
  if (!sl.copied && cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) != cudaSuccess) {
    sl.copied = nullptr;
    return EVR_ERR_CUDA;
  }
  if (sl.dcap < n) {
    if (sl.d) cudaFree(sl.d);
    sl.d = nullptr;
    sl.dcap = 0;
    const size_t cap = ((n < 4096 ? 4096 : n + n / 2) + 63) / 64 * 64;
    if (dev_alloc((void**)&sl.d, cap * 13) != cudaSuccess) {
      sl.d = nullptr;
      return EVR_ERR_OOM;
    }
    sl.dcap = cap;
  }
  return EVR_OK;
}

void drop_graphs(evr_stream* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
  for (auto& kv : s->fused) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  s->fused.clear();
}

// Clear the persistent solver's progress flags (required whenever the set of CTAs
// changes and after an aborted launch).
int clear_flags(evr_stream* s) {
  s->flag_base = 0;
  cudaError_t e = cudaMemsetAsync(s->P.flags, 0, sizeof(int) * (kMaxCtas + 2), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&s->P.sc->abort, 0, sizeof(int), s->stream);
  return cuda_err(e);
}

int solve_passes(const SolverCfg& cfg, int iters);

// The multi-launch iteration launches of one packet (unfused or kind 1):
// `iters` iterations from buffer `cur`.  Returns the buffer holding the result.
int enqueue_iterations(evr_stream* s, int iters, int cur, cudaStream_t st, int* launches,
                       const PrologueConsts* front = nullptr, const PushArgs* push = nullptr) {
  SolveConsts c = solve_consts(s);
  *launches = 0;
  if (s->cfg < 0) {
    for (int k = 0; k < iters; ++k) {
      if (launch_unfused_iteration(s->P, cur, c, st)) return -1;
      *launches += 2;
    }
    return cur;
  }
  const SolverCfg& cfg = kSolverCfgs[s->cfg];
  if (cfg.kind == 3 && cfg.R == 0) {  // one cluster over the sensor: one launch
    if (launch_cluster(s->P, cfg, cur, iters, 0, c, st, front, nullptr)) return -1;
    *launches = 1;
    return 1 - cur;
  }
  if (cfg.kind == 5) {  // resident: one cooperative launch
    if (launch_resident(s->P, cfg, cur, iters, c, st, front, push)) return -1;
    *launches = 1;
    return cur ^ (solve_passes(cfg, iters) & 1);
  }
  for (int done = 0, pass = 0; done < iters; done += cfg.R, ++pass) {
    int it = iters - done < cfg.R ? iters - done : cfg.R;
    const int e = cfg.kind == 3   ? launch_cluster(s->P, cfg, cur, it, pass, c, st, front, nullptr)
                  : cfg.kind == 4 ? launch_staged(s->P, cfg, cur, it, pass, c, st)
                                  : launch_tiled_pass(s->P, cfg, cur, it, pass, c, st, front, push);
    if (e) return -1;
    cur = 1 - cur;
    *launches += 1;
  }
  return cur;
}

// Passes of one packet's solve with configuration cfg (kind 1 or 3).
int solve_passes(const SolverCfg& cfg, int iters) {
  return (cfg.kind == 3 && cfg.R == 0) ? 1 : (iters + cfg.R - 1) / cfg.R;
}

// Kernel launches of one packet's solve (the front not counted).
int solve_launches(const SolverCfg& cfg, int iters) {
  return cfg.kind == 5 ? 1 : solve_passes(cfg, iters);
}

// Run one packet's iterations with configuration index `ci` (kind 1 or 2) directly
// on the handle's stream; updates s->cur.
int run_cfg_direct(evr_stream* s, int ci, int iters) {
  const SolverCfg& cfg = kSolverCfgs[ci];
  SolveConsts c = solve_consts(s);
  if (cfg.kind == 2) {
    if (launch_persistent(s->P, cfg, s->cur, iters, s->flag_base, c, s->stream)) return -1;
    const int passes = (iters + cfg.R - 1) / cfg.R;
    s->flag_base += passes - 1;
    s->cur ^= passes & 1;
    return 0;
  }
  int launches = 0;
  int r = enqueue_iterations(s, iters, s->cur, s->stream, &launches);
  if (r < 0) return -1;
  s->cur = r;
  return 0;
}

// Time every usable configuration on this sensor with the packet's iteration count
// and keep the fastest.  The live (u, p) is saved first and restored afterwards.
void autotune(evr_stream* s, int iters) {
  const size_t plane = (size_t)s->pitch * s->H * sizeof(float);
  float* save = nullptr;
  if (dev_alloc((void**)&save, 4 * plane) != cudaSuccess) {
    s->cfg = 0;
    return;
  }
  const int cur0 = s->cur;
  float* src[4] = {s->P.u[cur0], s->P.p1[cur0], s->P.p2[cur0], s->P.p3[cur0]};
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync((char*)save + k * plane, src[k], plane, cudaMemcpyDeviceToDevice, s->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time `reps` back-to-back solves of configuration ci (after `warm` untimed ones);
  // < 0: the configuration failed (launch error or a timed-out wait)
  auto trial = [&](int ci, int warm, int reps) -> float {
    s->cfg = ci;
    clear_flags(s);
    bool ok = true;
    for (int r = 0; r < warm && ok; ++r) ok = run_cfg_direct(s, ci, iters) == 0;
    cudaEventRecord(e0, s->stream);
    for (int r = 0; r < reps && ok; ++r) ok = run_cfg_direct(s, ci, iters) == 0;
    cudaEventRecord(e1, s->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int st = 0;
    cudaMemcpy(&st, &s->P.sc->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (st != 0) {  // a timed-out trial disqualifies the configuration
      ok = false;
      cudaMemset(&s->P.sc->status, 0, sizeof(int));
    }
    if (cudaGetLastError() != cudaSuccess) ok = false;
    return ok ? ms / (float)reps : -1.0f;
  };
  // screen: every usable configuration once (after one untimed solve that loads its
  // kernel); then the kScreenKeep fastest three more times each, keeping the best time
  std::vector<std::pair<float, int>> timed;  // (ms per solve, configuration)
  for (int ci = 0; ci < kNumSolverCfgs; ++ci) {
    // the persistent configurations were measured slower than relaunching on every
    // workload (their L2 flag exchange); they stay selectable through tile_config
    if (kSolverCfgs[ci].kind == 2) continue;
    if (s->P.storage != 0 && kSolverCfgs[ci].kind != 1) continue;  // 16-bit p: kind 1 only
    if (!solver_cfg_usable(s->P, kSolverCfgs[ci])) continue;
    const float ms = trial(ci, 1, 1);
    if (ms >= 0.f) timed.emplace_back(ms, ci);
  }
  std::sort(timed.begin(), timed.end());
  if (timed.size() > (size_t)kScreenKeep) timed.resize(kScreenKeep);
  for (auto& t : timed) {
    const float ms = trial(t.second, 0, 3);
    if (ms >= 0.f && ms < t.first) t.first = ms;
  }
  std::sort(timed.begin(), timed.end());
  float best = timed.empty() ? 0.f : timed[0].first;
  int best_cfg = timed.empty() ? 0 : timed[0].second;
  // candidates for the online refinement: configurations within 25 % of the best
  // back-to-back time (these trials run warm and without the packet's front launches;
  // real solves decide among them)
  s->n_cand = 0;
  s->refine_done = 0;
  for (const auto& t : timed)
    if (s->n_cand < kRefineCands && t.first <= 1.25f * best) s->cand[s->n_cand++] = t.second;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  float* dst[4] = {s->P.u[cur0], s->P.p1[cur0], s->P.p2[cur0], s->P.p3[cur0]};
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync(dst[k], (char*)save + k * plane, plane, cudaMemcpyDeviceToDevice, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaFree(save);
  s->cur = cur0;
  s->cfg = best_cfg;
  clear_flags(s);
}

int refresh_scalars(evr_stream* s) {
  cudaError_t e = cudaMemcpyAsync(s->h_sc, s->P.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  s->h_clock = s->h_sc->clock;
  s->h_have_clock = s->h_sc->t_init_set != 0;
  s->h_clock_valid = true;
  return EVR_OK;
}

// Synchronise, then report (and clear) the first pending device-side rejection.
int sync_status(evr_stream* s) {
  int rc = refresh_scalars(s);
  if (rc) return rc;
  int st = s->h_sc->status;
  if (st != 0) {
    if (cudaMemsetAsync(&s->P.sc->status, 0, sizeof(int), s->stream) != cudaSuccess)
      return EVR_ERR_CUDA;
    if (st == EVR_ERR_TIMEOUT && clear_flags(s) != EVR_OK) return EVR_ERR_CUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return EVR_ERR_CUDA;
    return st;
  }
  return EVR_OK;
}

void resolve_timing(evr_stream* s) {
  for (size_t k = 0; k < s->ev_used.size(); ++k) {
    cudaEventSynchronize(s->ev_used[k].second);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev_used[k].first, s->ev_used[k].second);
    s->t_ms += ms;
    s->t_launches += s->ev_launches[k];
    s->t_pixiters += s->ev_pixiters[k];
    s->ev_free.push_back(s->ev_used[k]);
  }
  s->ev_used.clear();
  s->ev_launches.clear();
  s->ev_pixiters.clear();
}

}  // namespace

namespace evr {

static size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Device bytes of one stream's state (see the layout in evr_internal.cuh); `solo`
// adds the gap partials, the gap result and the persistent solver's flags.
size_t state_bytes(int W, int H, bool solo) {
  const size_t plane = (size_t)((W + 31) / 32 * 32) * H;
  const size_t fb = al256(plane * 4), lb = al256(plane * 8);
  size_t total = 16 * fb + lb + al256(sizeof(DevScalars));
  if (solo)
    total += al256(sizeof(double) * 3 * kGapBlocks) + al256(sizeof(double) * 2) +
             al256(sizeof(int) * (kMaxCtas + 2));
  return total;
}

// Lay one stream's planes out from `base`; returns the first byte after them (for a
// solo stream: the 2-double gap result, followed by nothing else).
char* carve_state(char* base, int W, int H, bool solo, Planes* out) {
  Planes P{};
  P.W = W;
  P.H = H;
  P.Hm = H;
  P.pitch = (W + 31) / 32 * 32;
  const size_t plane = (size_t)P.pitch * H;
  const size_t fb = al256(plane * 4), lb = al256(plane * 8);
  char* q = base;
  auto take = [&](size_t b) {
    char* r = q;
    q += b;
    return r;
  };
  for (int b = 0; b < 2; ++b) {
    P.u[b] = (float*)take(fb);
    P.p1[b] = (float*)take(fb);
    P.p2[b] = (float*)take(fb);
    P.p3[b] = (float*)take(fb);
  }
  P.ubar = (float*)take(fb);
  P.f = (float*)take(fb);
  P.tx = (float*)take(fb);
  P.ty = (float*)take(fb);
  P.iG = (float*)take(fb);
  P.sG = (float*)take(fb);
  P.t_last = (long long*)take(lb);
  P.npos = (int*)take(fb);
  P.nneg = (int*)take(fb);
  P.sc = (DevScalars*)take(al256(sizeof(DevScalars)));
  P.partials = nullptr;
  P.flags = nullptr;
  char* gap = nullptr;
  if (solo) {
    P.partials = (double*)take(al256(sizeof(double) * 3 * kGapBlocks));
    gap = take(al256(sizeof(double) * 2));
    P.flags = (int*)take(al256(sizeof(int) * (kMaxCtas + 2)));
  }
  *out = P;
  return solo ? gap : q;
}

int check_params(const evr_params* p) { return params_valid(p); }

int check_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EVR_ERR_NOT_SUPPORTED;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return EVR_ERR_NOT_SUPPORTED;
  if (!(prop.major == 10 && prop.minor == 3)) return EVR_ERR_NOT_SUPPORTED;
  return EVR_OK;
}

}  // namespace evr

extern "C" {

int evr_default_params(evr_params* out) {
  if (!out) return EVR_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->lambda = 90.0f;
  out->delta_pos = 0.15f;
  out->delta_neg = 0.15f;
  out->u_min = (float)std::exp(-3.0);
  out->u_max = (float)std::exp(3.0);
  out->u_init = 1.0f;
  out->tau = (float)(1.0 / std::sqrt(8.0 + 4.0 * std::sqrt(2.0)));
  out->sigma = out->tau;
  out->time_scale = 1e-3f;
  out->t_max_us = 100000;
  out->t_init_us = EVR_T_INIT_FIRST;
  out->data_mode = 0;
  out->manifold = 1;
  out->solver = EVR_SOLVER_AUTO;
  out->tile_config = 0;
  out->storage = 0;
  out->data_term = 0;
  out->tvl1_iters = 0;
  out->tvl1_lambda = 1.0f;
  return EVR_OK;
}

int evr_create(int W, int H, const evr_params* params, evr_stream** out) {
  if (!out) return EVR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params || W <= 0 || H <= 0 || W > 65536 || H > 65536) return EVR_ERR_INVALID_ARG;
  if (!params_valid(params)) return EVR_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EVR_ERR_NOT_SUPPORTED;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return EVR_ERR_NOT_SUPPORTED;
  if (!(prop.major == 10 && prop.minor == 3)) return EVR_ERR_NOT_SUPPORTED;
  evr_stream* s = new (std::nothrow) evr_stream();
  if (!s) return EVR_ERR_OOM;
  s->W = W;
  s->H = H;
  s->device = dev;
  s->prm = *params;
  s->pitch = (W + 31) / 32 * 32;
  const size_t total = evr::state_bytes(W, H, true);
  char* base = nullptr;
  if (dev_alloc((void**)&base, total) != cudaSuccess) {
    delete s;
    return EVR_ERR_OOM;
  }
  s->dev_base = base;
  char* q = evr::carve_state(base, W, H, true, &s->P);
  s->P.storage = params->storage;
  s->d_gap = (double*)q;
  Planes& P = s->P;
  int rc = EVR_OK;
  if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      host_alloc((void**)&s->h_gap, sizeof(double) * 2) != cudaSuccess ||
      host_alloc((void**)&s->h_sc, sizeof(DevScalars)) != cudaSuccess)
    rc = EVR_ERR_CUDA;
  s->stream = s->own_stream;
  const bool first = params->t_init_us == EVR_T_INIT_FIRST;
  const long long t0 = first ? 0 : (long long)params->t_init_us;
  if (!rc && launch_init(P, params->u_init, t0, t0, first ? 0 : 1, s->stream)) rc = EVR_ERR_CUDA;
  if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = EVR_ERR_CUDA;
  if (rc) {
    evr_destroy(s);
    return rc;
  }
  s->h_clock = t0;
  s->h_have_clock = !first;
  s->h_clock_valid = true;
  if (params->solver == EVR_SOLVER_UNFUSED) {
    s->cfg = -1;
    s->tuned = true;
  } else if (params->tile_config > 0) {
    s->cfg = params->tile_config - 1;
    if (!solver_cfg_usable(s->P, kSolverCfgs[s->cfg])) {
      evr_destroy(s);
      return EVR_ERR_NOT_SUPPORTED;
    }
    s->tuned = true;
  }
  set_name(s);
  *out = s;
  return EVR_OK;
}

void evr_destroy(evr_stream* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  drop_graphs(s);
  resolve_timing(s);
  for (auto& e : s->ev_free) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  free_stage(s);
  for (auto& pr : s->ref_ev)
    for (auto& e : pr)
      if (e) cudaEventDestroy(e);
  if (s->h_gap) cudaFreeHost(s->h_gap);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  if (s->own_stream) cudaStreamDestroy(s->own_stream);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->dev_base) cudaFree(s->dev_base);
  delete s;
}

int evr_set_cuda_stream(evr_stream* s, void* cuda_stream) {
  if (!s) return EVR_ERR_INVALID_ARG;
  cudaStream_t ns = cuda_stream == EVR_OWN_STREAM ? s->own_stream : (cudaStream_t)cuda_stream;
  if (ns != s->stream) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return EVR_ERR_CUDA;
    s->stream = ns;
  }
  return EVR_OK;
}

}  // extern "C"

namespace {
// Immediate host checks of a host-array packet (in the order the device applies them)
// and its packed copy into the next pinned slot.  On success *slot is the slot and
// *clock the packet's last timestamp.
int stage_host(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
               const int8_t* pol, size_t n, StageSlot** slot, long long* clock_out) {
  long long clock = s->h_clock;
  bool have = s->h_have_clock && s->h_clock_valid;
  for (size_t i = 0; i < n; ++i) {
    if ((int)x[i] >= s->W || (int)y[i] >= s->H) return EVR_ERR_OUT_OF_RANGE;
    if (pol[i] == 0) return EVR_ERR_BAD_POLARITY;
    if (have && (long long)t_us[i] < clock) return EVR_ERR_NONMONOTONIC;
    have = true;
    clock = (long long)t_us[i];
  }
  StageSlot& sl = s->slot[s->next_slot];
  s->next_slot = (s->next_slot + 1) % kStageSlots;
  if (sl.pending) {
    if (cudaEventSynchronize(sl.done) != cudaSuccess) return EVR_ERR_CUDA;
    sl.pending = false;
  }
  int rc = ensure_stage(sl, n);
  if (rc) return rc;
  const Packed L(n);
  std::memcpy(sl.h, x, n * 2);
  std::memcpy(sl.h + L.off_y, y, n * 2);
  std::memcpy(sl.h + L.off_t, t_us, n * 8);
  std::memcpy(sl.h + L.off_p, pol, n);
  *slot = &sl;
  *clock_out = clock;
  return EVR_OK;
}

void note_clock(evr_stream* s, long long clock) {
  if (s->h_clock_valid) {
    s->h_clock = clock;
    s->h_have_clock = true;
  }
}
}  // namespace

extern "C" {

int evr_push_events(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
                    const int8_t* pol, size_t n) {
  Range range("evr_push_events");
  if (!s) return EVR_ERR_INVALID_ARG;
  if (n == 0) return EVR_OK;
  if (!x || !y || !t_us || !pol || n > (size_t)INT_MAX) return EVR_ERR_INVALID_ARG;
  StageSlot* sl = nullptr;
  long long clock = 0;
  int rc = stage_host(s, x, y, t_us, pol, n, &sl, &clock);
  if (rc == EVR_OK) rc = ensure_dstage(s, n);
  if (rc) return rc;
  const Packed L(n);
  cudaStream_t st = s->stream;
  cudaError_t e = cudaMemcpyAsync(s->dstage, sl->h, L.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl->done, st);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  sl->pending = true;
  char* d = s->dstage;
  if (launch_push(s->P, (const uint16_t*)d, (const uint16_t*)(d + L.off_y),
                  (const long long*)(d + L.off_t), (const int8_t*)(d + L.off_p), (int)n, st))
    return EVR_ERR_CUDA;
  note_clock(s, clock);
  return EVR_OK;
}

int evr_push_events_device(evr_stream* s, const uint16_t* x, const uint16_t* y,
                           const int64_t* t_us, const int8_t* pol, size_t n) {
  Range range("evr_push_events_device");
  if (!s) return EVR_ERR_INVALID_ARG;
  if (n == 0) return EVR_OK;
  if (!x || !y || !t_us || !pol || n > (size_t)INT_MAX) return EVR_ERR_INVALID_ARG;
  if (launch_push(s->P, x, y, (const long long*)t_us, pol, (int)n, s->stream))
    return EVR_ERR_CUDA;
  s->h_clock_valid = false;
  return EVR_OK;
}

// The packet's front launches on stream q: TV-L1 of the time surface (if enabled) and
// the prologue (metric, f, cleared counts).
int enqueue_front(evr_stream* s, cudaStream_t q) {
  PrologueConsts pc = prologue_consts(s);
  if (s->prm.tvl1_iters > 0 && s->prm.manifold) {
    // denoise the time surface in the free buffer (1 - cur) and the ubar plane
    const int o = 1 - s->cur;
    if (launch_tvl1(s->P, pc, s->prm.tvl1_iters, s->prm.tvl1_lambda, s->P.u[o], s->P.p1[o],
                    s->P.p2[o], s->P.p3[o], s->P.ubar, q))
      return -1;
    pc.tau_plane = s->P.p1[o];
  }
  return launch_prologue(s->P, s->cur, pc, q) ? -1 : 0;
}

}  // extern "C"

namespace {
// Whether the packet's front launch (the prologue) can be fused into the first iteration
// pass: a kind-1 configuration without a register cap, f from the current u
// (data_mode 0), no TV-L1 plane, at least two passes.
bool front_fused(const evr_stream* s, int iters) {
  if (s->cfg < 0) return false;
  const SolverCfg& cfg = kSolverCfgs[s->cfg];
  if (s->prm.data_mode != 0 || (s->prm.tvl1_iters > 0 && s->prm.manifold)) return false;
  if (cfg.kind == 3) return cfg.R == 0 || (iters + cfg.R - 1) / cfg.R >= 2;
  if (cfg.kind == 5) return s->P.storage == 0;
  if (cfg.kind != 1 || !tiled_front_fusable(cfg, s->P.storage)) return false;  // kind 4 too
  return (iters + cfg.R - 1) / cfg.R >= 2;
}

// Whether the packet's push runs inside the solver's one launch (one cluster over the
// sensor, or the resident solver; front fused, a packet the single-launch push takes).
bool push_in_solver(const evr_stream* s, size_t n, int iters) {
  if (s->cfg < 0) return false;
  const SolverCfg& cfg = kSolverCfgs[s->cfg];
  if (cfg.kind == 5) return n > 0 && n <= (size_t)kTiledPushMax && front_fused(s, iters);
  return cfg.kind == 3 && cfg.R == 0 && n > 0 && n <= 32768 && front_fused(s, iters);
}
}  // namespace

extern "C" {

int evr_solve(evr_stream* s, int iters) {
  Range range("evr_solve");
  if (!s || iters < 0) return EVR_ERR_INVALID_ARG;
  cudaStream_t st = s->stream;
  // Once tuned, a multi-launch solve is one graph: front launches + iteration passes
  // (pass 0 is a programmatic dependent of the prologue).  The persistent solver takes
  // the front launches directly on the stream.
  const int front_launches =
      1 + ((s->prm.tvl1_iters > 0 && s->prm.manifold) ? 1 + 2 * s->prm.tvl1_iters : 0);
  if (iters == 0) return enqueue_front(s, st) ? EVR_ERR_CUDA : EVR_OK;
  bool front_done = false;
  if (!s->tuned) {  // the first solve: front launches, then the autotuner (untimed)
    if (enqueue_front(s, st)) return EVR_ERR_CUDA;
    autotune(s, iters);
    s->tuned = true;
    set_name(s);
    front_done = true;
  }
  // online refinement: this solve runs the next candidate, timed
  const bool refining = !front_done && s->n_cand > 1 && s->refine_done < s->n_cand * kRefineReps;
  if (refining) {
    const int r = s->refine_done;
    s->cfg = s->cand[r % s->n_cand];
    for (auto& e : s->ref_ev[r])
      if (!e && cudaEventCreate(&e) != cudaSuccess) return EVR_ERR_CUDA;
    if (cudaEventRecord(s->ref_ev[r][0], st) != cudaSuccess) return EVR_ERR_CUDA;
  }
  const bool direct_front = !front_done && s->cfg >= 0 && kSolverCfgs[s->cfg].kind == 2;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (s->timing) {
    if ((int)s->ev_used.size() >= kMaxTimingPairs) resolve_timing(s);
    if (s->ev_free.empty()) {
      cudaEventCreate(&ev.first);
      cudaEventCreate(&ev.second);
    } else {
      ev = s->ev_free.back();
      s->ev_free.pop_back();
    }
    cudaEventRecord(ev.first, st);
  }
  if (direct_front && enqueue_front(s, st)) return EVR_ERR_CUDA;
  const bool graph_front = !front_done && !direct_front;
  const bool fuse = graph_front && front_fused(s, iters);
  const PrologueConsts pc = prologue_consts(s);
  // launches inside the timed region: the front launches unless the first solve ran
  // them before the autotuner or they are fused into the first pass, then the
  // iteration kernels
  int launches = (front_done || fuse) ? 0 : front_launches;
  if (s->cfg >= 0 && kSolverCfgs[s->cfg].kind == 2) {
    if (run_cfg_direct(s, s->cfg, iters)) return EVR_ERR_CUDA;
    launches += 1;
  } else {
    GraphKey key{iters, s->cur, graph_front ? 1 : 0, s->cfg};
    auto it = s->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    int end_cur = s->cur;
    if (it == s->graphs.end()) {
      cudaGraph_t g = nullptr;
      int captured = 0;
      if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return EVR_ERR_CUDA;
      int r = (graph_front && !fuse) ? enqueue_front(s, s->cap_stream) : 0;
      if (r == 0)
        r = enqueue_iterations(s, iters, s->cur, s->cap_stream, &captured, fuse ? &pc : nullptr);
      cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
      if (r < 0 || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return EVR_ERR_CUDA;
      }
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return EVR_ERR_CUDA;
      s->graphs[key] = exec;
    } else {
      exec = it->second;
    }
    if (s->cfg < 0) {
      launches += 2 * iters;
    } else {
      const int passes = solve_passes(kSolverCfgs[s->cfg], iters);
      launches += solve_launches(kSolverCfgs[s->cfg], iters);
      end_cur = (passes % 2) ? 1 - s->cur : s->cur;
    }
    if (cudaGraphLaunch(exec, st) != cudaSuccess) return EVR_ERR_CUDA;
    s->cur = end_cur;
  }
  if (s->timing) {
    cudaEventRecord(ev.second, st);
    s->ev_used.push_back(ev);
    s->ev_launches.push_back(launches);
    s->ev_pixiters.push_back((long long)s->W * s->H * iters);
  }
  if (refining) {
    if (cudaEventRecord(s->ref_ev[s->refine_done][1], st) != cudaSuccess) return EVR_ERR_CUDA;
    if (++s->refine_done == s->n_cand * kRefineReps) {  // decide: fastest best-of-reps
      float best = 1e30f;
      int pick = s->cand[0];
      for (int c = 0; c < s->n_cand; ++c) {
        float t_min = 1e30f;
        for (int r = c; r < s->n_cand * kRefineReps; r += s->n_cand) {
          float ms = 0.f;
          if (cudaEventSynchronize(s->ref_ev[r][1]) != cudaSuccess ||
              cudaEventElapsedTime(&ms, s->ref_ev[r][0], s->ref_ev[r][1]) != cudaSuccess)
            return EVR_ERR_CUDA;
          if (ms < t_min) t_min = ms;
        }
        if (t_min < best) {
          best = t_min;
          pick = s->cand[c];
        }
      }
      s->cfg = pick;
      set_name(s);
    }
  }
  return EVR_OK;
}

}  // extern "C"

namespace {
// Whether a step runs as one fused graph: the solver is settled (tuned, refinement over),
// multi-launch, and the packet fits the one-CTA push.
bool fused_ok(const evr_stream* s, size_t n, int iters) {
  const bool refining = s->n_cand > 1 && s->refine_done < s->n_cand * kRefineReps;
  return n > 0 && n <= 32768 && iters > 0 && s->tuned && !refining &&
         !(s->cfg >= 0 && kSolverCfgs[s->cfg].kind == 2);
}

// One packet as one graph: push of the events at x, y, t, pol (device arrays), the front
// launches and the iteration kernels (the push inside the first launch where the solver
// takes it).  The graph is cached per (iters, buffer, push form, configuration); later
// calls update the node that pushes.
int fused_step(evr_stream* s, int iters, int n, const uint16_t* x, const uint16_t* y,
               const long long* t, const int8_t* pol) {
  cudaStream_t st = s->stream;
  const bool fuse = front_fused(s, iters);  // the prologue inside the first pass
  // one cluster over the sensor: the push runs inside the solver's single launch; a
  // multi-launch tiled solve with its front fused takes a small packet into pass 0
  const bool in_solver = push_in_solver(s, (size_t)n, iters);
  const bool in_pass0 = !in_solver && fuse && n <= kTiledPushMax &&
                        kSolverCfgs[s->cfg].kind == 1 &&
                        tiled_push_fusable(kSolverCfgs[s->cfg], s->P.storage);
  const PrologueConsts pc = prologue_consts(s);
  const PushArgs pa{x, y, t, pol, n};
  GraphKey key{iters, s->cur, in_pass0 ? 12 : 2, s->cfg};
  auto it = s->fused.find(key);
  evr_stream::Fused* fg = nullptr;
  if (it == s->fused.end()) {
    evr_stream::Fused nf;
    int captured = 0;
    if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return EVR_ERR_CUDA;
    int r = 0;
    if (in_solver && kSolverCfgs[s->cfg].kind == 5) {
      if (launch_resident(s->P, kSolverCfgs[s->cfg], s->cur, iters, solve_consts(s),
                          s->cap_stream, &pc, &pa))
        r = -1;
    } else if (in_solver) {
      if (r == 0 && launch_cluster(s->P, kSolverCfgs[s->cfg], s->cur, iters, 0,
                                   solve_consts(s), s->cap_stream, &pc, &pa))
        r = -1;
    } else if (in_pass0) {
      if (r == 0 && enqueue_iterations(s, iters, s->cur, s->cap_stream, &captured, &pc, &pa) < 0)
        r = -1;
    } else {
      if (r == 0 && launch_push(s->P, x, y, t, pol, n, s->cap_stream)) r = -1;
      if (r == 0 && !fuse) r = enqueue_front(s, s->cap_stream);
      // enqueue_iterations returns the buffer holding the result, or -1
      if (r == 0 && enqueue_iterations(s, iters, s->cur, s->cap_stream, &captured,
                                       fuse ? &pc : nullptr) < 0)
        r = -1;
    }
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &nf.graph);
    size_t roots = 1;
    cudaGraphNode_t root = nullptr;
    if (r == 0 && e == cudaSuccess) e = cudaGraphGetRootNodes(nf.graph, &root, &roots);
    if (r == 0 && e == cudaSuccess && roots == 1) nf.push = root;
    if (r == 0 && e == cudaSuccess && roots == 1) e = cudaGraphInstantiate(&nf.exec, nf.graph, 0);
    if (r < 0 || e != cudaSuccess || roots != 1 || !nf.exec) {
      if (nf.exec) cudaGraphExecDestroy(nf.exec);
      if (nf.graph) cudaGraphDestroy(nf.graph);
      return EVR_ERR_CUDA;
    }
    fg = &(s->fused[key] = nf);
  } else {
    fg = &it->second;
    if (in_solver && kSolverCfgs[s->cfg].kind == 5) {  // the resident launch's arguments
      if (resident_node_set_push(fg->exec, fg->push, s->P, kSolverCfgs[s->cfg], s->cur, iters,
                                 solve_consts(s), pc, pa))
        return EVR_ERR_CUDA;
    } else if (in_solver) {  // the cluster launch's arguments with this call's packet
      if (cluster_node_set_push(fg->exec, fg->push, s->P, kSolverCfgs[s->cfg], s->cur, iters,
                                solve_consts(s), pc, pa))
        return EVR_ERR_CUDA;
    } else if (in_pass0) {  // pass 0's arguments with this call's packet
      if (tiled_node_set_push(fg->exec, fg->push, s->P, kSolverCfgs[s->cfg], s->cur, iters,
                              solve_consts(s), pc, pa))
        return EVR_ERR_CUDA;
    } else {
      // this call's packet: the push node's arguments (Planes, x, y, t, pol, n)
      cudaKernelNodeParams kp;
      if (cudaGraphKernelNodeGetParams(fg->push, &kp) != cudaSuccess) return EVR_ERR_CUDA;
      void* args[6] = {(void*)&s->P, (void*)&x, (void*)&y, (void*)&t, (void*)&pol, (void*)&n};
      kp.kernelParams = args;
      kp.extra = nullptr;
      if (cudaGraphExecKernelNodeSetParams(fg->exec, fg->push, &kp) != cudaSuccess)
        return EVR_ERR_CUDA;
    }
  }
  const int passes = (s->cfg < 0) ? 0 : solve_passes(kSolverCfgs[s->cfg], iters);
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (s->timing) {
    if ((int)s->ev_used.size() >= kMaxTimingPairs) resolve_timing(s);
    if (s->ev_free.empty()) {
      cudaEventCreate(&ev.first);
      cudaEventCreate(&ev.second);
    } else {
      ev = s->ev_free.back();
      s->ev_free.pop_back();
    }
    cudaEventRecord(ev.first, st);
  }
  if (cudaGraphLaunch(fg->exec, st) != cudaSuccess) return EVR_ERR_CUDA;
  if (s->timing) {
    cudaEventRecord(ev.second, st);
    s->ev_used.push_back(ev);
    const int front =
        fuse ? 0 : 1 + ((s->prm.tvl1_iters > 0 && s->prm.manifold) ? 1 + 2 * s->prm.tvl1_iters : 0);
    s->ev_launches.push_back((in_solver || in_pass0 ? 0 : 1) + front +
                             (s->cfg < 0 ? 2 * iters : solve_launches(kSolverCfgs[s->cfg], iters)));
    s->ev_pixiters.push_back((long long)s->W * s->H * iters);
  }
  if (s->cfg >= 0 && passes % 2) s->cur = 1 - s->cur;
  return EVR_OK;
}
}  // namespace

extern "C" {

int evr_step_device(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
                    const int8_t* pol, size_t n, int iters) {
  Range range("evr_step_device");
  if (!s || iters < 0) return EVR_ERR_INVALID_ARG;
  if (n > 0 && (!x || !y || !t_us || !pol)) return EVR_ERR_INVALID_ARG;
  if (n > (size_t)INT_MAX) return EVR_ERR_INVALID_ARG;
  if (!fused_ok(s, n, iters)) {
    int rc = n ? evr_push_events_device(s, x, y, t_us, pol, n) : EVR_OK;
    return rc ? rc : evr_solve(s, iters);
  }
  int rc = fused_step(s, iters, (int)n, x, y, (const long long*)t_us, pol);
  if (rc == EVR_OK) s->h_clock_valid = false;
  return rc;
}

int evr_step(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
             const int8_t* pol, size_t n, int iters) {
  Range range("evr_step");
  if (!s || iters < 0) return EVR_ERR_INVALID_ARG;
  if (n > 0 && (!x || !y || !t_us || !pol)) return EVR_ERR_INVALID_ARG;
  if (n > (size_t)INT_MAX) return EVR_ERR_INVALID_ARG;
  if (!fused_ok(s, n, iters)) {
    int rc = n ? evr_push_events(s, x, y, t_us, pol, n) : EVR_OK;
    return rc ? rc : evr_solve(s, iters);
  }
  StageSlot* sl = nullptr;
  long long clock = 0;
  int rc = stage_host(s, x, y, t_us, pol, n, &sl, &clock);
  if (rc) return rc;
  if ((rc = ensure_slot_device(s, *sl, n)) != EVR_OK) return rc;
  const Packed L(n);
  // the packet's copy runs on the copy stream while earlier packets still solve; the
  // packet's graph (on the handle's stream) waits for it
  cudaError_t e =
      cudaMemcpyAsync(sl->d, sl->h, L.bytes, cudaMemcpyHostToDevice, s->h2d_stream);
  if (e == cudaSuccess) e = cudaEventRecord(sl->copied, s->h2d_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, sl->copied, 0);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  char* d = sl->d;
  rc = fused_step(s, iters, (int)n, (const uint16_t*)d, (const uint16_t*)(d + L.off_y),
                  (const long long*)(d + L.off_t), (const int8_t*)(d + L.off_p));
  if (rc) return rc;
  // the slot (pinned and device copies) is free again once this packet's graph has run
  if (cudaEventRecord(sl->done, s->stream) != cudaSuccess) return EVR_ERR_CUDA;
  sl->pending = true;
  note_clock(s, clock);
  return EVR_OK;
}

int evr_get_image(evr_stream* s, float* out_host, size_t len) {
  Range range("evr_get_image");
  if (!s || !out_host || len < (size_t)s->W * s->H) return EVR_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpy2DAsync(out_host, (size_t)s->W * 4, s->P.u[s->cur],
                                    (size_t)s->pitch * 4, (size_t)s->W * 4, s->H,
                                    cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  return sync_status(s);
}

int evr_get_image_async(evr_stream* s, float* out_host, size_t len, uint64_t* ticket) {
  Range range("evr_get_image_async");
  if (!s || !out_host || !ticket || len < (size_t)s->W * s->H) return EVR_ERR_INVALID_ARG;
  const size_t img = (size_t)s->W * s->H;
  if (!s->h_img_status) {
    if (host_alloc((void**)&s->h_img_status, sizeof(int) * kImgRing) != cudaSuccess) {
      s->h_img_status = nullptr;
      return EVR_ERR_OOM;
    }
    if (dev_alloc((void**)&s->d_img_stage, sizeof(float) * img * kImgStage) != cudaSuccess) {
      cudaFreeHost(s->h_img_status);
      s->h_img_status = nullptr;
      s->d_img_stage = nullptr;
      return EVR_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return EVR_ERR_CUDA;
    for (auto& e : s->img_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return EVR_ERR_CUDA;
    for (auto& e : s->stage_ready)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return EVR_ERR_CUDA;
  }
  const unsigned long long t = s->img_ticket + 1;
  const int slot = (int)(t % kImgRing), stage = (int)(t % kImgStage);
  float* dst = s->d_img_stage + (size_t)stage * img;
  // a ring slot is reused only after the readback that held it has completed
  if (cudaEventSynchronize(s->img_ev[slot]) != cudaSuccess) return EVR_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  // the staging image is reused once its previous host copy (ticket t - kImgStage) is done
  if (t > kImgStage)
    e = cudaStreamWaitEvent(s->stream, s->img_ev[(t - kImgStage) % kImgRing], 0);
  // on the handle's stream, in order with the solves: the image into staging, the status
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(dst, (size_t)s->W * 4, s->P.u[s->cur], (size_t)s->pitch * 4,
                          (size_t)s->W * 4, s->H, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->h_img_status[slot], &s->P.sc->status, sizeof(int),
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->stage_ready[stage], s->stream);
  // on the copy stream: staging to the host, then the ticket's event
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, s->stage_ready[stage], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_host, dst, sizeof(float) * img, cudaMemcpyDeviceToHost,
                        s->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->img_ev[slot], s->copy_stream);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  s->img_ticket = t;
  *ticket = t;
  return EVR_OK;
}

int evr_wait_image(evr_stream* s, uint64_t ticket) {
  Range range("evr_wait_image");
  if (!s || ticket == 0 || ticket > s->img_ticket) return EVR_ERR_INVALID_ARG;
  const int slot = (int)(ticket % kImgRing);
  // a slot recorded again since belongs to a later readback, which completes later
  if (cudaEventSynchronize(s->img_ev[slot]) != cudaSuccess) return EVR_ERR_CUDA;
  if (s->img_ticket - ticket < kImgRing && s->h_img_status[slot] != 0) return sync_status(s);
  return EVR_OK;
}

int evr_get_image_device(evr_stream* s, float* out_dev, size_t len) {
  if (!s || !out_dev || len < (size_t)s->W * s->H) return EVR_ERR_INVALID_ARG;
  return cuda_err(cudaMemcpy2DAsync(out_dev, (size_t)s->W * 4, s->P.u[s->cur],
                                    (size_t)s->pitch * 4, (size_t)s->W * 4, s->H,
                                    cudaMemcpyDeviceToDevice, s->stream));
}

static void* plane_ptr(evr_stream* s, int which, size_t* elem) {
  *elem = 4;
  switch (which) {
    case EVR_STATE_U: return s->P.u[s->cur];
    case EVR_STATE_P1: return s->P.p1[s->cur];
    case EVR_STATE_P2: return s->P.p2[s->cur];
    case EVR_STATE_P3: return s->P.p3[s->cur];
    case EVR_STATE_F: return s->P.f;
    case EVR_STATE_SQRTG: return s->P.sG;
    case EVR_STATE_TX: return s->P.tx;
    case EVR_STATE_TY: return s->P.ty;
    case EVR_STATE_NPOS: return s->P.npos;
    case EVR_STATE_NNEG: return s->P.nneg;
    case EVR_STATE_TLAST: *elem = 8; return s->P.t_last;
    default: return nullptr;
  }
}

int evr_get_state(evr_stream* s, int which, void* out_host, size_t bytes) {
  if (!s || !out_host) return EVR_ERR_INVALID_ARG;
  if (which == EVR_STATE_CLOCK || which == EVR_STATE_TINIT) {
    if (bytes != 8) return EVR_ERR_INVALID_ARG;
    int rc = sync_status(s);
    long long v = which == EVR_STATE_CLOCK ? s->h_sc->clock
                                           : (s->h_sc->t_init_set ? s->h_sc->t_init : 0);
    std::memcpy(out_host, &v, 8);
    return rc;
  }
  size_t elem = 0;
  void* src = plane_ptr(s, which, &elem);
  if (!src || bytes != elem * s->W * s->H) return EVR_ERR_INVALID_ARG;
  if (s->P.storage != 0 && which >= EVR_STATE_P1 && which <= EVR_STATE_P3) {
    // 16-bit p: widen into the (otherwise unused) ubar plane first
    if (launch_p_convert(s->P, src, s->P.ubar, 1, s->stream)) return EVR_ERR_CUDA;
    src = s->P.ubar;
  }
  cudaError_t e = cudaMemcpy2DAsync(out_host, elem * s->W, src, elem * s->pitch, elem * s->W,
                                    s->H, cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return EVR_ERR_CUDA;
  int rc = sync_status(s);
  if (which == EVR_STATE_TLAST) {
    long long t_init = s->h_sc->t_init_set ? s->h_sc->t_init : s->h_sc->clock;
    long long* v = (long long*)out_host;
    for (size_t i = 0; i < (size_t)s->W * s->H; ++i)
      if (v[i] == kNeverFired) v[i] = t_init;
  }
  return rc;
}

int evr_set_state(evr_stream* s, int which, const void* in_host, size_t bytes) {
  if (!s || !in_host) return EVR_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (which == EVR_STATE_CLOCK || which == EVR_STATE_TINIT) {
    if (bytes != 8) return EVR_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return EVR_ERR_CUDA;
    long long v;
    std::memcpy(&v, in_host, 8);
    if (which == EVR_STATE_CLOCK) {
      e = cudaMemcpy(&s->P.sc->clock, &v, 8, cudaMemcpyHostToDevice);
    } else {
      const int one = 1;
      e = cudaMemcpy(&s->P.sc->t_init, &v, 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(&s->P.sc->t_init_set, &one, 4, cudaMemcpyHostToDevice);
    }
    s->h_clock_valid = false;  // the host mirror refreshes at the next synchronising call
    return cuda_err(e);
  }
  const bool plane = (which >= EVR_STATE_U && which <= EVR_STATE_F) || which == EVR_STATE_TLAST ||
                     which == EVR_STATE_NPOS || which == EVR_STATE_NNEG;
  if (!plane) return EVR_ERR_INVALID_ARG;
  size_t elem = 0;
  void* dst = plane_ptr(s, which, &elem);
  if (bytes != elem * s->W * s->H) return EVR_ERR_INVALID_ARG;
  const bool narrow = s->P.storage != 0 && which >= EVR_STATE_P1 && which <= EVR_STATE_P3;
  e = cudaMemcpy2DAsync(narrow ? (void*)s->P.ubar : dst, elem * s->pitch, in_host, elem * s->W,
                        elem * s->W, s->H, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && narrow && launch_p_convert(s->P, dst, s->P.ubar, 0, s->stream))
    e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (which == EVR_STATE_TLAST || which == EVR_STATE_NPOS || which == EVR_STATE_NNEG)
    s->h_clock_valid = false;
  return cuda_err(e);
}

int evr_gap(evr_stream* s, double* primal, double* dual) {
  Range range("evr_gap");
  if (!s || !primal || !dual) return EVR_ERR_INVALID_ARG;
  if (launch_gap(s->P, s->cur, solve_consts(s), s->d_gap, s->stream)) return EVR_ERR_CUDA;
  if (cudaMemcpyAsync(s->h_gap, s->d_gap, 16, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return EVR_ERR_CUDA;
  int rc = sync_status(s);
  *primal = s->h_gap[0];
  *dual = s->h_gap[1];
  return rc;
}

int evr_synchronize(evr_stream* s) {
  Range range("evr_synchronize");
  if (!s) return EVR_ERR_INVALID_ARG;
  return sync_status(s);
}

int evr_enable_kernel_timing(evr_stream* s, int enable) {
  if (!s) return EVR_ERR_INVALID_ARG;
  resolve_timing(s);
  s->t_ms = 0.0;
  s->t_launches = 0;
  s->t_pixiters = 0;
  s->timing = enable != 0;
  return EVR_OK;
}

int evr_kernel_time(evr_stream* s, double* ms, int64_t* launches, int64_t* pixel_iters) {
  if (!s || !ms || !launches || !pixel_iters) return EVR_ERR_INVALID_ARG;
  resolve_timing(s);
  *ms = s->t_ms;
  *launches = s->t_launches;
  *pixel_iters = s->t_pixiters;
  return cuda_err(cudaGetLastError());
}

int evr_selftest_wait_timeout(evr_stream* s) {
  if (!s) return EVR_ERR_INVALID_ARG;
  int ci = -1;
  for (int k = 0; k < kNumSolverCfgs && ci < 0; ++k)
    if (kSolverCfgs[k].kind == 2 && solver_cfg_usable(s->P, kSolverCfgs[k]) &&
        solver_cfg_ctas(s->P, kSolverCfgs[k]) >= 2)
      ci = k;
  if (ci < 0) return EVR_ERR_NOT_SUPPORTED;
  int rc = sync_status(s);  // report nothing stale as the test's result
  if (rc != EVR_OK && rc != EVR_ERR_TIMEOUT) return rc;
  const size_t plane = (size_t)s->pitch * s->H * sizeof(float);
  float* save = nullptr;
  if (dev_alloc((void**)&save, 4 * plane) != cudaSuccess) return EVR_ERR_OOM;
  const int cur0 = s->cur;
  float* live[4] = {s->P.u[cur0], s->P.p1[cur0], s->P.p2[cur0], s->P.p3[cur0]};
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync((char*)save + k * plane, live[k], plane, cudaMemcpyDeviceToDevice, s->stream);
  clear_flags(s);
  const SolverCfg& cfg = kSolverCfgs[ci];
  // three passes, so every CTA waits on its neighbours at least twice
  int e = launch_persistent(s->P, cfg, cur0, 3 * cfg.R, 0, solve_consts(s), s->stream, 0);
  rc = e ? EVR_ERR_CUDA : sync_status(s);  // clears status, flags and abort on a timeout
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync(live[k], (char*)save + k * plane, plane, cudaMemcpyDeviceToDevice, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaFree(save);
  clear_flags(s);
  s->cur = cur0;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return EVR_ERR_CUDA;
  return rc;
}

int evr_selftest_resident_wait_timeout(evr_stream* s) {
  if (!s) return EVR_ERR_INVALID_ARG;
  int ci = -1;  // a resident configuration of at least two CTAs that fits the sensor
  for (int k = 0; k < kNumSolverCfgs && ci < 0; ++k)
    if (kSolverCfgs[k].kind == 5 && solver_cfg_usable(s->P, kSolverCfgs[k]) &&
        solver_cfg_ctas(s->P, kSolverCfgs[k]) >= 2)
      ci = k;
  if (ci < 0) return EVR_ERR_NOT_SUPPORTED;
  int rc = sync_status(s);  // report nothing stale as the test's result
  if (rc != EVR_OK && rc != EVR_ERR_TIMEOUT) return rc;
  const size_t plane = (size_t)s->pitch * s->H * sizeof(float);
  float* save = nullptr;
  if (dev_alloc((void**)&save, 4 * plane) != cudaSuccess) return EVR_ERR_OOM;
  const int cur0 = s->cur;
  float* live[4] = {s->P.u[cur0], s->P.p1[cur0], s->P.p2[cur0], s->P.p3[cur0]};
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync((char*)save + k * plane, live[k], plane, cudaMemcpyDeviceToDevice, s->stream);
  const SolverCfg& cfg = kSolverCfgs[ci];
  // the barrier's arrival word starts far below any target (every byte 0x80: a large
  // negative count), so the first barrier's wait runs out in every CTA
  cudaError_t ce = cudaMemsetAsync(s->P.flags + kMaxCtas, 0x80, sizeof(int), s->stream);
  int e = ce != cudaSuccess ? 1
                            : launch_resident(s->P, cfg, cur0, 2 * cfg.R, solve_consts(s),
                                              s->stream, nullptr, nullptr);
  rc = e ? EVR_ERR_CUDA : sync_status(s);  // reads and clears the status and the flags
  if (rc != EVR_ERR_TIMEOUT && clear_flags(s) != EVR_OK) rc = EVR_ERR_CUDA;
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync(live[k], (char*)save + k * plane, plane, cudaMemcpyDeviceToDevice, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaFree(save);
  s->cur = cur0;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return EVR_ERR_CUDA;
  return rc;
}

int evr_selftest_cluster_wait_timeout(evr_stream* s) {
  if (!s) return EVR_ERR_INVALID_ARG;
  int ci = -1;  // a cluster configuration of at least two CTAs that fits the sensor
  for (int k = 0; k < kNumSolverCfgs && ci < 0; ++k)
    if (kSolverCfgs[k].kind == 3 && kSolverCfgs[k].cx * kSolverCfgs[k].cy >= 2 &&
        solver_cfg_usable(s->P, kSolverCfgs[k]))
      ci = k;
  if (ci < 0) return EVR_ERR_NOT_SUPPORTED;
  int rc = sync_status(s);  // report nothing stale as the test's result
  if (rc != EVR_OK && rc != EVR_ERR_TIMEOUT) return rc;
  const size_t plane = (size_t)s->pitch * s->H * sizeof(float);
  float* save = nullptr;
  if (dev_alloc((void**)&save, 4 * plane) != cudaSuccess) return EVR_ERR_OOM;
  const int cur0 = s->cur;
  float* live[4] = {s->P.u[cur0], s->P.p1[cur0], s->P.p2[cur0], s->P.p3[cur0]};
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync((char*)save + k * plane, live[k], plane, cudaMemcpyDeviceToDevice, s->stream);
  const SolverCfg& cfg = kSolverCfgs[ci];
  // rank 0 of every cluster sends nothing: its neighbours' waits for its edges run out
  const int iters = cfg.R > 0 ? cfg.R : 3;
  int e = launch_cluster(s->P, cfg, cur0, iters, 2, solve_consts(s), s->stream, nullptr,
                         nullptr, 0);
  rc = e ? EVR_ERR_CUDA : sync_status(s);  // reads and clears the status
  for (int k = 0; k < 4; ++k)
    cudaMemcpyAsync(live[k], (char*)save + k * plane, plane, cudaMemcpyDeviceToDevice, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaFree(save);
  s->cur = cur0;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return EVR_ERR_CUDA;
  return rc;
}

const char* evr_solver_name(evr_stream* s) { return s ? s->name : ""; }

int evr_solver_settled(evr_stream* s) {
  if (!s) return EVR_ERR_INVALID_ARG;
  const bool refining = s->n_cand > 1 && s->refine_done < s->n_cand * kRefineReps;
  return (s->tuned && !refining) ? 1 : 0;
}

int evr_test_fail_alloc_after(int n) {
  g_fail_countdown.store(n > 0 ? n : 0);
  return EVR_OK;
}

const char* evr_strerror(int code) {
  switch (code) {
    case EVR_OK: return "ok";
    case EVR_ERR_INVALID_ARG: return "invalid argument";
    case EVR_ERR_OUT_OF_RANGE: return "event outside the sensor";
    case EVR_ERR_BAD_POLARITY: return "event with polarity 0";
    case EVR_ERR_NONMONOTONIC: return "event timestamp decreases";
    case EVR_ERR_OOM: return "out of memory";
    case EVR_ERR_CUDA: return "CUDA error";
    case EVR_ERR_TIMEOUT: return "device wait timed out";
    case EVR_ERR_NOT_SUPPORTED: return "no sm_103a device or option not built";
    default: return "unknown error";
  }
}

}  // extern "C"
