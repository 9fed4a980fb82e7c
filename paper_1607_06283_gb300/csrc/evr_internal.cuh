// evr_internal.cuh -- device-side layout shared by the library's translation units.
//
// HBM layout of one stream (all planes W x H with a row pitch of `pitch` elements,
// pitch = W rounded up to a multiple of 32, so every row starts on a 128-byte line):
//   u[2], p1[2], p2[2], p3[2]   float  iterated state, ping-pong buffers (tiled solver)
//   ubar                        float  extrapolated primal (unfused solver only)
//   f, tx, ty, iG, sG           float  per-packet data image and metric (1/G, sqrt G)
//   t_last                      int64  surface of active events (sentinel: never fired)
//   npos, nneg                  int32  event counts since the last solve
//   sc                          DevScalars (clock, t_init, status)
//   partials                    double gap-reduction partial sums
#pragma once
#include <cstdint>

namespace evr {

constexpr long long kNeverFired = (-9223372036854775807LL - 1);  // INT64_MIN

struct DevScalars {
  long long clock;   // latest timestamp seen (stream clock)
  long long t_init;  // timestamp of never-fired pixels (valid when t_init_set)
  int t_init_set;
  int status;        // first device-side error code (rejection or timeout), 0 if none
  int first_bad;     // multi-CTA validation: lowest index of an invalid event
  int abort;         // persistent solver: set by a CTA whose neighbour wait timed out
  // a packet integrated inside the first tiled pass (every CTA reads the clock there):
  // its clock and t_init, committed by the second pass
  long long clock_next, t_init_next;
  int commit_pending;
};

// Persistent solver: at most this many CTAs (one progress flag each).
constexpr int kMaxCtas = 1024;

struct Planes {
  int W, H, pitch;
  int Hm;  // rows per image: H for a stream; n images of Hm rows stacked into H = n Hm
           // rows are independent (no forward difference across an image's last row)
  float* u[2];
  float* p1[2];
  float* p2[2];
  float* p3[2];
  float* ubar;
  float* f;
  float* tx;
  float* ty;
  float* iG;
  float* sG;
  long long* t_last;
  int* npos;
  int* nneg;
  DevScalars* sc;
  double* partials;
  int* flags;  // persistent solver: passes completed by each CTA (monotonic), then the
               // resident solver's barrier words (arrivals, leaves): kMaxCtas + 2 ints
  int storage; // format of the p planes: 0 FP32, 1 FP16, 2 BF16 (tiled solver only)
};

// Batched streams: per-stream plane descriptors and work items on the device.  A
// kernel given a null `descs` works on the single stream passed by value.
struct BatchRef {
  const Planes* descs;  // per-stream planes, or null
  const int2* work;     // work item per CTA: (stream, tile or block index)
  const int* curs;      // per-stream buffer holding the current (u, p)
  const int* active;    // per-stream: 1 when the stream has a packet in this step
};

// Copy a stream's plane descriptor (a __grid_constant__ kernel parameter or an element of
// a device array) into shared memory with the 32 lanes of one warp, word by word: the
// copy by a single thread was a serial chain of loads (about 1 us on GB300) that every CTA
// of every pass waited for at its first barrier.
__device__ __forceinline__ void stage_planes(Planes* dst, const Planes* src, int lane) {
  static_assert(sizeof(Planes) % 4 == 0, "the descriptor is copied in 4-byte words");
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int i = lane; i < (int)(sizeof(Planes) / 4); i += 32) d[i] = s[i];
}

struct SolveConsts {
  float tau, sigma, lambda, u_min, u_max;
  int data_term;  // 0 KL with box, 1 L2 (Eq. 7)
};

struct PrologueConsts {
  float time_scale, delta_pos, delta_neg;
  long long t_max_us;
  int manifold, data_mode;
  const float* tau_plane;  // denoised time surface (pitched), or null: from t_last
};

// Per-pixel arithmetic of the packet prologue, shared by the prologue kernel and by a
// first iteration pass that computes the packet's constants itself, so that both give
// the same bits (the operation order is fixed by explicit fmaf).
#ifdef __CUDACC__
// Time surface (time since the pixel's last event, Sec. 3.1), scaled and clamped.
__device__ __forceinline__ float time_surface(long long tl, long long clock, long long t_init,
                                              const PrologueConsts& c) {
  if (!c.manifold) return 0.0f;
  long long last = (tl == kNeverFired) ? t_init : tl;
  long long d = clock - last;
  if (c.t_max_us > 0 && d > c.t_max_us) d = c.t_max_us;
  return __fmul_rn((float)d, c.time_scale);
}
// forward difference of the time surface (a subtraction that is never contracted)
__device__ __forceinline__ float surface_diff(float t1, float t0) { return __fsub_rn(t1, t0); }
// G = 1 + t_x^2 + t_y^2 (text after Eq. 3)
__device__ __forceinline__ float metric_G(float a, float b) {
  return fmaf(b, b, fmaf(a, a, 1.0f));
}
// f = base exp(Delta+ n+ - Delta- n-) (Eq. intensity_update, compounded)
__device__ __forceinline__ float data_image(float base, int np, int nn,
                                           const PrologueConsts& c) {
  return __fmul_rn(base, expf(fmaf(c.delta_pos, (float)np, -(c.delta_neg * (float)nn))));
}
#endif

// A packet of n events (device arrays) that a solver launch integrates itself.
struct PushArgs {
  const uint16_t *x, *y;
  const long long* t;
  const int8_t* pol;
  int n;
};

// Tiled solvers.  A tile template is an extended tile of EW x EH pixels (an owned
// tile plus an R-pixel halo on every side) processed by 32 x NTY threads.  A solver
// configuration is a template, a halo width R and a kind:
//   kind 1: one launch per R iterations (state in HBM/L2 between launches);
//   kind 2: one cooperative launch per packet, state in registers, R-wide halo bands
//           exchanged with the 8 neighbouring CTAs through L2 every R iterations;
//   kind 3: thread-block clusters of cx x cy CTAs whose tiles form one super-tile; the
//           CTAs exchange their edge values every iteration through distributed shared
//           memory, and only the super-tile carries an R-pixel halo.  R = 0: one cluster
//           covers the sensor and runs every iteration of a packet (with the packet's
//           push and prologue) in one launch;
//   kind 4: as kind 1, with a persistent grid whose CTAs walk the tiles and stage each
//           tile's planes in shared memory with tensor copies, one tile ahead.
struct TileShape {
  int EW, EH, NTY;
};
struct SolverCfg {
  int kind, shape, R;
  int cx, cy;  // kind 3: cluster shape in CTAs
};
constexpr int kNumTileShapes = 8;
extern const TileShape kTileShapes[kNumTileShapes];
constexpr int kNumSolverCfgs = 80;
extern const SolverCfg kSolverCfgs[kNumSolverCfgs];

constexpr int kGapBlocks = 304;   // fixed: the reduction order does not depend on W, H
constexpr int kGapThreads = 256;

// host helpers shared by the single-stream and batched runtimes (evr_api.cu)
size_t state_bytes(int W, int H, bool solo);
char* carve_state(char* base, int W, int H, bool solo, Planes* out);
int check_device();

// kernel launchers (evr_kernels.cu); all return cudaError_t as int
int launch_init(const Planes& P, float u_init, long long clock0, long long t_init, int t_init_set,
                void* stream);
// Library allocations (device and page-locked host memory) go through these, so that a
// test can make the n-th next one fail (evr_test_fail_alloc_after).
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc(void** p, size_t bytes);

int launch_push(const Planes& P, const uint16_t* x, const uint16_t* y, const long long* t,
                const int8_t* pol, int n, void* stream);
int launch_prologue(const Planes& P, int cur, const PrologueConsts& c, void* stream);
// Anisotropic TV-L1 denoising of the time surface (Sec. 4) into s (pitched plane),
// with scratch planes t0, q1, q2, sbar; K iterations from s = t0, q = 0.
int launch_tvl1(const Planes& P, const PrologueConsts& c, int K, float lam, float* t0, float* s,
                float* q1, float* q2, float* sbar, void* stream);
// Batched: one CTA of 32 x 8 threads per work item (stream, block); blocks of a W x H
// stream are numbered by = b / ceil(W/32), bx = b % ceil(W/32).
int launch_prologue_batch(const BatchRef& B, int n_work, const PrologueConsts& c, void* stream);
// Batched push: CTA s validates and commits stream s's events
// [offsets[s], offsets[s+1]) and sets active[s] = (count > 0).
int launch_push_batch(const Planes* descs, int n_streams, const uint16_t* x, const uint16_t* y,
                      const long long* t, const int8_t* pol, const long long* offsets,
                      int* active, void* stream);
// Batched buffer flip after `passes` tiled passes: curs[s] ^= passes & 1 for active s.
int launch_batch_flip(int* curs, const int* active, int n_streams, int passes, void* stream);
int launch_unfused_iteration(const Planes& P, int cur, const SolveConsts& c, void* stream);
// kind 1: `iters` <= R iterations from buffer src into buffer 1 - src; `pass` is the
// pass's index within the packet (0 right after the prologue).
// With front != NULL the packet's front launches are fused into the passes: pass 0
// computes the prologue's constants itself (data_mode 0, no TV-L1 plane) and pass 1
// clears the event counts; the caller runs at least two passes.
int launch_tiled_pass(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
                      const SolveConsts& c, void* stream, const PrologueConsts* front = nullptr,
                      const PushArgs* push = nullptr);
// With front and push (FP32 tiles that fuse the front, packets of at most
// kTiledPushMax events): pass 0 also validates and integrates the packet itself -- every
// CTA scans it and merges the events of its extended tile from a shared-memory map, the
// owned pixels' t_last is written back, and pass 1 commits the stream clock.  The
// pass-0 node of a captured graph of an `iters`-iteration solve takes a new packet
// through tiled_node_set_push.
constexpr int kTiledPushMax = 2048;
bool tiled_push_fusable(const SolverCfg& cfg, int storage);
int tiled_node_set_push(void* graph_exec, void* node, const Planes& P, const SolverCfg& cfg,
                        int src, int iters, const SolveConsts& c, const PrologueConsts& front,
                        const PushArgs& push);
// Whether launch_tiled_pass supports a fused front for this configuration and storage
// (tiles without a register cap).
int tiled_front_fusable(const SolverCfg& cfg, int storage);
// The unrolled solve's passes (FP32, the 32 x 32 tile with one pixel pair per thread and
// an R-pixel halo): `iters` <= R iterations from buffer src into 1 - src; with a tape,
// iteration it also writes the p it starts from, its primal argument v and its ubar
// into tape slot tape_first + it (planes p1 p2 p3 v ubar of tape_plane floats).
constexpr int kTapeKX = 1, kTapeKY = 2, kTapeNTY = 16;
int launch_tiled_tape(const Planes& P, int R, int src, int iters, int pass,
                      const SolveConsts& c, float* tape, long long tape_plane, int tape_first,
                      void* stream);
// kind 1 over a batch: one CTA per work item (stream, tile); pass j of a step reads
// buffer curs[s] ^ (j & 1).  Inactive streams are skipped.
int launch_tiled_pass_batch(const BatchRef& B, int n_work, const SolverCfg& cfg, int pass,
                            int iters, const SolveConsts& c, int storage, void* stream);
// kind 2: all `iters` iterations from buffer cur; the result lands in buffer
// cur ^ (ceil(iters / R) & 1).  `base` is the value of every CTA's progress flag at
// launch (flags cleared by the host start at 0; each launch adds passes - 1).
// Returns cudaErrorCooperativeLaunchTooLarge when the grid cannot be co-resident.
// silent_cta >= 0 (wait self-test only): that CTA never publishes its progress flag, so
// its neighbours' bounded waits run out and the launch ends with EVR_ERR_TIMEOUT.
int launch_persistent(const Planes& P, const SolverCfg& cfg, int cur, int iters, int base,
                      const SolveConsts& c, void* stream, int silent_cta = -1);
// kind 5: one cooperative launch of all `iters` iterations from buffer cur; the result
// lands in buffer cur ^ (ceil(iters / R) & 1).  front != NULL: the packet's front is
// computed in the launch and the event counts are cleared (data_mode 0, no TV-L1 plane);
// push != NULL as well: the launch first validates and integrates the packet (n <=
// kTiledPushMax) and commits the stream clock.  FP32 storage; needs the solo state's
// flags (two barrier words after kMaxCtas progress flags).  Returns
// cudaErrorCooperativeLaunchTooLarge when the grid cannot be co-resident.
int launch_resident(const Planes& P, const SolverCfg& cfg, int cur, int iters,
                    const SolveConsts& c, void* stream, const PrologueConsts* front,
                    const PushArgs* push);
// Updates the kernel node of an instantiated graph, captured by launch_resident with a
// push, to push the packet `push` instead (all other arguments as captured).
int resident_node_set_push(void* graph_exec, void* node, const Planes& P, const SolverCfg& cfg,
                           int cur, int iters, const SolveConsts& c, const PrologueConsts& front,
                           const PushArgs& push);
// kind 3 (evr_cluster.cu): `iters` iterations from buffer src into 1 - src, at most R per
// launch (R = 0: all of them).  front != NULL: the packet's front is fused (R = 0: the
// one launch computes the prologue's constants and clears the event counts; R > 0: as
// kind 1, pass 0 computes them and pass 1 clears the counts).  push != NULL (R = 0 only):
// the launch first validates and integrates the packet x, y, t, pol of n events
// (n <= 32768).  silent_rank >= 0 (wait self-test only): that CTA of the cluster sends
// nothing, so its neighbours' bounded waits run out and the launch ends with
// EVR_ERR_TIMEOUT.
int launch_cluster(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
                   const SolveConsts& c, void* stream, const PrologueConsts* front,
                   const PushArgs* push, int silent_rank = -1);
// Updates the kernel node `node` of an instantiated graph, captured by launch_cluster with
// a push, to push the packet `push` instead (all other arguments as captured).
int cluster_node_set_push(void* graph_exec, void* node, const Planes& P, const SolverCfg& cfg,
                          int src, int iters, const SolveConsts& c, const PrologueConsts& front,
                          const PushArgs& push);
bool cluster_cfg_usable(const Planes& P, const SolverCfg& cfg);
int cluster_cfg_ctas(const Planes& P, const SolverCfg& cfg);
// kind 4 (evr_staged.cu, FP32): a persistent pass of `iters` <= R iterations from buffer
// src into 1 - src whose CTAs stage each tile's planes with tensor copies one tile ahead
// (the packet's prologue runs as its own launch before the first pass).
int launch_staged(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
                  const SolveConsts& c, void* stream);
bool staged_cfg_usable(const Planes& P, const SolverCfg& cfg);
int staged_cfg_ctas(const Planes& P, const SolverCfg& cfg);

// Whether the configuration can run on this sensor (tile fits, grid co-resident).
bool solver_cfg_usable(const Planes& P, const SolverCfg& cfg);
int solver_cfg_ctas(const Planes& P, const SolverCfg& cfg);
int launch_gap(const Planes& P, int cur, const SolveConsts& c, double* out2, void* stream);
// Convert one pitched plane between the p storage format (P.storage) and FP32:
// to_f32 = 1 widens p_plane into f_plane, 0 narrows f_plane into p_plane.
int launch_p_convert(const Planes& P, void* p_plane, float* f_plane, int to_f32, void* stream);

}  // namespace evr
