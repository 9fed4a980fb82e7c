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
  int status;        // first device-side rejection code, 0 if none
  int first_bad;     // multi-CTA validation: lowest index of an invalid event
  int pad;
};

struct Planes {
  int W, H, pitch;
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
};

struct SolveConsts {
  float tau, sigma, lambda, u_min, u_max;
};

struct PrologueConsts {
  float time_scale, delta_pos, delta_neg;
  long long t_max_us;
  int manifold, data_mode;
};

// Tiled-solver shapes: extended tile EW x EH (owned tile plus an R-pixel halo on
// every side), 32 x NTY threads, R iterations per launch.
struct TileShape {
  int EW, EH, NTY, R;
};

constexpr int kNumTileShapes = 16;
extern const TileShape kTileShapes[kNumTileShapes];

constexpr int kGapBlocks = 304;   // fixed: the reduction order does not depend on W, H
constexpr int kGapThreads = 256;

// kernel launchers (evr_kernels.cu); all return cudaError_t as int
int launch_init(const Planes& P, float u_init, long long clock0, long long t_init, int t_init_set,
                void* stream);
int launch_push(const Planes& P, const uint16_t* x, const uint16_t* y, const long long* t,
                const int8_t* pol, int n, void* stream);
int launch_prologue(const Planes& P, int cur, const PrologueConsts& c, void* stream);
int launch_unfused_iteration(const Planes& P, int cur, const SolveConsts& c, void* stream);
int launch_tiled_pass(const Planes& P, int shape, int src, int iters, const SolveConsts& c,
                      void* stream);
int tiled_pass_blocks(const Planes& P, int shape);
int launch_gap(const Planes& P, int cur, const SolveConsts& c, double* out2, void* stream);

}  // namespace evr
