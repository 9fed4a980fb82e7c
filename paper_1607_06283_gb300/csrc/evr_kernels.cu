// evr_kernels.cu -- sm_103a kernels of the event-manifold reconstruction, except
// the tiled solvers (evr_solvers.cu).
//
// Reinbacher, Graber, Pock, BMVC 2016.  Per packet: event scatter (Sec. 3, Sec. 3.1),
// prologue (time surface, metric of Eq. 2 / Eq. 3, data image of Eq.
// intensity_update), then primal-dual iterations (Eq. cont_iterates, Eq.
// update_rules).  The unfused iteration here uses IEEE division and square root in
// FP32; the FP64 gap reduction is the convergence check.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>

#include "evr_internal.cuh"
#include "evr_push.cuh"

namespace evr {


// ---------------------------------------------------------------- pointwise maps
// L_g u at one pixel from the forward differences (ux, uy) (Eq. 3), with
// a = L_x t, b = L_y t, iG = 1/G.  Written as M (ux, uy) with
// M = (1/G) [[1+b^2, -ab], [-ab, 1+a^2], [a, b]].
__device__ __forceinline__ void apply_M(float a, float b, float iG, float ux, float uy, float& g1,
                                        float& g2, float& g3) {
  float w = b * ux - a * uy;
  g1 = iG * (ux + b * w);
  g2 = iG * (uy - a * w);
  g3 = iG * (a * ux + b * uy);
}

// M^T p: the vector field whose ordinary divergence is div_g p = -L_g^* p.
__device__ __forceinline__ void apply_MT(float a, float b, float iG, float p1, float p2, float p3,
                                         float& q1, float& q2) {
  float z = b * p1 - a * p2;
  q1 = iG * (p1 + b * z + a * p3);
  q2 = iG * (p2 - a * z + b * p3);
}

// Closed-form KL proximal root with clamping (Eq. update_rules, first line):
// 1/2 (v - beta + sqrt((v - beta)^2 + 4 beta f)).  For v - beta < 0 the same root is
// evaluated as 2 beta f / (sqrt(...) - (v - beta)), which avoids the cancellation of
// two nearly equal terms when beta >> v.
__device__ __forceinline__ float prox_kl(float v, float beta, float f, float umin, float umax) {
  float d = v - beta;
  float bf = beta * f;
  float disc = sqrtf(d * d + 4.0f * bf);
  float r = (d >= 0.0f) ? 0.5f * (d + disc) : (2.0f * bf) / (disc - d);
  return fminf(fmaxf(r, umin), umax);
}

// Projection onto the metric ball |p| <= sqrt(G) (Eq. update_rules, second line).
__device__ __forceinline__ void project(float& p1, float& p2, float& p3, float sG) {
  float nrm = sqrtf(p1 * p1 + p2 * p2 + p3 * p3);
  float den = fmaxf(1.0f, nrm / sG);
  p1 = p1 / den;
  p2 = p2 / den;
  p3 = p3 / den;
}

// ---------------------------------------------------------------- initialisation
__global__ void k_init(Planes P, float u_init, long long clock0, long long t_init, int t_init_set) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x == 0 && y == 0) {
    P.sc->clock = clock0;
    P.sc->t_init = t_init;
    P.sc->t_init_set = t_init_set;
    P.sc->status = 0;
    P.sc->first_bad = INT_MAX;
    P.sc->abort = 0;
    P.sc->clock_next = clock0;
    P.sc->t_init_next = t_init;
    P.sc->commit_pending = 0;
  }
  if (P.flags && y == 0 && x < kMaxCtas) P.flags[x] = 0;  // solo streams only
  if (x >= P.pitch || y >= P.H) return;
  size_t i = (size_t)y * P.pitch + x;
  for (int b = 0; b < 2; ++b) {
    P.u[b][i] = u_init;
    P.p1[b][i] = 0.0f;
    P.p2[b][i] = 0.0f;
    P.p3[b][i] = 0.0f;
  }
  P.ubar[i] = u_init;
  P.f[i] = u_init;
  P.tx[i] = 0.0f;
  P.ty[i] = 0.0f;
  P.iG[i] = 1.0f;
  P.sG[i] = 1.0f;
  P.t_last[i] = kNeverFired;
  P.npos[i] = 0;
  P.nneg[i] = 0;
}

int launch_init(const Planes& P, float u_init, long long clock0, long long t_init, int t_init_set,
                void* stream) {
  int gx = (P.pitch > kMaxCtas ? P.pitch : kMaxCtas);
  dim3 blk(32, 8), grd((gx + 31) / 32, (P.H + 7) / 8);
  k_init<<<grd, blk, 0, (cudaStream_t)stream>>>(P, u_init, clock0, t_init, t_init_set);
  return (int)cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_push_one_cta(Planes P, const uint16_t* __restrict__ x,
                                                       const uint16_t* __restrict__ y,
                                                       const long long* __restrict__ t,
                                                       const int8_t* __restrict__ pol, int n) {
  // a programmatically dependent prologue may launch now: it waits for this grid's
  // completion (griddepcontrol.wait) before reading anything this kernel writes
  asm volatile("griddepcontrol.launch_dependents;" :::);
  push_cta(P, x, y, t, pol, n, threadIdx.x, blockDim.x);
}

constexpr int kErrInvalidArg = -1;
constexpr int kMaxBatchPacket = 32768;

// Batched push: CTA s handles stream s.  Packets above kMaxBatchPacket events are
// rejected with EVR_ERR_INVALID_ARG (state unchanged).
__global__ void __launch_bounds__(1024) k_push_batch(const Planes* __restrict__ descs,
                                                     const uint16_t* __restrict__ x,
                                                     const uint16_t* __restrict__ y,
                                                     const long long* __restrict__ t,
                                                     const int8_t* __restrict__ pol,
                                                     const long long* __restrict__ offsets,
                                                     int* active) {
  const int s = blockIdx.x;
  const long long a = offsets[s], b = offsets[s + 1];
  const Planes& P = descs[s];
  if (threadIdx.x == 0) active[s] = b > a ? 1 : 0;
  if (b <= a) return;
  if (b - a > kMaxBatchPacket) {
    if (threadIdx.x == 0) atomicCAS(&P.sc->status, 0, kErrInvalidArg);
    return;
  }
  push_cta(P, x + a, y + a, t + a, pol + a, (int)(b - a), threadIdx.x, blockDim.x);
}

int launch_push_batch(const Planes* descs, int n_streams, const uint16_t* x, const uint16_t* y,
                      const long long* t, const int8_t* pol, const long long* offsets,
                      int* active, void* stream) {
  if (n_streams <= 0) return 0;
  k_push_batch<<<n_streams, 1024, 0, (cudaStream_t)stream>>>(descs, x, y, t, pol, offsets,
                                                             active);
  return (int)cudaGetLastError();
}

__global__ void k_batch_flip(int* curs, const int* active, int n, int passes) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && active[s] && (passes & 1)) curs[s] ^= 1;
}

int launch_batch_flip(int* curs, const int* active, int n_streams, int passes, void* stream) {
  if (n_streams <= 0) return 0;
  k_batch_flip<<<(n_streams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(curs, active,
                                                                          n_streams, passes);
  return (int)cudaGetLastError();
}

// Large packets: grid-wide validation, then a commit kernel that checks the result.
__global__ void k_push_validate(Planes P, const uint16_t* __restrict__ x,
                                const uint16_t* __restrict__ y, const long long* __restrict__ t,
                                const int8_t* __restrict__ pol, int n) {
  long long clock = P.sc->clock;
  int have = P.sc->t_init_set;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (event_code(x, y, t, pol, i, P.W, P.H, clock, have) != 0) atomicMin(&P.sc->first_bad, i);
}

__global__ void k_push_commit(Planes P, const uint16_t* __restrict__ x,
                              const uint16_t* __restrict__ y, const long long* __restrict__ t,
                              const int8_t* __restrict__ pol, int n) {
  int bad = P.sc->first_bad;
  if (bad < n) return;
  int first = blockIdx.x * blockDim.x + threadIdx.x;
  commit_events(P, x, y, t, pol, n, first, gridDim.x * blockDim.x);
}

// Finishes a large push: records the rejection, or advances the clock; re-arms
// first_bad for the next push.
__global__ void k_push_finish(Planes P, const uint16_t* __restrict__ x,
                              const uint16_t* __restrict__ y, const long long* __restrict__ t,
                              const int8_t* __restrict__ pol, int n) {
  int bad = P.sc->first_bad;
  long long clock = P.sc->clock;
  int have = P.sc->t_init_set;
  if (bad < n) {
    atomicCAS(&P.sc->status, 0, event_code(x, y, t, pol, bad, P.W, P.H, clock, have));
  } else {
    if (!have) {
      P.sc->t_init = t[0];
      P.sc->t_init_set = 1;
    }
    P.sc->clock = t[n - 1] > clock ? t[n - 1] : clock;
  }
  P.sc->first_bad = INT_MAX;
}

int launch_push(const Planes& P, const uint16_t* x, const uint16_t* y, const long long* t,
                const int8_t* pol, int n, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (n <= 0) return 0;
  if (n <= 32768) {
    k_push_one_cta<<<1, 1024, 0, st>>>(P, x, y, t, pol, n);
  } else {
    int blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    k_push_validate<<<blocks, 256, 0, st>>>(P, x, y, t, pol, n);
    k_push_commit<<<blocks, 256, 0, st>>>(P, x, y, t, pol, n);
    k_push_finish<<<1, 1, 0, st>>>(P, x, y, t, pol, n);
  }
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- packet prologue

// One pixel of the prologue (block `blk` of the stream's 32 x 8 blocks).
__device__ __forceinline__ void prologue_px_body(const Planes& P, int cur, const PrologueConsts& c,
                                                 int blk) {
  const int nbx = (P.W + 31) / 32;
  const int x = (blk % nbx) * 32 + threadIdx.x;
  const int y = (blk / nbx) * 8 + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  long long clock = P.sc->clock;
  long long t_init = P.sc->t_init_set ? P.sc->t_init : clock;
  size_t i = (size_t)y * P.pitch + x;
  float a, b;
  if (c.tau_plane) {  // surface denoised beforehand (TV-L1)
    const float* T = c.tau_plane;
    a = (x < P.W - 1) ? T[i + 1] - T[i] : 0.0f;
    b = (y < P.H - 1) ? T[i + P.pitch] - T[i] : 0.0f;
  } else {
    float t0 = time_surface(P.t_last[i], clock, t_init, c);
    a = (x < P.W - 1) ? surface_diff(time_surface(P.t_last[i + 1], clock, t_init, c), t0) : 0.0f;
    b = (y < P.H - 1) ? surface_diff(time_surface(P.t_last[i + P.pitch], clock, t_init, c), t0)
                      : 0.0f;
  }
  float G = metric_G(a, b);
  P.tx[i] = a;
  P.ty[i] = b;
  P.iG[i] = 1.0f / G;
  P.sG[i] = sqrtf(G);
  float base = (c.data_mode == 0) ? P.u[cur][i] : P.f[i];
  P.f[i] = data_image(base, P.npos[i], P.nneg[i], c);
  P.npos[i] = 0;
  P.nneg[i] = 0;
}

// Per pixel: L_x t, L_y t (forward differences, zero on the last column/row), G,
// 1/G, sqrt G (Eq. 2, text after Eq. 3), and the data image
// f = base * exp(Delta+ n+ - Delta- n-) (Eq. intensity_update, one factor per event);
// the counts are then cleared.  One kernel serves a single stream (B.descs null,
// blocks numbered over its image) and a batch (one work item per CTA).
__global__ void __launch_bounds__(256) k_prologue(const __grid_constant__ Planes P, int cur,
                                                  PrologueConsts c, BatchRef B) {
  // Launched as a programmatic dependent of the push (in the fused push-and-solve
  // graph): wait for its completion before reading the pixel state (a no-op when
  // launched without that relation).  The first iteration pass may launch now; it
  // reads nothing of ours before its own griddepcontrol.wait, which returns once this
  // grid has completed.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
  __shared__ Planes sP;  // this CTA's stream, staged once
  int blk = blockIdx.x;
  if (B.descs) {
    const int2 w = B.work[blockIdx.x];
    if (!B.active[w.x]) return;
    cur = B.curs[w.x];
    blk = w.y;
    if (threadIdx.y == 0) stage_planes(&sP, &B.descs[w.x], threadIdx.x);
  } else if (threadIdx.y == 0) {
    stage_planes(&sP, &P, threadIdx.x);
  }
  __syncthreads();
  prologue_px_body(sP, cur, c, blk);
}

// ---------------------------------------------------------------- TV-L1 of the surface
// Anisotropic TV-L1 (Sec. 4: the timestamps are denoised with a few TV-L1 iterations
// before the surface is used): min_s sum |L_x s| + |L_y s| + lam sum |s - t0|,
// Chambolle-Pock with steps 1/sqrt(8), from s = t0, q = 0.
__global__ void k_tvl1_init(Planes P, PrologueConsts c, float* t0, float* s, float* q1,
                            float* q2) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  long long clock = P.sc->clock;
  long long t_init = P.sc->t_init_set ? P.sc->t_init : clock;
  size_t i = (size_t)y * P.pitch + x;
  float v = time_surface(P.t_last[i], clock, t_init, c);
  t0[i] = v;
  s[i] = v;
  q1[i] = 0.0f;
  q2[i] = 0.0f;
}

// s+ = t0 + shrink(s + st div q - t0, st lam), sbar = 2 s+ - s
__global__ void k_tvl1_primal(Planes P, float st, float lam, const float* t0, float* s,
                              const float* q1, const float* q2, float* sbar) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  size_t i = (size_t)y * P.pitch + x;
  float div = 0.0f;
  if (x < P.W - 1) div += q1[i];
  if (x > 0) div -= q1[i - 1];
  if (y < P.H - 1) div += q2[i];
  if (y > 0) div -= q2[i - P.pitch];
  float d = s[i] + st * div - t0[i];
  float a = st * lam;
  float sh = (d > a) ? d - a : ((d < -a) ? d + a : 0.0f);
  float sn = t0[i] + sh;
  sbar[i] = 2.0f * sn - s[i];
  s[i] = sn;
}

// q = clip(q + st grad(sbar), -1, 1) per component
__global__ void k_tvl1_dual(Planes P, float st, const float* sbar, float* q1, float* q2) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  size_t i = (size_t)y * P.pitch + x;
  float gx = (x < P.W - 1) ? sbar[i + 1] - sbar[i] : 0.0f;
  float gy = (y < P.H - 1) ? sbar[i + P.pitch] - sbar[i] : 0.0f;
  q1[i] = fminf(1.0f, fmaxf(-1.0f, q1[i] + st * gx));
  q2[i] = fminf(1.0f, fmaxf(-1.0f, q2[i] + st * gy));
}

int launch_tvl1(const Planes& P, const PrologueConsts& c, int K, float lam, float* t0, float* s,
                float* q1, float* q2, float* sbar, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  dim3 blk(32, 8), grd((P.W + 31) / 32, (P.H + 7) / 8);
  const float step = 1.0f / sqrtf(8.0f);
  k_tvl1_init<<<grd, blk, 0, st>>>(P, c, t0, s, q1, q2);
  for (int k = 0; k < K; ++k) {
    k_tvl1_primal<<<grd, blk, 0, st>>>(P, step, lam, t0, s, q1, q2, sbar);
    k_tvl1_dual<<<grd, blk, 0, st>>>(P, step, sbar, q1, q2);
  }
  return (int)cudaGetLastError();
}

int launch_prologue(const Planes& P, int cur, const PrologueConsts& c, void* stream) {
  const int nb = ((P.W + 31) / 32) * ((P.H + 7) / 8);
  // programmatic stream serialisation: the prologue may start while its predecessor
  // (the push) drains; it waits for it before reading (griddepcontrol.wait)
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(nb);
  lc.blockDim = dim3(32, 8);
  lc.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&lc, k_prologue, P, cur, c,
                                 BatchRef{nullptr, nullptr, nullptr, nullptr});
}

int launch_prologue_batch(const BatchRef& B, int n_work, const PrologueConsts& c, void* stream) {
  if (n_work <= 0) return 0;
  Planes dummy{};
  k_prologue<<<n_work, dim3(32, 8), 0, (cudaStream_t)stream>>>(dummy, 0, c, B);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- unfused iteration
// Primal step at every pixel: v = u + tau div_g p, u+ = prox(v), ubar = 2u+ - u.
__global__ void k_primal(Planes P, int cur, SolveConsts c) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  size_t i = (size_t)y * P.pitch + x;
  const float *p1 = P.p1[cur], *p2 = P.p2[cur], *p3 = P.p3[cur];
  float q1, q2, q1m = 0.0f, q2m = 0.0f, d1, d2;
  apply_MT(P.tx[i], P.ty[i], P.iG[i], p1[i], p2[i], p3[i], q1, q2);
  if (x > 0) apply_MT(P.tx[i - 1], P.ty[i - 1], P.iG[i - 1], p1[i - 1], p2[i - 1], p3[i - 1], q1m, d2);
  if (y > 0) {
    size_t j = i - P.pitch;
    apply_MT(P.tx[j], P.ty[j], P.iG[j], p1[j], p2[j], p3[j], d1, q2m);
  }
  float div = ((x < P.W - 1) ? q1 : 0.0f) - q1m + ((y < P.H - 1) ? q2 : 0.0f) - q2m;
  float u = P.u[cur][i];
  float v = u + c.tau * div;
  float beta = c.tau * c.lambda * P.sG[i];
  float un = c.data_term ? (v + beta * P.f[i]) / (1.0f + beta)  // Eq. 7, no box
                         : prox_kl(v, beta, P.f[i], c.u_min, c.u_max);
  P.u[cur][i] = un;
  P.ubar[i] = 2.0f * un - u;
}

// Dual step at every pixel: p = proj(p + sigma L_g ubar).
__global__ void k_dual(Planes P, int cur, SolveConsts c) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  size_t i = (size_t)y * P.pitch + x;
  float ub = P.ubar[i];
  float ux = (x < P.W - 1) ? P.ubar[i + 1] - ub : 0.0f;
  float uy = (y < P.H - 1) ? P.ubar[i + P.pitch] - ub : 0.0f;
  float g1, g2, g3;
  apply_M(P.tx[i], P.ty[i], P.iG[i], ux, uy, g1, g2, g3);
  float p1 = P.p1[cur][i] + c.sigma * g1;
  float p2 = P.p2[cur][i] + c.sigma * g2;
  float p3 = P.p3[cur][i] + c.sigma * g3;
  project(p1, p2, p3, P.sG[i]);
  P.p1[cur][i] = p1;
  P.p2[cur][i] = p2;
  P.p3[cur][i] = p3;
}

int launch_unfused_iteration(const Planes& P, int cur, const SolveConsts& c, void* stream) {
  dim3 blk(32, 8), grd((P.W + 31) / 32, (P.H + 7) / 8);
  k_primal<<<grd, blk, 0, (cudaStream_t)stream>>>(P, cur, c);
  k_dual<<<grd, blk, 0, (cudaStream_t)stream>>>(P, cur, c);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 gap
// Per pixel, in FP64 from the FP32 state: the g-tensor norm term sqrt(G) |L_g u|,
// the data term sqrt(G)(u - f log u) (Eq. 5), and the dual term
// min_{u in box} a (u - f log u) + w u with a = lambda sqrt(G), w = -div_g p, whose
// minimiser is clamp(a f / (a + w)) for a + w > 0 and u_max otherwise.
// p component at pixel i in the stream's storage format, widened
__device__ __forceinline__ float ld_p(const Planes& P, const float* plane, size_t i) {
  if (P.storage == 1) return __half2float(((const __half*)plane)[i]);
  if (P.storage == 2) return __bfloat162float(((const __nv_bfloat16*)plane)[i]);
  return plane[i];
}

__device__ __forceinline__ void mt64(const Planes& P, size_t i, int cur, double& q1, double& q2) {
  double a = P.tx[i], b = P.ty[i];
  double G = 1.0 + a * a + b * b;
  double p1 = ld_p(P, P.p1[cur], i), p2 = ld_p(P, P.p2[cur], i), p3 = ld_p(P, P.p3[cur], i);
  q1 = ((1.0 + b * b) * p1 - a * b * p2 + a * p3) / G;
  q2 = (-a * b * p1 + (1.0 + a * a) * p2 + b * p3) / G;
}

__global__ void __launch_bounds__(kGapThreads) k_gap_partial(Planes P, int cur, SolveConsts c) {
  __shared__ double s[3][kGapThreads];
  double reg = 0.0, dat = 0.0, dua = 0.0;
  const int n = P.W * P.H;
  const double lam = c.lambda, umin = c.u_min, umax = c.u_max;
  for (int k = blockIdx.x * kGapThreads + threadIdx.x; k < n; k += kGapBlocks * kGapThreads) {
    int x = k % P.W, y = k / P.W;
    size_t i = (size_t)y * P.pitch + x;
    const float* U = P.u[cur];
    double a = P.tx[i], b = P.ty[i];
    double G = 1.0 + a * a + b * b, sG = sqrt(G);
    double u = U[i], f = P.f[i];
    double ux = (x < P.W - 1) ? (double)U[i + 1] - u : 0.0;
    double uy = (y < P.H - 1) ? (double)U[i + P.pitch] - u : 0.0;
    double g1 = ((1.0 + b * b) * ux - a * b * uy) / G;
    double g2 = ((1.0 + a * a) * uy - a * b * ux) / G;
    double g3 = (a * ux + b * uy) / G;
    reg += sqrt(G * (g1 * g1 + g2 * g2 + g3 * g3));
    if (c.data_term)
      dat += 0.5 * (u - f) * (u - f) * sG;  // Eq. 7
    else
      dat += (u - (f == 0.0 ? 0.0 : f * log(u))) * sG;
    double q1, q2, q1m = 0.0, q2m = 0.0, d;
    mt64(P, i, cur, q1, q2);
    if (x > 0) mt64(P, i - 1, cur, q1m, d);
    if (y > 0) mt64(P, i - P.pitch, cur, d, q2m);
    double div = ((x < P.W - 1) ? q1 : 0.0) - q1m + ((y < P.H - 1) ? q2 : 0.0) - q2m;
    double aa = lam * sG, w = -div;
    if (c.data_term) {  // min_u (aa/2)(u - f)^2 + w u = w f - w^2 / (2 aa)
      dua += w * f - w * w / (2.0 * aa);
    } else {
      double us = (aa + w > 0.0) ? aa * f / (aa + w) : umax;
      us = fmin(fmax(us, umin), umax);
      dua += aa * (us - (f == 0.0 ? 0.0 : f * log(us))) + w * us;
    }
  }
  s[0][threadIdx.x] = reg;
  s[1][threadIdx.x] = dat;
  s[2][threadIdx.x] = dua;
  __syncthreads();
  for (int h = kGapThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 3; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) P.partials[3 * blockIdx.x + j] = s[j][0];
}

__global__ void __launch_bounds__(512) k_gap_final(Planes P, SolveConsts c, double* out2) {
  __shared__ double s[3][512];
  for (int j = 0; j < 3; ++j)
    s[j][threadIdx.x] = (threadIdx.x < kGapBlocks) ? P.partials[3 * threadIdx.x + j] : 0.0;
  __syncthreads();
  for (int h = 256; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 3; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = s[0][0] + (double)c.lambda * s[1][0];
    out2[1] = s[2][0];
  }
}

__global__ void k_p_convert(Planes P, void* pp, float* fp, int to_f32) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  size_t i = (size_t)y * P.pitch + x;
  if (to_f32) {
    fp[i] = ld_p(P, (const float*)pp, i);
  } else if (P.storage == 1) {
    ((__half*)pp)[i] = __float2half_rn(fp[i]);
  } else if (P.storage == 2) {
    ((__nv_bfloat16*)pp)[i] = __float2bfloat16_rn(fp[i]);
  } else {
    ((float*)pp)[i] = fp[i];
  }
}

int launch_p_convert(const Planes& P, void* p_plane, float* f_plane, int to_f32, void* stream) {
  dim3 blk(32, 8), grd((P.W + 31) / 32, (P.H + 7) / 8);
  k_p_convert<<<grd, blk, 0, (cudaStream_t)stream>>>(P, p_plane, f_plane, to_f32);
  return (int)cudaGetLastError();
}

int launch_gap(const Planes& P, int cur, const SolveConsts& c, double* out2, void* stream) {
  static_assert(kGapBlocks <= 512, "final reduction covers all partials");
  cudaStream_t st = (cudaStream_t)stream;
  k_gap_partial<<<kGapBlocks, kGapThreads, 0, st>>>(P, cur, c);
  k_gap_final<<<1, 512, 0, st>>>(P, c, out2);
  return (int)cudaGetLastError();
}

}  // namespace evr
