// evr_grad.cu -- differentiation of one packet's solve (K unrolled iterations of
// Eq. cont_iterates with Eq. update_rules) by a hand-written adjoint, with (u, p)
// checkpoints every `every` iterations.  The iterations themselves (forward, and the
// recomputation of each checkpoint segment) are the solver's tiled FP32 passes, and so
// is the reverse pass (k_rev_tiled); the lambda gradient is summed in FP32 per warp and
// iteration and in FP64 from there, the contrast-threshold sums in FP64.
//
// All memory (inputs, outputs and the workspace) belongs to the caller; nothing here
// allocates.  Planes are H rows of `pitch` floats; a dual variable is 3 such planes
// back to back (plane stride pitch * H).
#include <cuda_runtime.h>

#include <new>

#include "../../include/evr.h"
#include "evr_internal.cuh"
#include "evr_tma.cuh"

namespace {

namespace tma = evr::tma;

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 1024;

// Launch accounting of the calls below for benchmarks (process-wide, not thread-safe):
// while on, every kernel launch is counted and the first kMaxTimed reverse-pass launches
// are bracketed by CUDA events on their stream.
constexpr int kMaxTimed = 16384;
struct LaunchTiming {
  bool on = false;
  long long launches = 0;
  int n = 0;                     // recorded reverse-pass launches
  long long px_iters = 0;        // their reversed pixel-iterations
  long long px_launches = 0;     // their pixels x launches
  cudaEvent_t* ev = nullptr;     // 2 kMaxTimed events, created on the first start
};
LaunchTiming g_timing;

inline void counted(int k = 1) {
  if (g_timing.on) g_timing.launches += k;
}

// n images of W x Hm stacked vertically into one W x (n Hm) image (H = n Hm): the
// forward differences and divergences use the row within the member, so the members
// stay independent (zero y-difference on each member's last row).
struct Geo {
  int W, H, pitch;
  size_t plane;  // pitch * H
  int Hm;        // rows per member
};

struct Coef {
  float tau, sigma, lambda, u_min, u_max;
};

// Per-pixel metric of the packet (Eq. 3): L_x t, L_y t and, computed once per call by
// k_metric with IEEE division and square root, 1/G and sqrt(G), G = 1 + a^2 + b^2.
struct Met {
  const float* tx;
  const float* ty;
  const float* iG;
  const float* sG;
};

__device__ __forceinline__ void metric(const Met& m, size_t i, float& a, float& b, float& iG) {
  a = m.tx[i];
  b = m.ty[i];
  iG = m.iG[i];
}

// M (ux, uy) with M = (1/G)[[1+b^2,-ab],[-ab,1+a^2],[a,b]] (Eq. 3)
__device__ __forceinline__ void Mg(float a, float b, float iG, float ux, float uy, float& g1,
                                   float& g2, float& g3) {
  float w = b * ux - a * uy;
  g1 = iG * (ux + b * w);
  g2 = iG * (uy - a * w);
  g3 = iG * (a * ux + b * uy);
}

// L_g w at (x, y) for a scalar plane w
__device__ __forceinline__ void Lg(const Geo& g, const Met& m, const float* w, int x, int yl,
                                   size_t i, float& g1, float& g2, float& g3) {
  float a, b, iG;
  metric(m, i, a, b, iG);
  float wx = (x < g.W - 1) ? w[i + 1] - w[i] : 0.0f;
  float wy = (yl < g.Hm - 1) ? w[i + g.pitch] - w[i] : 0.0f;
  Mg(a, b, iG, wx, wy, g1, g2, g3);
}

#define PIXEL                                             \
  const int x = blockIdx.x * blockDim.x + threadIdx.x;     \
  const int y = blockIdx.y * blockDim.y + threadIdx.y;     \
  if (x >= g.W || y >= g.H) return;                        \
  const size_t i = (size_t)y * g.pitch + x;                \
  const int yl = y % g.Hm;

__global__ void k_metric(Geo g, const float* tx, const float* ty, float* iG, float* sG) {
  PIXEL
  (void)yl;
  const float a = tx[i], b = ty[i];
  const float G = 1.0f + a * a + b * b;
  iG[i] = 1.0f / G;
  sG[i] = sqrtf(G);
}

// ---- the reverse pass, tiled ----
// One launch reverses up to kRevR consecutive iterations k_hi, k_hi - 1, ... of one
// checkpoint segment on overlapped tiles: a 32 x 2 kRevNTY tile (one lane per column,
// a vertical pair of pixels per thread) owns its interior and carries a kRevR-pixel
// halo.  Reversing an iteration reads tau a_v of the later iteration at x+1 and y+1 (in
// L_g) and the new a_pt at x-1 and y-1 (in div_g), so, as in the forward, the values
// stay exact on the tile shrunk by one pixel per side and iteration.  The adjoint state
// (a_u, a_pt, tau a_v and the accumulated dL/df) stays in registers across the launch's
// iterations; per iteration only the tape's p, v and ubar are read, from a shared-memory
// copy of the slot staged one iteration ahead where the tape's rows are a multiple of 16
// bytes (the pitch a multiple of 4), else directly.
//
// Reversing iteration k (state k = tape slot, adjoints of u_{k+1}, p_{k+1} given):
//   a_p(k+1) = a_pt(k+1) - L_g(tau a_v(k+1))   (the given one if k = K-1)
//   projection adjoint: pt = p_k + sigma L_g ubar_k; outside the ball
//     a_pt = (sqrt(G)/|pt|) (a_p - pt (pt . a_p) / |pt|^2), else a_pt = a_p
//   a_ubar = -div_g(sigma a_pt)
//   KL root r(v, beta, f) with d = v - beta, s = sqrt(d^2 + 4 beta f):
//     a_r = (a_u + 2 a_ubar) where r lies inside [u_min, u_max], else 0
//     a_v = a_r (1 + d / s) / 2;  dL/df += a_r beta / s;
//     dL/dlambda += a_r (-1 + (2 f - v + beta) / s) / 2 * tau sqrt(G)
//   a_u(k) = -a_ubar + a_v
// 1/|pt| and 1/s are MUFU reciprocal square roots (no divisions).  The lambda terms are
// summed in FP32 over each tile's owned pixels in a fixed order and in FP64 from there on
// (GB300 issues FP64 arithmetic at a small fraction of the FP32 rate).
constexpr int kRevR = 4;
constexpr int kRevNTY = 16;
// Where the tape's rows are a multiple of 16 bytes, the tape slot of each reversed
// iteration is staged in shared memory by one tensor copy
// (x, row, plane) issued one iteration ahead into the second of two stages: a box of
// 5 planes x (2 kRevNTY + 1) rows x (32 + 8) columns, starting at the tile's x rounded
// down to 8 elements (the 16-byte rule of tensor copies) and one row longer than the tile
// for the y + 1 neighbour of its last row.
constexpr int kRevBW = 40, kRevBH = 2 * kRevNTY + 1;
constexpr int kRevPlaneF = kRevBW * kRevBH;                  // floats per staged plane
constexpr int kRevStageF = (5 * kRevPlaneF + 31) / 32 * 32;  // 128-byte aligned stages
constexpr size_t kRevSmem = 2 * sizeof(float) * kRevStageF;
constexpr unsigned kRevSpin = 1u << 22;  // polls of a stage's mbarrier before giving up

struct RevArgs {
  Geo g;
  Coef c;
  Met m;
  const float* f;
  const float* tape;  // slots of 5 planes (p1 p2 p3 v ubar), plane stride g.plane
  int slot_hi;        // tape slot of iteration k_hi
  int k_hi, iters;
  int first;          // iteration k_hi is the last one: its a_p(k+1) is given in a_in[1..3]
  // a_u, a_pt (3 planes), tau a_v at the start (a null plane reads as 0) and at the end
  const float* a_in[5];
  float* a_out[5];
  float* gf;
  double* glam;       // per (iteration, tile) lambda sums
  int tiles_x, tiles_total;
  int staged;  // 1: the tape slots come through tape_map (rows of a multiple of 16 bytes)
};

__global__ void __launch_bounds__(32 * kRevNTY, 2)
    k_rev_tiled(RevArgs A, const __grid_constant__ CUtensorMap tape_map) {
  constexpr int NT = kRevNTY, EW = 32, EH = 2 * NT, R = kRevR;
  constexpr int OW = EW - 2 * R, OH = EH - 2 * R;
  extern __shared__ __align__(128) float rstage[];  // [2][kRevStageF]: tape slots
  // neighbours in x are adjacent lanes (warp shuffles); in y the next thread row's
  // first pixel (tau a_v) and the previous row's last (q2) go through shared memory
  __shared__ float tv[EH + 1][EW];   // tau a_v of the even rows; row EH: zero pad
  __shared__ float q2s[EH + 1][EW];  // (M^T sigma a_pt)_2 masked; row 0: zero pad
  __shared__ float lsum[NT];            // the warps' lambda sums of an iteration
  __shared__ __align__(8) unsigned long long s_mb[2];
  __shared__ int s_bail;
  const Geo& g = A.g;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tile = blockIdx.x;
  const int gx0 = (tile % A.tiles_x) * OW - R, gy0 = (tile / A.tiles_x) * OH - R;
  const int x = gx0 + lane;
  const float tau = A.c.tau, sigma = A.c.sigma;
  float E1[2], E2[2], E3[2], E4[2], E5[2], E6[2], sg[2], fi[2];
  float au[2], a1[2], a2[2], a3[2], tav[2], gfa[2];
  bool in[2], own[2];
  unsigned idx[2];     // pixel index (planes hold fewer than 2^31 floats)
  unsigned ydiff = 0;  // bit h: pixel h has a y + 1 neighbour in its member
  for (int h = 0; h < 2; ++h) {
    const int ly = 2 * ty + h, y = gy0 + ly;
    in[h] = x >= 0 && x < g.W && y >= 0 && y < g.H;
    own[h] = in[h] && lane >= R && lane < R + OW && ly >= R && ly < R + OH;
    E1[h] = E2[h] = E3[h] = E4[h] = E5[h] = E6[h] = sg[h] = fi[h] = 0.0f;
    au[h] = a1[h] = a2[h] = a3[h] = tav[h] = gfa[h] = 0.0f;
    idx[h] = 0;
    if (in[h]) {
      const unsigned i = (unsigned)y * (unsigned)g.pitch + (unsigned)x;
      const int yl = y % g.Hm;
      const float mx = x < g.W - 1 ? 1.0f : 0.0f, my = yl < g.Hm - 1 ? 1.0f : 0.0f;
      idx[h] = i;
      if (yl < g.Hm - 1) ydiff |= 1u << h;
      const float a = A.m.tx[i], b = A.m.ty[i], ig = A.m.iG[i];
      const float m12 = -(ig * (a * b));
      E1[h] = mx * (ig * fmaf(b, b, 1.0f));
      E2[h] = mx * m12;
      E3[h] = mx * (ig * a);
      E4[h] = my * m12;
      E5[h] = my * (ig * fmaf(a, a, 1.0f));
      E6[h] = my * (ig * b);
      sg[h] = A.m.sG[i];
      fi[h] = A.f[i];
      au[h] = A.a_in[0] ? A.a_in[0][i] : 0.0f;
      a1[h] = A.a_in[1] ? A.a_in[1][i] : 0.0f;
      a2[h] = A.a_in[2] ? A.a_in[2][i] : 0.0f;
      a3[h] = A.a_in[3] ? A.a_in[3][i] : 0.0f;
      tav[h] = A.a_in[4] ? A.a_in[4][i] : 0.0f;
      if (own[h]) gfa[h] = A.gf[i];
    }
    tv[ly][lane] = tav[h];
  }
  const int tid = ty * 32 + lane;
  for (int i = tid; i < EW; i += 32 * NT) {
    tv[EH][i] = 0.0f;
    q2s[0][i] = 0.0f;
  }
  const int sx0 = gx0 & ~7;  // the staged box's first column
  auto issue = [&](int it, int b) {  // thread 0: the tape slot of reversed iteration it
    const uint32_t mb = tma::smem_u32(&s_mb[b]);
    tma::mbar_arm(mb, 5u * kRevPlaneF * 4u);
    tma::load_3d(tma::smem_u32(rstage + b * kRevStageF), &tape_map, sx0, gy0,
                 5 * (A.slot_hi - it), mb);
  };
  if (tid == 0) {
    s_bail = 0;
    if (A.staged) {
      tma::mbar_init1(tma::smem_u32(&s_mb[0]));
      tma::mbar_init1(tma::smem_u32(&s_mb[1]));
      tma::mbar_init_fence();
      issue(0, 0);
    }
  }
  __syncthreads();
  const float tl = tau * A.c.lambda;
  const unsigned PL = (unsigned)g.plane;  // plane stride (< 2^31 floats, checked)
  // x + 1 neighbour where the x-difference exists (else the pixel itself: that difference
  // is masked out); y + 1: pixel 1 of the pair for pixel 0, the next row for pixel 1,
  // where the y-difference exists
  const unsigned ox = x < g.W - 1 ? 1u : 0u;
  const unsigned oy1 = (ydiff & 2u) ? (unsigned)g.pitch : 0u;
  for (int it = 0; it < A.iters; ++it) {
    float p1[2], p2[2], p3[2], ub[2], ubx[2], vk[2];
    float uby1 = 0.0f;
    if (A.staged) {
      // the next iteration's slot into the other stage (read one iteration ago, by every
      // thread before that iteration's barriers), then wait for this one's (bounded)
      if (tid == 0 && it + 1 < A.iters) {
        tma::fence_proxy_async();
        issue(it + 1, (it + 1) & 1);
      }
      const uint32_t mb = tma::smem_u32(&s_mb[it & 1]);
      for (unsigned n = 0; !tma::mbar_done(mb, (uint32_t)(it >> 1) & 1u);)
        if (++n > kRevSpin) {
          s_bail = 1;
          break;
        }
      const float* slot = rstage + (it & 1) * kRevStageF;
      // the iteration's tape values of both pixels from the staged slot
      for (int h = 0; h < 2; ++h) {
        p1[h] = p2[h] = p3[h] = ub[h] = ubx[h] = vk[h] = 0.0f;
        if (in[h]) {
          const int o = (2 * ty + h) * kRevBW + lane + (gx0 - sx0);
          p1[h] = slot[o];
          p2[h] = slot[kRevPlaneF + o];
          p3[h] = slot[2 * kRevPlaneF + o];
          vk[h] = slot[3 * kRevPlaneF + o];
          ub[h] = slot[4 * kRevPlaneF + o];
          ubx[h] = slot[4 * kRevPlaneF + o + (int)ox];
          if (h == 1) uby1 = slot[4 * kRevPlaneF + o + ((ydiff & 2u) ? kRevBW : 0)];
        }
      }
    } else {
      const float* slot = A.tape + (size_t)(A.slot_hi - it) * 5 * g.plane;  // uniform
      // the iteration's tape values of both pixels, all loads issued together
      for (int h = 0; h < 2; ++h) {
        p1[h] = p2[h] = p3[h] = ub[h] = ubx[h] = vk[h] = 0.0f;
        if (in[h]) {
          const unsigned i = idx[h];
          p1[h] = slot[i];
          p2[h] = slot[PL + i];
          p3[h] = slot[2 * PL + i];
          vk[h] = slot[3 * PL + i];
          ub[h] = slot[4 * PL + i];
          ubx[h] = slot[4 * PL + i + ox];
          if (h == 1) uby1 = slot[4 * PL + i + oy1];
        }
      }
    }
    float q1o[2], q2o[2];  // this thread's own (M^T sigma a_pt) entries
    // projection adjoint
    for (int h = 0; h < 2; ++h) {
      const int ly = 2 * ty + h;
      float b1 = a1[h], b2 = a2[h], b3 = a3[h];
      // tau a_v of the x + 1 neighbour: the lane to the right (lane 31, a halo column
      // whose value is inexact after the first reversed iteration whatever it reads,
      // takes its own)
      const float tvx = __shfl_down_sync(0xffffffffu, tav[h], 1);
      if (!(A.first && it == 0)) {
        const float tyn = h == 0 ? tav[1] : tv[ly + 1][lane];
        const float dx = tvx - tav[h], dy = tyn - tav[h];
        b1 -= fmaf(E4[h], dy, E1[h] * dx);
        b2 -= fmaf(E5[h], dy, E2[h] * dx);
        b3 -= fmaf(E6[h], dy, E3[h] * dx);
      }
      const float uyn = h == 0 ? ((ydiff & 1u) ? ub[1] : ub[0]) : uby1;
      const float ux = ubx[h] - ub[h], uy = in[h] ? uyn - ub[h] : 0.0f;
      const float t1 = fmaf(sigma, fmaf(E4[h], uy, E1[h] * ux), p1[h]);
      const float t2 = fmaf(sigma, fmaf(E5[h], uy, E2[h] * ux), p2[h]);
      const float t3 = fmaf(sigma, fmaf(E6[h], uy, E3[h] * ux), p3[h]);
      const float n2 = fmaf(t1, t1, fmaf(t2, t2, t3 * t3));
      const float inv = rsqrtf(n2);  // n2 = 0: inf, and n2 * inv is NaN: inside the ball
      if (n2 * inv > sg[h]) {
        const float dot = fmaf(t1, b1, fmaf(t2, b2, t3 * b3)) * (inv * inv);
        const float sc = sg[h] * inv;
        b1 = sc * fmaf(-t1, dot, b1);
        b2 = sc * fmaf(-t2, dot, b2);
        b3 = sc * fmaf(-t3, dot, b3);
      }
      a1[h] = b1;
      a2[h] = b2;
      a3[h] = b3;
      // rounded products (no contraction into the later differences): a neighbour's
      // value read from shared memory and the thread's own from a register are the same
      // number, so a pixel's result does not depend on its place in the tile
      q1o[h] = __fmul_rn(sigma, fmaf(E3[h], b3, fmaf(E2[h], b2, E1[h] * b1)));
      q2o[h] = __fmul_rn(sigma, fmaf(E6[h], b3, fmaf(E5[h], b2, E4[h] * b1)));
      if (h == 1) q2s[ly + 1][lane] = q2o[h];  // read by the thread row below
    }
    __syncthreads();
    // primal adjoint
    float lam = 0.0f;
    for (int h = 0; h < 2; ++h) {
      const int ly = 2 * ty + h;
      const float q2m = h == 0 ? q2s[ly][lane] : q2o[0];
      // x - 1 neighbour: the lane to the left (lane 0, a halo column, takes its own)
      const float q1m = __shfl_up_sync(0xffffffffu, q1o[h], 1);
      const float div = (q1o[h] - q1m) + (q2o[h] - q2m);
      const float aub = -div;
      float av = 0.0f;  // outside the image: no data term (and no 0/0)
      if (in[h]) {
        const float v = vk[h];
        const float beta = tl * sg[h];
        const float d = v - beta;
        const float disc = fmaf(d, d, 4.0f * beta * fi[h]);
        const float rs = rsqrtf(disc);  // 1 / s
        const float r = 0.5f * fmaf(disc, rs, d);
        const float aun = fmaf(2.0f, aub, au[h]);
        const float ar = (r < A.c.u_min || r > A.c.u_max) ? 0.0f : aun;
        av = ar * 0.5f * fmaf(d, rs, 1.0f);
        if (own[h]) {
          gfa[h] = fmaf(ar, beta * rs, gfa[h]);
          lam = fmaf(ar * 0.5f * fmaf(2.0f * fi[h] - v + beta, rs, -1.0f), tau * sg[h], lam);
        }
      }
      au[h] = av - aub;
      tav[h] = __fmul_rn(tau, av);
      if (h == 0) tv[ly][lane] = tav[h];  // the y + 1 neighbour of the thread row above
    }
    // the tile's lambda sum of the iteration, in FP32 in a fixed order (within each warp,
    // then over the warps by warp 0)
    for (int o = 16; o > 0; o >>= 1) lam += __shfl_down_sync(0xffffffffu, lam, o);
    if (lane == 0) lsum[ty] = lam;
    __syncthreads();
    if (ty == 0) {
      float t = lane < NT ? lsum[lane] : 0.0f;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) A.glam[(size_t)(A.k_hi - it) * A.tiles_total + tile] = (double)t;
    }
  }
  // a stage wait that ran out poisons this tile's outputs (NaN), so that a failed copy
  // cannot pass for a gradient
  __syncthreads();
  const bool bail = s_bail != 0;
  for (int h = 0; h < 2; ++h) {
    if (!own[h]) continue;
    const unsigned i = idx[h];
    const float nan = __int_as_float(0x7fc00000);
    A.a_out[0][i] = bail ? nan : au[h];
    A.a_out[1][i] = bail ? nan : a1[h];
    A.a_out[2][i] = bail ? nan : a2[h];
    A.a_out[3][i] = bail ? nan : a3[h];
    A.a_out[4][i] = bail ? nan : tav[h];
    A.gf[i] = bail ? nan : gfa[h];
  }
}

// The adjoint of p_0: a_p = a_pt - L_g(tau a_v) of the reversed iteration 0 (a_pt with
// plane stride g.plane, the output with plane stride out_plane).
__global__ void k_b_pupdate(Geo g, Met m, const float* apt, const float* tav, float* ap,
                            size_t out_plane) {
  PIXEL
  float g1, g2, g3;
  Lg(g, m, tav, x, yl, i, g1, g2, g3);
  ap[i] = apt[i] - g1;
  ap[out_plane + i] = apt[g.plane + i] - g2;
  ap[2 * out_plane + i] = apt[2 * g.plane + i] - g3;
}

__global__ void k_zero(Geo g, float* a, int planes) {
  PIXEL
  (void)yl;
  for (int k = 0; k < planes; ++k) a[k * g.plane + i] = 0.0f;
}

__global__ void k_copy(Geo g, const float* src, float* dst, int planes) {
  PIXEL
  (void)yl;
  for (int k = 0; k < planes; ++k) dst[k * g.plane + i] = src[k * g.plane + i];
}

// Fixed-order FP64 reduction of up to 4 per-pixel double planes into out[0..n-1].
__global__ void __launch_bounds__(kRedThreads) k_red_partial(Geo g, const double* a, int n,
                                                            double* partials) {
  __shared__ double s[4][kRedThreads];
  double acc[4] = {0, 0, 0, 0};
  const int N = g.W * g.H;
  for (int k = blockIdx.x * kRedThreads + threadIdx.x; k < N; k += kRedBlocks * kRedThreads) {
    const size_t i = (size_t)(k / g.W) * g.pitch + (k % g.W);
    for (int j = 0; j < n; ++j) acc[j] += a[j * g.plane + i];
  }
  for (int j = 0; j < 4; ++j) s[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 4; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) partials[4 * blockIdx.x + j] = s[j][0];
}

__global__ void __launch_bounds__(kRedBlocks) k_red_final(const double* partials, int n,
                                                         double* out) {
  __shared__ double s[4][kRedBlocks];
  for (int j = 0; j < 4; ++j) s[j][threadIdx.x] = partials[4 * threadIdx.x + j];
  __syncthreads();
  for (int h = kRedBlocks / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 4; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < n; ++j) out[j] = s[j][0];
}

// Data image f = u_prev exp(Delta+ n+ - Delta- n-) (Eq. intensity_update, compounded).
__global__ void k_data_image(Geo g, const float* u_prev, const int* npos, const int* nneg,
                             float dpos, float dneg, float* f) {
  PIXEL
  (void)yl;
  f[i] = u_prev[i] * expf(dpos * (float)npos[i] - dneg * (float)nneg[i]);
}

// Its backward: g_uprev = gf exp(...), per-pixel terms of dL/dDelta+ = sum gf f n+ and
// dL/dDelta- = -sum gf f n-.
__global__ void k_data_image_bwd(Geo g, const float* f, const float* u_prev, const int* npos,
                                 const int* nneg, float dpos, float dneg, const float* gf,
                                 float* g_uprev, double* terms) {
  PIXEL
  (void)yl;
  float e = expf(dpos * (float)npos[i] - dneg * (float)nneg[i]);
  if (g_uprev) g_uprev[i] = gf[i] * e;
  const float gff = gf[i] * f[i];  // FP32 products (GB300's FP64 rate is low), FP64 sums
  terms[i] = (double)(gff * (float)npos[i]);
  terms[g.plane + i] = -(double)(gff * (float)nneg[i]);
}

struct Workspace {
  float* ck;       // n_ck checkpoints x 4 planes
  float* tape_last;  // the last checkpoint segment's tape, written by the forward: one
                     // slot of 5 planes per iteration (p1 p2 p3 of the state it starts
                     // from, then its v and ubar)
  float* tape;       // the backward's replay of one earlier segment (every slots), or
                     // NULL with a single segment
  float* adj;      // 2 x 5 planes: ping-pong adjoint states (a_u, a_pt, tau a_v)
  float* xs;       // 2 states x 4 planes: ping-pong buffers of the passes
  float* iG;       // 1 plane: 1/G
  float* sG;       // 1 plane: sqrt(G)
  double* glam;    // K x (reverse tiles): per-tile lambda-gradient sums
  double* partials;  // 4 * kRedBlocks doubles
};

constexpr int kBlkX = 32, kBlkY = 8;  // pixel-kernel block

// Tiles of the reverse pass over a W x H image (kRevR-pixel halos).
void rev_tiles(int W, int H, int* tx, int* total) {
  const int OW = 32 - 2 * kRevR, OH = 2 * kRevNTY - 2 * kRevR;
  *tx = (W + OW - 1) / OW;
  *total = *tx * ((H + OH - 1) / OH);
}

size_t lam_slots(int W, int H) {
  int tx, total;
  rev_tiles(W, H, &tx, &total);
  return (size_t)total;
}

size_t ws_layout(int W, int H, int pitch, int K, int every, char* base, Workspace* w) {
  const size_t plane = (size_t)pitch * H;
  const size_t bpl = (plane * 4 + 255) / 256 * 256;  // bytes per plane slot
  const int n_ck = (K + every - 1) / every;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) / 256 * 256;
    return base ? base + o : nullptr;
  };
  Workspace t;
  t.ck = (float*)take(bpl * 4 * (size_t)(n_ck > 0 ? n_ck : 1));
  const int len_last = K - (n_ck - 1) * every;
  t.tape_last = (float*)take(bpl * 5 * (size_t)len_last);
  t.tape = n_ck > 1 ? (float*)take(bpl * 5 * (size_t)every) : nullptr;
  t.adj = (float*)take(bpl * 10);
  t.xs = (float*)take(bpl * 8);
  t.iG = (float*)take(bpl);
  t.sG = (float*)take(bpl);
  t.glam = (double*)take(sizeof(double) * (size_t)K * lam_slots(W, H));
  t.partials = (double*)take(sizeof(double) * 4 * kRedBlocks);
  if (w) *w = t;
  return off;
}

// The iterations of the forward pass and of the reverse pass's recomputation run as the
// solver's tiled passes (FP32, a kUnrolledR-pixel halo) over the stacked images; their
// per-pixel arithmetic does not depend on how the iterations are split into launches,
// so the recomputed states equal the forward's bit for bit.
constexpr int kUnrolledR = 5;

// The packet's planes as the tiled passes' descriptor (the state buffers are set per pass).
evr::Planes unrolled_planes(int W, int H, int Hm, int pitch, const float* tx, const float* ty,
                            const float* f, float* iG, float* sG) {
  evr::Planes P{};
  P.W = W;
  P.H = H;
  P.Hm = Hm;
  P.pitch = pitch;
  P.tx = const_cast<float*>(tx);
  P.ty = const_cast<float*>(ty);
  P.f = const_cast<float*>(f);
  P.iG = iG;
  P.sG = sG;
  P.storage = 0;
  return P;
}

// A state (u, p1, p2, p3): four planes anywhere (the workspace's, or the caller's).
struct State {
  float* u;
  float* p[3];
};

State ws_state(float* base, size_t fpl) {
  return State{base, {base + fpl, base + 2 * fpl, base + 3 * fpl}};
}

// The forward's passes (no tape) run on the solver's 32 x 48 tile with two pixel pairs
// per thread (384 threads, two CTAs per SM); the tape passes on the 32 x 32 one-pair tile.
// Both compute each pixel with the same explicitly rounded operations, so the replayed
// states equal the forward's bit for bit.
constexpr evr::SolverCfg kForwardCfg{1, 6, kUnrolledR};

// One tiled pass of `iters` iterations from state a into state b (a is only read).
int tiled_pass(evr::Planes P, const State& a, const State& b, int iters, int pass,
               const evr::SolveConsts& sc, float* tape, size_t fpl, int tape_first,
               cudaStream_t st) {
  P.u[0] = a.u;
  P.p1[0] = a.p[0];
  P.p2[0] = a.p[1];
  P.p3[0] = a.p[2];
  P.u[1] = b.u;
  P.p1[1] = b.p[0];
  P.p2[1] = b.p[1];
  P.p3[1] = b.p[2];
  counted();
  if (!tape) return evr::launch_tiled_pass(P, kForwardCfg, 0, iters, pass, sc, st);
  return evr::launch_tiled_tape(P, kUnrolledR, 0, iters, pass, sc, tape, (long long)fpl,
                                tape_first, st);
}

// The passes of one checkpoint segment of len iterations from state `from`: through the
// two ping-pong states xs, the last pass writing into `to` (not one of xs), or, with
// to = NULL, into whichever of xs is free (with a tape, every iteration's p, v and ubar
// go to tape slots 0 .. len-1).
int segment_passes(const evr::Planes& P, const State& from, const State* to, int len,
                   const evr::SolveConsts& sc, float* xs, float* tape, size_t fpl,
                   cudaStream_t st) {
  const State x[2] = {ws_state(xs, fpl), ws_state(xs + 4 * fpl, fpl)};
  State a = from;
  for (int done = 0, pass = 0; done < len; ++pass) {
    const int r = (len - done) < kUnrolledR ? (len - done) : kUnrolledR;
    const State b = (done + r == len && to) ? *to : x[pass & 1];
    if (tiled_pass(P, a, b, r, pass, sc, tape, fpl, done, st)) return 1;
    a = b;
    done += r;
  }
  return 0;
}

// A state in the workspace is u | p1 | p2 | p3 with the 256-byte-aligned plane size.
int check_args(int W, int H, int pitch, int K, int every, int n) {
  if (W <= 0 || H <= 0 || pitch < W || K < 1 || every < 1 || n < 1) return EVR_ERR_INVALID_ARG;
  if ((long long)H * n > 65535LL * 8) return EVR_ERR_INVALID_ARG;  // grid.y limit
  if ((long long)pitch * H * n >= 0x7fffffffLL) return EVR_ERR_INVALID_ARG;  // 32-bit indices
  if ((long long)K * (long long)lam_slots(W, H * n) > 0x7fffffffLL)
    return EVR_ERR_INVALID_ARG;  // the lambda sums are reduced with int indices
  return EVR_OK;
}

}  // namespace

extern "C" size_t evr_unrolled_workspace_bytes(int W, int H, int pitch, int n, int K,
                                               int every) {
  if (check_args(W, H, pitch, K, every, n)) return 0;
  return ws_layout(W, H * n, pitch, K, every, nullptr, nullptr);
}

// Forward with checkpoints.  u0, p0 (3 planes) are read; u_out, p_out written.
extern "C" int evr_unrolled_forward(const float* tx, const float* ty, const float* f,
                                    const float* u0, const float* p0, int W, int Hm, int pitch,
                                    int n, float lambda, float tau, float sigma, float u_min,
                                    float u_max, int K, int every, void* workspace,
                                    float* u_out, float* p_out, void* cuda_stream) {
  if (check_args(W, Hm, pitch, K, every, n)) return EVR_ERR_INVALID_ARG;
  const int H = Hm * n;
  if (!tx || !ty || !f || !u0 || !p0 || !workspace || !u_out || !p_out)
    return EVR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace w;
  ws_layout(W, H, pitch, K, every, (char*)workspace, &w);
  Geo g{W, H, pitch, (size_t)pitch * H, Hm};
  const size_t fpl = ((size_t)pitch * H * 4 + 255) / 256 * 256 / 4;  // floats per plane slot
  dim3 blk(kBlkX, kBlkY), grd((W + kBlkX - 1) / kBlkX, (H + kBlkY - 1) / kBlkY);
  k_metric<<<grd, blk, 0, st>>>(g, tx, ty, w.iG, w.sG);
  // checkpoint 0 = (u0, p0); checkpoint j + 1 and the result are written by the last pass
  // of segment j
  k_copy<<<grd, blk, 0, st>>>(g, u0, w.ck, 1);
  for (int k = 0; k < 3; ++k) k_copy<<<grd, blk, 0, st>>>(g, p0 + k * g.plane, w.ck + (1 + k) * fpl, 1);
  counted(5);
  const evr::Planes P = unrolled_planes(W, H, Hm, pitch, tx, ty, f, w.iG, w.sG);
  const evr::SolveConsts sc{tau, sigma, lambda, u_min, u_max, 0};
  const State out{u_out, {p_out, p_out + g.plane, p_out + 2 * g.plane}};
  // the last segment's passes also write its tape, which the backward then uses as is
  // (with every >= K: the whole tape, and the backward replays nothing)
  for (int k0 = 0, seg = 0; k0 < K; k0 += every, ++seg) {
    const int len = (K - k0 < every) ? K - k0 : every;
    const bool last = k0 + len == K;
    const State from = ws_state(w.ck + (size_t)seg * 4 * fpl, fpl);
    const State to = last ? out : ws_state(w.ck + (size_t)(seg + 1) * 4 * fpl, fpl);
    if (segment_passes(P, from, &to, len, sc, w.xs, last ? w.tape_last : nullptr, fpl, st))
      return EVR_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

// Backward from dL/du_K (gu_K) and dL/dp_K (gp_K, NULL = 0).  Outputs dL/du0, dL/dp0
// (3 planes), dL/df and glambda_dev[0] = dL/dlambda.  gu0, gp0 may be NULL.
extern "C" int evr_unrolled_backward(const float* tx, const float* ty, const float* f, int W,
                                     int Hm, int pitch, int n, float lambda, float tau,
                                     float sigma, float u_min, float u_max, int K, int every,
                                     void* workspace, const float* gu_K, const float* gp_K,
                                     float* gu0, float* gp0, float* gf, double* glambda_dev,
                                     void* cuda_stream) {
  if (check_args(W, Hm, pitch, K, every, n)) return EVR_ERR_INVALID_ARG;
  const int H = Hm * n;
  if (!tx || !ty || !f || !workspace || !gu_K || !gf || !glambda_dev) return EVR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace w;
  ws_layout(W, H, pitch, K, every, (char*)workspace, &w);
  Geo g{W, H, pitch, (size_t)pitch * H, Hm};
  Coef c{tau, sigma, lambda, u_min, u_max};
  const size_t fpl = ((size_t)pitch * H * 4 + 255) / 256 * 256 / 4;
  Geo g4 = g;
  g4.plane = fpl;
  dim3 blk(kBlkX, kBlkY), grd((W + kBlkX - 1) / kBlkX, (H + kBlkY - 1) / kBlkY);
  k_metric<<<grd, blk, 0, st>>>(g, tx, ty, w.iG, w.sG);
  const Met m{tx, ty, w.iG, w.sG};
  k_zero<<<grd, blk, 0, st>>>(g, gf, 1);
  counted(2);
  const evr::Planes PR = unrolled_planes(W, H, Hm, pitch, tx, ty, f, w.iG, w.sG);
  const evr::SolveConsts sc{tau, sigma, lambda, u_min, u_max, 0};
  // the reverse passes: the first reads the given adjoints (gu_K, and gp_K as a_p of the
  // last iteration; NULL reads as 0), then two ping-pong adjoint states in the workspace;
  // the last writes a_u straight into gu0
  RevArgs ra{};
  ra.g = g4;
  ra.c = c;
  ra.m = m;
  ra.f = f;
  ra.gf = gf;
  ra.glam = w.glam;
  rev_tiles(W, H, &ra.tiles_x, &ra.tiles_total);
  float* adj[2] = {w.adj, w.adj + 5 * fpl};
  // the two staged tape slots exceed the default 48 KiB of dynamic shared memory
  if (cudaFuncSetAttribute((const void*)k_rev_tiled,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRevSmem) !=
      cudaSuccess)
    return EVR_ERR_CUDA;
  const float* given[5] = {gu_K, gp_K, gp_K ? gp_K + g.plane : nullptr,
                           gp_K ? gp_K + 2 * g.plane : nullptr, nullptr};
  int cur = -1;  // the adjoint state's buffer; -1: the given adjoints
  const int n_ck = (K + every - 1) / every;
  for (int cseg = n_ck - 1; cseg >= 0; --cseg) {
    const int k0 = cseg * every, k1 = (k0 + every < K) ? k0 + every : K;
    // the last segment's tape is the forward's; an earlier one is replayed from its
    // checkpoint, every iteration writing the p it starts from, its v and its ubar to
    // slot k - k0 of the replay tape (the states themselves go to the ping-pong buffers
    // only).  Checkpoints and the forward's tape stay as they are: the call can repeat.
    const bool last = cseg == n_ck - 1;
    const State from = ws_state(w.ck + (size_t)cseg * 4 * fpl, fpl);
    if (!last && segment_passes(PR, from, nullptr, k1 - k0, sc, w.xs, w.tape, fpl, st))
      return EVR_ERR_CUDA;
    ra.tape = last ? w.tape_last : w.tape;
    // reverse the segment's iterations, kRevR per launch
    for (int k = k1 - 1; k >= k0;) {
      const int r = (k - k0 + 1) < kRevR ? (k - k0 + 1) : kRevR;
      const int nxt = cur == 0 ? 1 : 0;
      ra.slot_hi = k - k0;
      ra.k_hi = k;
      ra.iters = r;
      ra.first = (k == K - 1);
      for (int q = 0; q < 5; ++q) {
        ra.a_in[q] = cur < 0 ? given[q] : adj[cur] + q * fpl;
        ra.a_out[q] = adj[nxt] + q * fpl;
      }
      if (k - r < 0 && gu0) ra.a_out[0] = gu0;  // the last launch: dL/du0 itself
      const bool timed = g_timing.on && g_timing.n < kMaxTimed;
      // the tape as a 3-D tensor (x, row, plane) over the slots this launch reads, where
      // its rows are a multiple of 16 bytes (a tensor copy's stride rule); else the
      // launch reads the tape directly
      CUtensorMap tape_map{};
      const uint64_t dims[3] = {(uint64_t)W, (uint64_t)H, 5ull * (uint64_t)(ra.slot_hi + 1)};
      const uint32_t box[3] = {(uint32_t)kRevBW, (uint32_t)kRevBH, 5u};
      ra.staged = (pitch % 4 == 0) &&
                  tma::encode_f32(&tape_map, ra.tape, 3, dims, (uint64_t)pitch * sizeof(float),
                                  (uint64_t)fpl * sizeof(float), box)
                      ? 1
                      : 0;
      if (timed) cudaEventRecord(g_timing.ev[2 * g_timing.n], st);
      k_rev_tiled<<<ra.tiles_total, dim3(32, kRevNTY), ra.staged ? kRevSmem : 0, st>>>(ra,
                                                                                  tape_map);
      counted();
      if (timed) {
        cudaEventRecord(g_timing.ev[2 * g_timing.n + 1], st);
        ++g_timing.n;
        g_timing.px_iters += (long long)W * H * r;
        g_timing.px_launches += (long long)W * H;
      }
      cur = nxt;
      k -= r;
    }
  }
  if (gp0) {  // the adjoint of p_0 from the reversed iteration 0
    k_b_pupdate<<<grd, blk, 0, st>>>(g4, m, adj[cur] + fpl, adj[cur] + 4 * fpl, gp0, g.plane);
    counted();
  }
  // dL/dlambda: the K x tiles sums, in index order
  const long long nl = (long long)K * (long long)lam_slots(W, H);
  Geo gd{(int)nl, 1, (int)nl, 0, 1};
  k_red_partial<<<kRedBlocks, kRedThreads, 0, st>>>(gd, w.glam, 1, w.partials);
  k_red_final<<<1, kRedBlocks, 0, st>>>(w.partials, 1, glambda_dev);
  counted(2);
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

extern "C" int evr_data_image(const float* u_prev, const int32_t* npos, const int32_t* nneg,
                              int W, int H, int pitch, float delta_pos, float delta_neg,
                              float* f_out, void* cuda_stream) {
  if (!u_prev || !npos || !nneg || !f_out || W <= 0 || H <= 0 || pitch < W)
    return EVR_ERR_INVALID_ARG;
  Geo g{W, H, pitch, (size_t)pitch * H, H};
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  counted();
  k_data_image<<<grd, blk, 0, (cudaStream_t)cuda_stream>>>(g, u_prev, npos, nneg, delta_pos,
                                                           delta_neg, f_out);
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

// scratch: 2 double planes (pitch * H each) + 4 * 256 doubles, caller-owned.
extern "C" int evr_data_image_backward(const float* f, const float* u_prev, const int32_t* npos,
                                       const int32_t* nneg, int W, int H, int pitch,
                                       float delta_pos, float delta_neg, const float* gf,
                                       float* g_uprev, double* scratch, double* g_delta_dev,
                                       void* cuda_stream) {
  if (!f || !u_prev || !npos || !nneg || !gf || !scratch || !g_delta_dev || W <= 0 || H <= 0 ||
      pitch < W)
    return EVR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Geo g{W, H, pitch, (size_t)pitch * H, H};
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  k_data_image_bwd<<<grd, blk, 0, st>>>(g, f, u_prev, npos, nneg, delta_pos, delta_neg, gf,
                                        g_uprev, scratch);
  k_red_partial<<<kRedBlocks, kRedThreads, 0, st>>>(g, scratch, 2, scratch + 2 * g.plane);
  k_red_final<<<1, kRedBlocks, 0, st>>>(scratch + 2 * g.plane, 2, g_delta_dev);
  counted(3);
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

extern "C" int evr_unrolled_timing_start(void) {
  if (!g_timing.ev) {
    g_timing.ev = new (std::nothrow) cudaEvent_t[2 * kMaxTimed];
    if (!g_timing.ev) return EVR_ERR_OOM;
    for (int i = 0; i < 2 * kMaxTimed; ++i)
      if (cudaEventCreate(&g_timing.ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(g_timing.ev[j]);
        delete[] g_timing.ev;
        g_timing.ev = nullptr;
        return EVR_ERR_CUDA;
      }
  }
  g_timing.on = true;
  g_timing.launches = 0;
  g_timing.n = 0;
  g_timing.px_iters = 0;
  g_timing.px_launches = 0;
  return EVR_OK;
}

extern "C" int evr_unrolled_timing_stop(double* rev_ms, long long* rev_launches,
                                        long long* rev_px_iters, long long* rev_px_launches,
                                        long long* launches) {
  if (!rev_ms || !rev_launches || !rev_px_iters || !rev_px_launches || !launches)
    return EVR_ERR_INVALID_ARG;
  double ms = 0.0;
  for (int i = 0; i < g_timing.n; ++i) {
    float t = 0.0f;
    if (cudaEventSynchronize(g_timing.ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, g_timing.ev[2 * i], g_timing.ev[2 * i + 1]) != cudaSuccess)
      return EVR_ERR_CUDA;
    ms += t;
  }
  *rev_ms = ms;
  *rev_launches = g_timing.n;
  *rev_px_iters = g_timing.px_iters;
  *rev_px_launches = g_timing.px_launches;
  *launches = g_timing.launches;
  g_timing.on = false;
  return EVR_OK;
}
