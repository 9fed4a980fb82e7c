// evr_grad.cu -- differentiation of one packet's solve (K unrolled iterations of
// Eq. cont_iterates with Eq. update_rules) by a hand-written adjoint, with (u, p)
// checkpoints every `every` iterations.  The iterations themselves (forward, and the
// recomputation of each checkpoint segment) are the solver's tiled FP32 passes; the
// adjoint kernels use IEEE division and square root; the lambda gradient and the
// contrast-threshold sums are reduced in FP64.
//
// All memory (inputs, outputs and the workspace) belongs to the caller; nothing here
// allocates.  Planes are H rows of `pitch` floats; a dual variable is 3 such planes
// back to back (plane stride pitch * H).
#include <cuda_runtime.h>

#include "../../include/evr.h"
#include "evr_internal.cuh"

namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

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

// M^T p with M = (1/G)[[1+b^2,-ab],[-ab,1+a^2],[a,b]] (Eq. 3)
__device__ __forceinline__ void MT(float a, float b, float iG, float p1, float p2, float p3,
                                   float& q1, float& q2) {
  float z = b * p1 - a * p2;
  q1 = iG * (p1 + b * z + a * p3);
  q2 = iG * (p2 - a * z + b * p3);
}

__device__ __forceinline__ void Mg(float a, float b, float iG, float ux, float uy, float& g1,
                                   float& g2, float& g3) {
  float w = b * ux - a * uy;
  g1 = iG * (ux + b * w);
  g2 = iG * (uy - a * w);
  g3 = iG * (a * ux + b * uy);
}

// div(M^T q) at (x, y) for a 3-plane field q (div_g q = -L_g^T q); yl = row in the member
__device__ __forceinline__ float div_g(const Geo& g, const Met& m, const float* q, int x, int yl,
                                       size_t i) {
  float a, b, iG, q1, q2, q1m = 0.0f, q2m = 0.0f, d;
  metric(m, i, a, b, iG);
  MT(a, b, iG, q[i], q[g.plane + i], q[2 * g.plane + i], q1, q2);
  if (x > 0) {
    metric(m, i - 1, a, b, iG);
    MT(a, b, iG, q[i - 1], q[g.plane + i - 1], q[2 * g.plane + i - 1], q1m, d);
  }
  if (yl > 0) {
    const size_t j = i - g.pitch;
    metric(m, j, a, b, iG);
    MT(a, b, iG, q[j], q[g.plane + j], q[2 * g.plane + j], d, q2m);
  }
  return ((x < g.W - 1) ? q1 : 0.0f) - q1m + ((yl < g.Hm - 1) ? q2 : 0.0f) - q2m;
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

// ---- backward of one iteration from state (u, p) ----
// step 1: the adjoint through the projection, apt = J_proj ap_next, written scaled by
// sigma (it is what L_g^T acts on); ubar is this iteration's, from the tape.
// ap_next, the adjoint of the next iteration's p, is read from `ap` for the last
// iteration, else formed here from that iteration's sigma apt (in `sapt`, updated in
// place: each pixel reads and writes only its own entries) and tau a_v (`tav`):
// ap_next = apt - L_g(tau a_v).
__global__ void k_b_dual(Geo g, Coef c, Met m, const float* ub, const float* p,
                         const float* ap, const float* tav, float* sapt) {
  PIXEL
  float g1, g2, g3;
  float a1, a2, a3;
  if (tav) {
    Lg(g, m, tav, x, yl, i, g1, g2, g3);
    a1 = sapt[i] / c.sigma - g1;
    a2 = sapt[g.plane + i] / c.sigma - g2;
    a3 = sapt[2 * g.plane + i] / c.sigma - g3;
  } else {
    a1 = ap[i];
    a2 = ap[g.plane + i];
    a3 = ap[2 * g.plane + i];
  }
  Lg(g, m, ub, x, yl, i, g1, g2, g3);
  const float sG = m.sG[i];
  float t1 = p[i] + c.sigma * g1, t2 = p[g.plane + i] + c.sigma * g2,
        t3 = p[2 * g.plane + i] + c.sigma * g3;
  float nrm = sqrtf(t1 * t1 + t2 * t2 + t3 * t3);
  if (nrm > sG) {
    float dot = (t1 * a1 + t2 * a2 + t3 * a3) / (nrm * nrm);
    float s = sG / nrm;
    a1 = s * (a1 - t1 * dot);
    a2 = s * (a2 - t2 * dot);
    a3 = s * (a3 - t3 * dot);
  }
  sapt[i] = c.sigma * a1;
  sapt[g.plane + i] = c.sigma * a2;
  sapt[2 * g.plane + i] = c.sigma * a3;
}

// step 2: a_ub = -div_g(sigma apt); the primal step backwards from this iteration's
// argument v (from the tape).  Writes the new au (in place), tau * a_v, accumulates df, and writes this
// block's FP64 sum of the lambda-gradient terms to glam_part[blk] (one slot per block and
// iteration: the final sum has a fixed order).
__global__ void __launch_bounds__(256) k_b_primal(Geo g, Coef c, Met m, const float* f,
                                                  const float* v_in, const float* sapt,
                                                  float* au, float* tav, float* gf,
                                                  double* glam_part) {
  __shared__ double s_l[256];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  double lam_term = 0.0;
  if (x < g.W && y < g.H) {
    const size_t i = (size_t)y * g.pitch + x;
    const int yl = y % g.Hm;
    const float sG = m.sG[i];
    const float aub = -div_g(g, m, sapt, x, yl, i);
    const float v = v_in[i];
    const float beta = c.tau * c.lambda * sG;
    const float d = v - beta;
    const float fi = f[i];
    const float s = sqrtf(d * d + 4.0f * beta * fi);
    const float r = 0.5f * (d + s);
    const float aun = au[i] + 2.0f * aub;
    const float ar = (r < c.u_min || r > c.u_max) ? 0.0f : aun;
    const float av = ar * 0.5f * (1.0f + d / s);
    gf[i] += ar * (beta / s);
    lam_term = (double)(ar * 0.5f * (-1.0f + (2.0f * fi - v + beta) / s)) *
               ((double)c.tau * (double)sG);
    au[i] = -aub + av;
    tav[i] = c.tau * av;
  }
  s_l[t] = lam_term;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) s_l[t] += s_l[t + h];
    __syncthreads();
  }
  if (t == 0) glam_part[blockIdx.y * gridDim.x + blockIdx.x] = s_l[0];
}

// step 3: ap = apt - L_g(tau a_v)   (apt = sapt / sigma)
__global__ void k_b_pupdate(Geo g, Coef c, Met m, const float* sapt, const float* tav,
                            float* ap) {
  PIXEL
  float g1, g2, g3;
  Lg(g, m, tav, x, yl, i, g1, g2, g3);
  ap[i] = sapt[i] / c.sigma - g1;
  ap[g.plane + i] = sapt[g.plane + i] / c.sigma - g2;
  ap[2 * g.plane + i] = sapt[2 * g.plane + i] / c.sigma - g3;
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
  terms[i] = (double)gf[i] * (double)f[i] * (double)npos[i];
  terms[g.plane + i] = -(double)gf[i] * (double)f[i] * (double)nneg[i];
}

struct Workspace {
  float* ck;       // n_ck checkpoints x 4 planes
  float* tape;     // max(every, 2) + 1 slots x 6 planes: u p1 p2 p3 of a state, then the
                   // v and ubar of the iteration that starts from it
  float* sapt;     // 3 planes
  float* au;       // 1 plane
  float* ap;       // 3 planes
  float* tav;      // 1 plane
  float* xs;       // 2 states x 4 planes: ping-pong buffers of the recomputing passes
  float* iG;       // 1 plane: 1/G
  float* sG;       // 1 plane: sqrt(G)
  double* glam;    // K x (blocks of the pixel grid): per-block lambda-gradient sums
  double* partials;  // 4 * kRedBlocks doubles
};

constexpr int kBlkX = 32, kBlkY = 8;  // pixel-kernel block

size_t pixel_blocks(int W, int H) {
  return (size_t)((W + kBlkX - 1) / kBlkX) * ((H + kBlkY - 1) / kBlkY);
}

size_t ws_layout(int W, int H, int pitch, int K, int every, char* base, Workspace* w) {
  const size_t plane = (size_t)pitch * H;
  const size_t fpl = (plane * 4 + 255) / 256 * 256;
  const int n_ck = (K + every - 1) / every;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) / 256 * 256;
    return base ? base + o : nullptr;
  };
  Workspace t;
  t.ck = (float*)take(fpl * 4 * (size_t)(n_ck > 0 ? n_ck : 1));
  t.tape = (float*)take(fpl * 6 * (size_t)((every > 2 ? every : 2) + 1));
  t.sapt = (float*)take(fpl * 3);
  t.au = (float*)take(fpl);
  t.ap = (float*)take(fpl * 3);
  t.tav = (float*)take(fpl);
  t.xs = (float*)take(fpl * 8);
  t.iG = (float*)take(fpl);
  t.sG = (float*)take(fpl);
  t.glam = (double*)take(sizeof(double) * (size_t)K * pixel_blocks(W, H));
  t.partials = (double*)take(sizeof(double) * 4 * kRedBlocks);
  if (w) *w = t;
  return off;
}

// The iterations of the forward pass and of the reverse pass's recomputation run as the
// solver's tiled passes (FP32, one pixel pair per thread, a kUnrolledR-pixel halo) over
// the stacked images; their per-pixel arithmetic does not depend on how the iterations
// are split into launches, so the recomputed states equal the forward's bit for bit.
constexpr int kUnrolledR = 5;

// The two ping-pong states a0, a1 (u | p1 | p2 | p3, plane stride fpl floats) and the
// packet's planes as the tiled passes' descriptor.
evr::Planes unrolled_planes(int W, int H, int Hm, int pitch, const float* tx, const float* ty,
                            const float* f, float* iG, float* sG, float* a0, float* a1,
                            size_t fpl) {
  evr::Planes P{};
  P.W = W;
  P.H = H;
  P.Hm = Hm;
  P.pitch = pitch;
  float* st[2] = {a0, a1};
  for (int b = 0; b < 2; ++b) {
    P.u[b] = st[b];
    P.p1[b] = st[b] + fpl;
    P.p2[b] = st[b] + 2 * fpl;
    P.p3[b] = st[b] + 3 * fpl;
  }
  P.tx = const_cast<float*>(tx);
  P.ty = const_cast<float*>(ty);
  P.f = const_cast<float*>(f);
  P.iG = iG;
  P.sG = sG;
  P.storage = 0;
  return P;
}

// A state in the workspace is u | p1 | p2 | p3 with the 256-byte-aligned plane size.
int check_args(int W, int H, int pitch, int K, int every, int n) {
  if (W <= 0 || H <= 0 || pitch < W || K < 1 || every < 1 || n < 1) return EVR_ERR_INVALID_ARG;
  if ((long long)H * n > 65535LL * 8) return EVR_ERR_INVALID_ARG;  // grid.y limit
  if ((long long)K * (long long)pixel_blocks(W, H * n) > 0x7fffffffLL)
    return EVR_ERR_INVALID_ARG;  // per-block lambda sums are indexed with int
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
  // state buffers: two ping-pong states in the tape area (u | p1 p2 p3)
  float* su[2] = {w.tape, w.tape + 4 * fpl};
  Geo g4 = g;
  g4.plane = fpl;  // states use the aligned plane stride
  // copy (u0, p0) into state 0
  k_copy<<<grd, blk, 0, st>>>(g, u0, su[0], 1);
  for (int k = 0; k < 3; ++k) k_copy<<<grd, blk, 0, st>>>(g, p0 + k * g.plane, su[0] + (1 + k) * fpl, 1);
  const evr::Planes P = unrolled_planes(W, H, Hm, pitch, tx, ty, f, w.iG, w.sG, su[0], su[1],
                                        fpl);
  const evr::SolveConsts sc{tau, sigma, lambda, u_min, u_max, 0};
  int cur = 0;
  for (int k0 = 0; k0 < K; k0 += every) {  // a checkpoint, then the segment's passes
    k_copy<<<grd, blk, 0, st>>>(g4, su[cur], w.ck + (size_t)(k0 / every) * 4 * fpl, 4);
    for (int left = (K - k0 < every) ? K - k0 : every, pass = 0; left > 0; ++pass) {
      const int r = left < kUnrolledR ? left : kUnrolledR;
      if (evr::launch_tiled_tape(P, kUnrolledR, cur, r, pass, sc, nullptr, 0, 0, st))
        return EVR_ERR_CUDA;
      cur ^= 1;
      left -= r;
    }
  }
  k_copy<<<grd, blk, 0, st>>>(g, su[cur], u_out, 1);
  for (int k = 0; k < 3; ++k) k_copy<<<grd, blk, 0, st>>>(g, su[cur] + (1 + k) * fpl, p_out + k * g.plane, 1);
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
  const size_t nblk = pixel_blocks(W, H);
  k_metric<<<grd, blk, 0, st>>>(g, tx, ty, w.iG, w.sG);
  const Met m{tx, ty, w.iG, w.sG};
  // adjoint of the final state: au = gu_K, ap = gp_K or 0; gf = 0
  k_copy<<<grd, blk, 0, st>>>(g, gu_K, w.au, 1);
  if (gp_K) {
    for (int k = 0; k < 3; ++k) k_copy<<<grd, blk, 0, st>>>(g, gp_K + k * g.plane, w.ap + k * fpl, 1);
  } else {
    k_zero<<<grd, blk, 0, st>>>(g4, w.ap, 3);
  }
  k_zero<<<grd, blk, 0, st>>>(g, gf, 1);
  const evr::Planes PR =
      unrolled_planes(W, H, Hm, pitch, tx, ty, f, w.iG, w.sG, w.xs, w.xs + 4 * fpl, fpl);
  const evr::SolveConsts sc{tau, sigma, lambda, u_min, u_max, 0};
  const int n_ck = (K + every - 1) / every;
  for (int cseg = n_ck - 1; cseg >= 0; --cseg) {
    const int k0 = cseg * every, k1 = (k0 + every < K) ? k0 + every : K;
    // recompute iterations k0 .. k1-1 into the tape (slot j: state k0 + j, then the v
    // and ubar of iteration k0 + j): the checkpoint into slot 0 and into the passes'
    // first ping-pong state, then tiled passes that write what every iteration computes
    k_copy<<<grd, blk, 0, st>>>(g4, w.ck + (size_t)cseg * 4 * fpl, w.tape, 4);
    k_copy<<<grd, blk, 0, st>>>(g4, w.ck + (size_t)cseg * 4 * fpl, w.xs, 4);
    for (int done = 0, pass = 0, src = 0; done < k1 - k0; ++pass) {
      const int left = k1 - k0 - done;
      const int r = left < kUnrolledR ? left : kUnrolledR;
      if (evr::launch_tiled_tape(PR, kUnrolledR, src, r, pass, sc, w.tape, (long long)fpl,
                                 done, st))
        return EVR_ERR_CUDA;
      src ^= 1;
      done += r;
    }
    for (int k = k1 - 1; k >= k0; --k) {
      const float* s0 = w.tape + (size_t)(k - k0) * 6 * fpl;
      // the adjoint of p_{k+1}: the given one for the last iteration, else from the
      // reversed iteration k + 1 (fused here)
      k_b_dual<<<grd, blk, 0, st>>>(g4, c, m, s0 + 5 * fpl, s0 + fpl, w.ap,
                                    k == K - 1 ? nullptr : w.tav, w.sapt);
      k_b_primal<<<grd, blk, 0, st>>>(g4, c, m, f, s0 + 4 * fpl, w.sapt, w.au, w.tav, gf,
                                      w.glam + (size_t)k * nblk);
    }
  }
  if (gu0) k_copy<<<grd, blk, 0, st>>>(g, w.au, gu0, 1);
  if (gp0) {  // the adjoint of p_0 from the reversed iteration 0
    k_b_pupdate<<<grd, blk, 0, st>>>(g4, c, m, w.sapt, w.tav, w.ap);
    for (int k = 0; k < 3; ++k) k_copy<<<grd, blk, 0, st>>>(g, w.ap + k * fpl, gp0 + k * g.plane, 1);
  }
  // dL/dlambda: the K x nblk per-block sums, in index order
  const long long nl = (long long)K * (long long)nblk;
  Geo gd{(int)nl, 1, (int)nl, 0, 1};
  k_red_partial<<<kRedBlocks, kRedThreads, 0, st>>>(gd, w.glam, 1, w.partials);
  k_red_final<<<1, kRedBlocks, 0, st>>>(w.partials, 1, glambda_dev);
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}

extern "C" int evr_data_image(const float* u_prev, const int32_t* npos, const int32_t* nneg,
                              int W, int H, int pitch, float delta_pos, float delta_neg,
                              float* f_out, void* cuda_stream) {
  if (!u_prev || !npos || !nneg || !f_out || W <= 0 || H <= 0 || pitch < W)
    return EVR_ERR_INVALID_ARG;
  Geo g{W, H, pitch, (size_t)pitch * H, H};
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
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
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}
