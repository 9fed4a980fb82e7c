// evr_tile.cuh -- one CTA's extended tile of the tiled primal-dual solvers (Eq.
// cont_iterates with Eq. update_rules): storage formats of p and ubar, paired FP32
// arithmetic, and the Tile whose iterate() runs one iteration on register-resident
// state.  Shared by the multi-launch and persistent solvers (evr_solvers.cu) and the
// cluster solver (evr_cluster.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "evr_internal.cuh"

namespace evr {

// ---------------------------------------------------------------- storage formats
// p (between launches, in HBM/L2) and ubar (in shared memory) are stored as ST; all
// arithmetic is FP32.  With a 16-bit ST both are rounded to ST every iteration (p
// after the projection, ubar when formed), so the result does not depend on how the
// iterations are split into launches.
template <typename ST>
struct Stor;
template <>
struct Stor<float> {
  static __device__ __forceinline__ float ld(const float* a, size_t i) { return a[i]; }
  static __device__ __forceinline__ float ldcg(const float* a, size_t i) { return __ldcg(a + i); }
  static __device__ __forceinline__ float enc(float v) { return v; }
  static __device__ __forceinline__ float dec(float v) { return v; }
  static __device__ __forceinline__ float rnd(float v) { return v; }
  using T2 = float2;  // two vertically adjacent pixels
  static __device__ __forceinline__ float2 enc2(float2 v) { return v; }
  static __device__ __forceinline__ float2 dec2(float2 v) { return v; }
};
template <>
struct Stor<__half> {
  static __device__ __forceinline__ float ld(const __half* a, size_t i) { return __half2float(a[i]); }
  static __device__ __forceinline__ float ldcg(const __half* a, size_t i) {
    return __half2float(__ldcg(a + i));
  }
  static __device__ __forceinline__ __half enc(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float dec(__half v) { return __half2float(v); }
  static __device__ __forceinline__ float rnd(float v) { return __half2float(__float2half_rn(v)); }
  using T2 = __half2;
  static __device__ __forceinline__ __half2 enc2(float2 v) { return __floats2half2_rn(v.x, v.y); }
  static __device__ __forceinline__ float2 dec2(__half2 v) { return __half22float2(v); }
};
template <>
struct Stor<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* a, size_t i) {
    return __bfloat162float(a[i]);
  }
  static __device__ __forceinline__ float ldcg(const __nv_bfloat16* a, size_t i) {
    return __bfloat162float(__ldcg(a + i));
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ float rnd(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
  }
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ __nv_bfloat162 enc2(float2 v) {
    return __floats2bfloat162_rn(v.x, v.y);
  }
  static __device__ __forceinline__ float2 dec2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
};

// ---------------------------------------------------------------- one tile
template <int KX, int KY, int NTY, typename ST = float>
struct TileSmem {
  static constexpr int EW = 32 * KX, EH = NTY * KY;
  // q1 and ubar of rows 2r and 2r + 1 interleaved in row r (the two pixels of a pair):
  // one 64-bit (32-bit for 16-bit ST) access per pair
  float2 q1[EH / 2][EW + 1];             // column 0: left pad (zero)
  typename Stor<ST>::T2 ub[EH / 2][EW + 1];  // column EW: right pad (zero)
  float q2last[NTY + 1][EW];  // row ty + 1: q2 of strip ty's last pixel; row 0 pad
  ST ubfirst[NTY + 1][EW];    // row ty: ubar of strip ty's first pixel; row NTY pad
};

// Paired FP32 arithmetic: one packed instruction (FFMA2 / FADD2 / FMUL2 on sm_100 and
// later) for two pixels, each half rounded exactly like its scalar counterpart.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
// MUFU reciprocal square root and reciprocal (approximate, a few ulp), subnormal
// arguments flushed to zero.  Their arguments here are positive normal numbers, or
// zero where the (infinite) result is not selected, so the flush never applies; the
// forms that keep subnormals cost extra instructions per call (18 % more instructions
// per iteration measured on the 346 x 260 stream).
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_mufu(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// element h of a pair (h a compile-time constant after unrolling)
__device__ __forceinline__ float& el(float2& v, int h) { return h ? v.y : v.x; }

// Halo exchange with neighbouring CTAs inside one iteration (the cluster solver's
// ClusterX, evr_cluster.cu); the tiled and persistent solvers exchange nothing.
struct NoExchange {
  static constexpr bool kOn = false;
  __device__ __forceinline__ void send_q(int, int, float2, bool, int, float) {}
  __device__ __forceinline__ void send_u(int, int, float2, bool) {}
  __device__ __forceinline__ void after_bar1() {}
  __device__ __forceinline__ void after_bar2() {}
};

// The extended tile held by one CTA.  Thread (tx, ty) holds pixels
// (tx + 32 kx, KY ty + ky): pixel-local state in registers, vertical neighbours
// inside the strip in registers, and only q1 (read at x-1), ubar (read at x+1) and
// the strip ends in shared memory -- for tiles one warp wide (KX = 1) without a
// neighbour exchange, q1 and ubar of the x neighbours come from the adjacent lanes by
// warp shuffles and only the strip ends go through shared memory.  Lanes 0 and 31 then
// read their own value where the shared-memory form read a zero pad: both are halo
// columns (every tile has R >= 1), whose values are inexact after the first iteration
// either way and reach the owned pixels in no case (the exact region shrinks by one
// pixel per side and iteration from the tile's edge whatever the edge reads).  Pixels k = 2j and 2j + 1 (vertical neighbours in
// one strip, KY even) form pair j of every per-pixel array and are updated by paired
// instructions.  The image-border rules (forward differences zero on the last
// column/row, the matching divergence) are per-pixel 0/1 factors: q is zero where its
// difference does not exist and off the sensor, so the divergence needs no tests.
template <int KX, int KY, int NTY, typename ST = float>
struct Tile {
  static_assert(KY % 2 == 0, "pairs are vertical neighbours within a strip");
  static constexpr int EW = 32 * KX, EH = NTY * KY, K = KX * KY, KP = K / 2;
  using S = Stor<ST>;
  float2 u[KP], p1[KP], p2[KP], p3[KP];  // iterated state
  // packet constants.  With M = (1/G)[[1+b^2, -ab], [-ab, 1+a^2], [a, b]] (Eq. 3;
  // a = L_x t, b = L_y t) and the border masks m_x, m_y (1 where the forward difference
  // in x (y) exists, else 0): E1..E3 = m_x (M11, M12, M31), E4..E6 = m_y (M12, M22, M32).
  // Then q = (m_x (M^T p)_1, m_y (M^T p)_2) = (E1 p1 + E2 p2 + E3 p3, E4 p1 + E5 p2 + E6 p3)
  // and M (m_x dx, m_y dy) = (E1 dx + E4 dy, E2 dx + E5 dy, E3 dx + E6 dy): the same six
  // coefficients serve both operators.  sqrt(G); data term: KL (-beta, 4 beta f,
  // 2 beta f) with beta = tau lambda sqrt(G), or L2 (1 / (1 + beta), beta f, unused).
  float2 E1[KP], E2[KP], E3[KP], E4[KP], E5[KP], E6[KP], SG[KP];
  float2 D1[KP], D2[KP], D3[KP];
  float2 vs[KP], ubs[KP];  // tape mode: the last iteration's primal argument and ubar
  int gx0, gy0, R, OW, OH;
  int ox0, ox1, oy0, oy1;  // owned pixels: local x in [ox0, ox1), y in [oy0, oy1)

  __device__ __forceinline__ int lx(int k) const { return threadIdx.x + 32 * (k / KY); }
  __device__ __forceinline__ int ly(int k) const { return KY * threadIdx.y + (k % KY); }

  __device__ __forceinline__ void setup(int tile, int tiles_x, int R_) {
    R = R_;
    OW = EW - 2 * R;
    OH = EH - 2 * R;
    gx0 = (tile % tiles_x) * OW - R;
    gy0 = (tile / tiles_x) * OH - R;
    ox0 = R;
    ox1 = R + OW;
    oy0 = R;
    oy1 = R + OH;
  }

  // Cluster solver: CTA (rx, ry) of a cluster of CX x CY CTAs whose tiles form one
  // super-tile, an owned region of (CX EW - 2R) x (CY EH - 2R) pixels plus an R-pixel
  // halo on every side (R = 0: one super-tile covers the sensor).  Super-tile `sup` of
  // sup_x per row.  The owned pixels of this CTA are its share of the owned region.
  __device__ __forceinline__ void setup_cluster(int sup, int sup_x, int CX, int CY, int rx,
                                                int ry, int R_) {
    R = R_;
    const int SOW = CX * EW - 2 * R, SOH = CY * EH - 2 * R;
    gx0 = (sup % sup_x) * SOW - R + rx * EW;
    gy0 = (sup / sup_x) * SOH - R + ry * EH;
    ox0 = max(0, R - rx * EW);
    ox1 = min(EW, R + SOW - rx * EW);
    oy0 = max(0, R - ry * EH);
    oy1 = min(EH, R + SOH - ry * EH);
    OW = ox1 - ox0;
    OH = oy1 - oy0;
  }

  __device__ __forceinline__ static void zero_pads(TileSmem<KX, KY, NTY, ST>& sm) {
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int i = tid; i < EH / 2; i += 32 * NTY) {
      sm.q1[i][0] = dup2(0.0f);
      sm.ub[i][EW] = S::enc2(dup2(0.0f));
    }
    for (int i = tid; i < EW; i += 32 * NTY) {
      sm.q2last[0][i] = 0.0f;
      sm.ubfirst[NTY][i] = S::enc(0.0f);
    }
  }

  __device__ __forceinline__ bool on(int k, int W, int H) const {
    const int gx = gx0 + lx(k), gy = gy0 + ly(k);
    return gx >= 0 && gx < W && gy >= 0 && gy < H;
  }
  __device__ __forceinline__ bool owned(int k) const {
    const int x = lx(k), y = ly(k);
    return x >= ox0 && x < ox1 && y >= oy0 && y < oy1;
  }
  __device__ __forceinline__ bool band(int k) const {  // owned, within R of the owned border
    const int x = lx(k), y = ly(k);
    return owned(k) && (x < 2 * R || x >= OW || y < 2 * R || y >= OH);
  }
  __device__ __forceinline__ size_t gidx(const Planes& P, int k) const {
    return (size_t)(gy0 + ly(k)) * P.pitch + (gx0 + lx(k));
  }

  // Packet constants of pixel k from its metric (a = L_x t, b = L_y t, 1/G, sqrt(G)), f
  // and its border masks.
  __device__ __forceinline__ void set_consts(int k, float a, float b, float ig, float sg,
                                             float f, float mx, float my, float tl,
                                             const SolveConsts& c) {
    const int j = k >> 1, h = k & 1;
    const float m12 = -(ig * (a * b));
    el(E1[j], h) = mx * (ig * fmaf(b, b, 1.0f));
    el(E2[j], h) = mx * m12;
    el(E3[j], h) = mx * (ig * a);
    el(E4[j], h) = my * m12;
    el(E5[j], h) = my * (ig * fmaf(a, a, 1.0f));
    el(E6[j], h) = my * (ig * b);
    el(SG[j], h) = sg;
    const float beta = tl * sg;
    if (c.data_term) {  // Eq. 7: u+ = (v + beta f) / (1 + beta)
      el(D1[j], h) = 1.0f / (1.0f + beta);
      el(D2[j], h) = beta * f;
      el(D3[j], h) = 0.0f;
    } else {
      el(D1[j], h) = -beta;
      el(D2[j], h) = 4.0f * beta * f;
      el(D3[j], h) = 2.0f * beta * f;
    }
  }

  // Packet constants from the planes the prologue wrote.
  __device__ __forceinline__ void load_consts(const Planes& P, const SolveConsts& c) {
    const float tl = c.tau * c.lambda;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float a = 0.0f, b = 0.0f, ig = 1.0f, sg = 1.0f, f = 1.0f, mx = 0.0f, my = 0.0f;
      if (on(k, P.W, P.H)) {  // off the sensor: finite filler, masked out of every term
        const size_t i = gidx(P, k);
        a = P.tx[i];
        b = P.ty[i];
        ig = P.iG[i];
        sg = P.sG[i];
        f = P.f[i];
        mx = (gx0 + lx(k) < P.W - 1) ? 1.0f : 0.0f;
        const int gy = gy0 + ly(k);
        my = ((P.Hm == P.H ? gy : gy % P.Hm) < P.Hm - 1) ? 1.0f : 0.0f;
      }
      set_consts(k, a, b, ig, sg, f, mx, my, tl, c);
    }
  }

  // Packet constants computed here, as the prologue computes them (the first pass of a
  // packet whose front launch is fused into it): time surface, metric and f = u exp(...)
  // from the integrated events, the current u (load_state first) and the stream clock.
  // The owned pixels' values are written to the planes for the later passes.
  __device__ __forceinline__ void front_consts(const Planes& P, const SolveConsts& c,
                                               const PrologueConsts& pc) {
    const float tl = c.tau * c.lambda;
    const long long clock = P.sc->clock;
    const long long t_init = P.sc->t_init_set ? P.sc->t_init : clock;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float a = 0.0f, b = 0.0f, ig = 1.0f, sg = 1.0f, f = 1.0f, mx = 0.0f, my = 0.0f;
      if (on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        const int gx = gx0 + lx(k), gy = gy0 + ly(k);
        const float t0 = time_surface(P.t_last[i], clock, t_init, pc);
        a = (gx < P.W - 1) ? surface_diff(time_surface(P.t_last[i + 1], clock, t_init, pc), t0)
                           : 0.0f;
        b = (gy < P.H - 1)
                ? surface_diff(time_surface(P.t_last[i + P.pitch], clock, t_init, pc), t0)
                : 0.0f;
        const float G = metric_G(a, b);
        ig = 1.0f / G;
        sg = sqrtf(G);
        f = data_image(el(u[k >> 1], k & 1), P.npos[i], P.nneg[i], pc);
        mx = (gx < P.W - 1) ? 1.0f : 0.0f;
        my = (gy % P.Hm < P.Hm - 1) ? 1.0f : 0.0f;
        if (owned(k)) {
          P.tx[i] = a;
          P.ty[i] = b;
          P.iG[i] = ig;
          P.sG[i] = sg;
          P.f[i] = f;
        }
      }
      set_consts(k, a, b, ig, sg, f, mx, my, tl, c);
    }
  }

  // As front_consts, for a packet that is not yet in the planes: its events over the
  // extended tile plus one column and one row (mw = EW + 1 per map row) are merged from
  // shared-memory maps -- mt the latest event time of each pixel (kNeverFired: none),
  // mc its event counts (positive in the low, negative in the high 16 bits) -- with the
  // t_last and counts already in the planes, exactly as the push followed by the
  // prologue would leave them (max and sum do not depend on the order).  clock and t_init
  // are the stream's after the packet.  The owned pixels' merged t_last is written back.
  // The event counts of this thread's pixels (0 off the sensor).
  __device__ __forceinline__ void load_counts(const Planes& P, int* np, int* nn) const {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      np[k] = 0;
      nn[k] = 0;
      if (on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        np[k] = P.npos[i];
        nn[k] = P.nneg[i];
      }
    }
  }

  // front_consts with the packet integrated in shared memory (the push fused into the
  // first pass): mt holds the merged t_last of the extended tile plus one column and row
  // (row stride EW + 1), mc the packet's events per pixel (positive in the low 16 bits,
  // negative in the high), np and nn the counts before the packet.  The owned pixels'
  // constants are written to the planes, and their t_last where events hit them.
  __device__ __forceinline__ void front_consts_push(const Planes& P, const SolveConsts& c,
                                                    const PrologueConsts& pc,
                                                    const long long* mt, const int* mc,
                                                    const int* np, const int* nn,
                                                    long long clock, long long t_init) {
    constexpr int MW = EW + 1;
    const float tl = c.tau * c.lambda;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float a = 0.0f, b = 0.0f, ig = 1.0f, sg = 1.0f, f = 1.0f, mx = 0.0f, my = 0.0f;
      if (on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        const int gx = gx0 + lx(k), gy = gy0 + ly(k), m = ly(k) * MW + lx(k);
        const long long t_own = mt[m];
        const float t0 = time_surface(t_own, clock, t_init, pc);
        a = (gx < P.W - 1) ? surface_diff(time_surface(mt[m + 1], clock, t_init, pc), t0)
                           : 0.0f;
        b = (gy < P.H - 1) ? surface_diff(time_surface(mt[m + MW], clock, t_init, pc), t0)
                           : 0.0f;
        const float G = metric_G(a, b);
        ig = 1.0f / G;
        sg = sqrtf(G);
        const int cnt = mc[m];
        f = data_image(el(u[k >> 1], k & 1), np[k] + (cnt & 0xffff), nn[k] + (cnt >> 16), pc);
        mx = (gx < P.W - 1) ? 1.0f : 0.0f;
        my = (gy % P.Hm < P.Hm - 1) ? 1.0f : 0.0f;
        if (owned(k)) {
          P.tx[i] = a;
          P.ty[i] = b;
          P.iG[i] = ig;
          P.sG[i] = sg;
          P.f[i] = f;
          if (cnt != 0) P.t_last[i] = t_own;
        }
      }
      set_consts(k, a, b, ig, sg, f, mx, my, tl, c);
    }
  }

  // The owned pixels' event counts, consumed by the previous pass's front_consts.
  __device__ __forceinline__ void clear_counts(const Planes& P) const {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (owned(k) && on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        P.npos[i] = 0;
        P.nneg[i] = 0;
      }
  }

  // Tape mode: the dual state p_k the iteration starts from (before it), then its primal
  // argument v and ubar (after it), into one slot of 5 FP32 planes p1 p2 p3 v ubar of
  // `plane` floats each, at the owned pixels' indices ti[k] (~0u: not written).
  __device__ __forceinline__ void store_tape_p(float* slot, unsigned plane,
                                               const unsigned* ti) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = k >> 1, h = k & 1;
      if (ti[k] != ~0u) {
        slot[ti[k]] = el(p1[j], h);
        slot[plane + ti[k]] = el(p2[j], h);
        slot[2 * plane + ti[k]] = el(p3[j], h);
      }
    }
  }
  __device__ __forceinline__ void store_tape_vub(float* slot, unsigned plane,
                                                 const unsigned* ti) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = k >> 1, h = k & 1;
      if (ti[k] != ~0u) {
        slot[3 * plane + ti[k]] = el(vs[j], h);
        slot[4 * plane + ti[k]] = el(ubs[j], h);
      }
    }
  }

  // Iterated state (u, p) from buffer buf.
  __device__ __forceinline__ void load_state(const Planes& P, int buf) {
    const float* U = P.u[buf];
    const ST *P1 = (const ST*)P.p1[buf], *P2 = (const ST*)P.p2[buf], *P3 = (const ST*)P.p3[buf];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = k >> 1, h = k & 1;
      if (on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        el(u[j], h) = U[i];
        el(p1[j], h) = S::ld(P1, i);
        el(p2[j], h) = S::ld(P2, i);
        el(p3[j], h) = S::ld(P3, i);
      } else {
        el(u[j], h) = 1.0f;
        el(p1[j], h) = el(p2[j], h) = el(p3[j], h) = 0.0f;
      }
    }
  }

  __device__ __forceinline__ void load(const Planes& P, int buf, const SolveConsts& c) {
    load_consts(P, c);
    load_state(P, buf);
  }

  // One primal-dual iteration over the extended tile (two CTA barriers).
  // L2: the data term of Eq. 7 instead of KL (a template argument, so that the loop body
  // carries no branch on it).
  // SAVE: keep this iteration's primal argument v and ubar in vs, ubs (tape mode).
  // X: exchange of the tile's edge values with neighbouring CTAs (cluster solver): q of
  // the last column and row after they are formed, ubar of the first column and row
  // after the primal step, and the waits for the neighbours' values after each barrier.
  template <bool L2, bool SAVE = false, class X = NoExchange>
  __device__ __forceinline__ void iterate(TileSmem<KX, KY, NTY, ST>& sm, const SolveConsts& c,
                                          X* xc = nullptr) {
    // one warp across the tile and no exchange with other CTAs: x neighbours by shuffles
    constexpr bool kShfl = KX == 1 && !X::kOn;
    float2 q1r[KP], q2r[KP];
    const int ty0 = threadIdx.y;
    const float2 one_neg = dup2(-1.0f);
    // q = M^T p, zero where the matching forward difference does not exist
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int k0 = 2 * j, k1 = k0 + 1;
      q1r[j] = fma2(E3[j], p3[j], fma2(E2[j], p2[j], mul2(E1[j], p1[j])));
      q2r[j] = fma2(E6[j], p3[j], fma2(E5[j], p2[j], mul2(E4[j], p1[j])));
      if constexpr (!kShfl) sm.q1[ly(k0) / 2][lx(k0) + 1] = q1r[j];
      if (k1 % KY == KY - 1) sm.q2last[ty0 + 1][lx(k1)] = q2r[j].y;
      if constexpr (X::kOn) xc->send_q(lx(k0), ly(k0) / 2, q1r[j], k1 % KY == KY - 1, lx(k1),
                                       q2r[j].y);
    }
    __syncthreads();
    if constexpr (X::kOn) xc->after_bar1();
    // primal step: v = u + tau div(M^T p), u+ = prox(v), ubar = 2 u+ - u
    const float2 tau2 = dup2(c.tau);
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int k0 = 2 * j;
      float2 q1m;
      if constexpr (kShfl) {  // x - 1 neighbour: the lane to the left (lane 0: its own)
        q1m.x = __shfl_up_sync(0xffffffffu, q1r[j].x, 1);
        q1m.y = __shfl_up_sync(0xffffffffu, q1r[j].y, 1);
      } else {
        q1m = sm.q1[ly(k0) / 2][lx(k0)];
      }
      // y - 1 neighbour: pixel k1's is k0; pixel k0's is the pair above or the strip above
      const float2 q2m = make_float2((k0 % KY == 0) ? sm.q2last[ty0][lx(k0)] : q2r[j - 1].y,
                                     q2r[j].x);
      const float2 div = add2(fma2(one_neg, q1m, q1r[j]), fma2(one_neg, q2m, q2r[j]));
      const float2 v = fma2(tau2, div, u[j]);
      if constexpr (SAVE) vs[j] = v;
      float2 un;
      if constexpr (L2) {
        un = mul2(add2(v, D2[j]), D1[j]);
      } else {
        // KL root (Eq. update_rules): MUFU reciprocal square root and reciprocal (a few
        // ulp); for v < beta the root 2 beta f / (sqrt(.) - (v - beta)) avoids the
        // cancellation of (v - beta + sqrt(.)) / 2.
        const float2 d = add2(v, D1[j]);       // v - beta
        const float2 disc = fma2(d, d, D2[j]);  // + 4 beta f > 0
        const float2 sq = mul2(disc, make_float2(rsqrt_mufu(disc.x), rsqrt_mufu(disc.y)));
        const float2 rp = mul2(dup2(0.5f), add2(d, sq));
        const float2 den = fma2(one_neg, d, sq);
        const float2 rn = mul2(D3[j], make_float2(rcp_mufu(den.x), rcp_mufu(den.y)));
        un.x = fminf(fmaxf(d.x >= 0.0f ? rp.x : rn.x, c.u_min), c.u_max);
        un.y = fminf(fmaxf(d.y >= 0.0f ? rp.y : rn.y, c.u_min), c.u_max);
      }
      float2 ub = fma2(one_neg, u[j], add2(un, un));
      ub.x = S::rnd(ub.x);
      ub.y = S::rnd(ub.y);
      u[j] = un;
      q1r[j] = ub;  // from here on: ubar of pair j
      if constexpr (SAVE) ubs[j] = ub;
      if constexpr (!kShfl) sm.ub[ly(k0) / 2][lx(k0)] = S::enc2(ub);
      if (k0 % KY == 0) sm.ubfirst[ty0][lx(k0)] = S::enc(ub.x);
      if constexpr (X::kOn) xc->send_u(lx(k0), ly(k0) / 2, ub, k0 % KY == 0);
    }
    __syncthreads();
    if constexpr (X::kOn) xc->after_bar2();
    // dual step: p = proj(p + sigma M (D_x ubar, D_y ubar))
    const float2 sig2 = dup2(c.sigma);
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int k0 = 2 * j, k1 = k0 + 1;
      const float2 ub = q1r[j];
      float2 ubx;
      if constexpr (kShfl) {  // x + 1 neighbour: the lane to the right (lane 31: its own)
        ubx.x = __shfl_down_sync(0xffffffffu, ub.x, 1);
        ubx.y = __shfl_down_sync(0xffffffffu, ub.y, 1);
      } else {
        ubx = S::dec2(sm.ub[ly(k0) / 2][lx(k0) + 1]);
      }
      // y + 1 neighbour: pixel k0's is k1; pixel k1's is the next pair or the strip below
      const float2 uby = make_float2(
          ub.y, (k1 % KY == KY - 1) ? S::dec(sm.ubfirst[ty0 + 1][lx(k1)]) : q1r[j + 1].x);
      const float2 dx = fma2(one_neg, ub, ubx);
      const float2 dy = fma2(one_neg, ub, uby);
      // M (m_x dx, m_y dy) (Eq. 3)
      const float2 g1 = fma2(E4[j], dy, mul2(E1[j], dx));
      const float2 g2 = fma2(E5[j], dy, mul2(E2[j], dx));
      const float2 g3 = fma2(E6[j], dy, mul2(E3[j], dx));
      const float2 a1 = fma2(sig2, g1, p1[j]);
      const float2 a2 = fma2(sig2, g2, p2[j]);
      const float2 a3 = fma2(sig2, g3, p3[j]);
      // projection onto |p| <= sqrt(G) (Eq. update_rules, second line):
      // p / max(1, |p| / sqrt(G)) = p min(1, sqrt(G) / |p|); |p| = 0 gives min(1, inf)
      const float2 n2 = fma2(a1, a1, fma2(a2, a2, mul2(a3, a3)));
      const float2 t = mul2(SG[j], make_float2(rsqrt_mufu(n2.x), rsqrt_mufu(n2.y)));
      const float2 sc = make_float2(fminf(t.x, 1.0f), fminf(t.y, 1.0f));
      p1[j] = mul2(a1, sc);
      p2[j] = mul2(a2, sc);
      p3[j] = mul2(a3, sc);
      p1[j].x = S::rnd(p1[j].x);
      p1[j].y = S::rnd(p1[j].y);
      p2[j].x = S::rnd(p2[j].x);
      p2[j].y = S::rnd(p2[j].y);
      p3[j].x = S::rnd(p3[j].x);
      p3[j].y = S::rnd(p3[j].y);
    }
  }

  // Write (u, p) of the owned pixels (all of them, or only the border band).
  __device__ __forceinline__ void store(const Planes& P, int buf, bool band_only) {
    float* U = P.u[buf];
    ST *P1 = (ST*)P.p1[buf], *P2 = (ST*)P.p2[buf], *P3 = (ST*)P.p3[buf];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = k >> 1, h = k & 1;
      if ((band_only ? band(k) : owned(k)) && on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        U[i] = el(u[j], h);
        P1[i] = S::enc(el(p1[j], h));
        P2[i] = S::enc(el(p2[j], h));
        P3[i] = S::enc(el(p3[j], h));
      }
    }
  }

  // Read (u, p) of the halo pixels from the neighbours' bands, through L2.
  __device__ __forceinline__ void reload_halo(const Planes& P, int buf) {
    const float* U = P.u[buf];
    const ST *P1 = (const ST*)P.p1[buf], *P2 = (const ST*)P.p2[buf], *P3 = (const ST*)P.p3[buf];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = k >> 1, h = k & 1;
      if (!owned(k) && on(k, P.W, P.H)) {
        const size_t i = gidx(P, k);
        el(u[j], h) = __ldcg(U + i);
        el(p1[j], h) = S::ldcg(P1, i);
        el(p2[j], h) = S::ldcg(P2, i);
        el(p3[j], h) = S::ldcg(P3, i);
      }
    }
  }
};

}  // namespace evr
