// evr_staged.cu -- TMA-staged solver passes (kind 4) for sm_103a: the tiled primal-dual
// iterations (Eq. cont_iterates with Eq. update_rules) of the multi-launch solver, with a
// persistent grid whose CTAs walk the sensor's tiles and stage each tile's inputs in
// shared memory with tensor-memory-access (TMA) copies, one tile ahead.
//
// A pass of R iterations reads, per tile, the extended tile (owned pixels plus an
// R-pixel halo) of nine planes: u, p1, p2, p3 of the current buffer and the packet's
// L_x t, L_y t, f, 1/G and sqrt G.  One thread of each
// CTA issues the nine 2-D tensor copies of the next tile into the second of two
// shared-memory stages as soon as every thread has moved the current tile into
// registers; the copies then run while the current tile iterates, and an mbarrier's
// transaction count says when they have landed.  The per-pixel arithmetic is that of
// the multi-launch solver (evr_tile.cuh), so both give the same bits.
//
// A tensor copy must start at a 16-byte boundary: a tile starts at x = gx0, so each copy
// starts at gx0 rounded down to a multiple of 8 elements and is 8 elements wider than
// the tile; the threads index past the offset.  Rows and columns outside the sensor are
// filled with zeros by the copy and replaced by the solver's finite filler.  Only this
// GPU's own memory is read; there is no multicast.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets EVR_ERR_TIMEOUT in the
// stream's status and the CTA stops taking tiles (after waiting, again bounded, for its
// copies still in flight).
#include <cuda_runtime.h>

#include <cstdint>

#include "evr_internal.cuh"
#include "evr_tile.cuh"
#include "evr_tma.cuh"

namespace evr {

namespace {

constexpr int kErrTimeoutSt = -7;              // EVR_ERR_TIMEOUT
constexpr unsigned kStageSpin = 1u << 22;      // polls of an mbarrier before giving up
constexpr int kStagePlanes = 9;  // u, p1, p2, p3, L_x t, L_y t, f, 1/G, sqrt G
constexpr int kStageAlign = 8;                 // elements: 32 bytes, a multiple of 16

struct StageMaps {
  CUtensorMap m[2][4];  // [buffer][u, p1, p2, p3]
  CUtensorMap tx, ty, f, iG, sG;
};

struct StageArgs {
  Planes P;
  SolveConsts c;
  int src, iters, R, tiles_x, n_tiles;
};

using tma::fence_proxy_async;
using tma::mbar_arm;
using tma::mbar_done;
using tma::mbar_init1;
using tma::smem_u32;

template <int KX, int KY, int NTY>
struct StageShape {
  static constexpr int EW = 32 * KX, EH = NTY * KY;
  static constexpr int BW = EW + kStageAlign;  // copied box width (elements)
  static constexpr int PLANE = BW * EH;        // floats per staged plane
  static constexpr int STAGE = kStagePlanes * PLANE;
  static constexpr uint32_t BYTES = STAGE * 4u;
  static constexpr size_t SMEM = 2 * (size_t)BYTES;  // two stages, dynamic shared memory
  static_assert((PLANE * 4) % 128 == 0, "each staged plane starts on a 128-byte line");
};

__device__ __forceinline__ int floor_align(int x) { return x & ~(kStageAlign - 1); }

// The 512-thread tile with one pixel pair per thread is held to 64 registers: two of its
// CTAs (two stages each) fit on an SM.
template <int KX, int KY, int NTY>
constexpr int kStagedMinBlocks = (NTY == 16 && KX * KY == 2) ? 2 : 1;

template <int KX, int KY, int NTY>
__global__ void __launch_bounds__(32 * NTY, (kStagedMinBlocks<KX, KY, NTY>))
    k_staged(const __grid_constant__ StageMaps M, const __grid_constant__ StageArgs a) {
  using SS = StageShape<KX, KY, NTY>;
  using TT = Tile<KX, KY, NTY, float>;
  extern __shared__ __align__(128) float stage[];  // [2][kStagePlanes][EH][BW]
  __shared__ TileSmem<KX, KY, NTY, float> sm;
  __shared__ __align__(8) unsigned long long s_mb[2];
  __shared__ int s_bail;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const Planes& P = a.P;
  const int OW = SS::EW - 2 * a.R, OH = SS::EH - 2 * a.R;
  TT::zero_pads(sm);
  if (tid == 0) {
    s_bail = 0;
    mbar_init1(smem_u32(&s_mb[0]));
    mbar_init1(smem_u32(&s_mb[1]));
    tma::mbar_init_fence();
  }
  __syncthreads();
  // the previous pass wrote (u, p) of buffer src: wait for it before the first copy
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);

  auto issue = [&](int tile, int b) {  // thread 0 only
    const int gx0 = (tile % a.tiles_x) * OW - a.R, gy0 = (tile / a.tiles_x) * OH - a.R;
    const int x0 = floor_align(gx0);
    const uint32_t mb = smem_u32(&s_mb[b]);
    const uint32_t dst = smem_u32(stage + (size_t)b * SS::STAGE);
    mbar_arm(mb, SS::BYTES);
    for (int q = 0; q < 4; ++q)
      tma::load_2d(dst + q * SS::PLANE * 4u, &M.m[a.src][q], x0, gy0, mb);
    tma::load_2d(dst + 4 * SS::PLANE * 4u, &M.tx, x0, gy0, mb);
    tma::load_2d(dst + 5 * SS::PLANE * 4u, &M.ty, x0, gy0, mb);
    tma::load_2d(dst + 6 * SS::PLANE * 4u, &M.f, x0, gy0, mb);
    tma::load_2d(dst + 7 * SS::PLANE * 4u, &M.iG, x0, gy0, mb);
    tma::load_2d(dst + 8 * SS::PLANE * 4u, &M.sG, x0, gy0, mb);
  };
  const int first = blockIdx.x;
  if (tid == 0 && first < a.n_tiles) issue(first, 0);
  const float tl = a.c.tau * a.c.lambda;
  int i = 0;
  uint32_t wait_mb = 0, wait_parity = 0;  // the stage whose copies this CTA waits for
  for (int tile = first; tile < a.n_tiles; tile += gridDim.x, ++i) {
    const int b = i & 1;
    // the stage of this tile: its copies have landed (bounded wait)
    wait_mb = smem_u32(&s_mb[b]);
    wait_parity = (uint32_t)(i >> 1) & 1u;
    for (unsigned n = 0; !mbar_done(wait_mb, wait_parity);) {
      if (++n > kStageSpin) {
        atomicCAS(&P.sc->status, 0, kErrTimeoutSt);
        s_bail = 1;
        break;
      }
    }
    TT T;
    T.setup(tile, a.tiles_x, a.R);
    {
      const float* st = stage + (size_t)b * SS::STAGE;
      const int dx = T.gx0 - floor_align(T.gx0);
#pragma unroll
      for (int k = 0; k < TT::K; ++k) {
        const int j = k >> 1, h = k & 1;
        float av = 0.f, bv = 0.f, ig = 1.f, sg = 1.f, f = 1.f, mx = 0.f, my = 0.f;
        if (T.on(k, P.W, P.H)) {
          const int o = T.ly(k) * SS::BW + T.lx(k) + dx;
          el(T.u[j], h) = st[o];
          el(T.p1[j], h) = st[SS::PLANE + o];
          el(T.p2[j], h) = st[2 * SS::PLANE + o];
          el(T.p3[j], h) = st[3 * SS::PLANE + o];
          av = st[4 * SS::PLANE + o];
          bv = st[5 * SS::PLANE + o];
          f = st[6 * SS::PLANE + o];
          ig = st[7 * SS::PLANE + o];
          sg = st[8 * SS::PLANE + o];
          mx = (T.gx0 + T.lx(k) < P.W - 1) ? 1.0f : 0.0f;
          const int gy = T.gy0 + T.ly(k);
          my = ((P.Hm == P.H ? gy : gy % P.Hm) < P.Hm - 1) ? 1.0f : 0.0f;
        } else {  // off the sensor: finite filler, masked out of every term
          el(T.u[j], h) = 1.0f;
          el(T.p1[j], h) = el(T.p2[j], h) = el(T.p3[j], h) = 0.0f;
        }
        T.set_consts(k, av, bv, ig, sg, f, mx, my, tl, a.c);
      }
    }
    // every thread has its tile in registers: the other stage (read by the previous
    // tile, before the previous pass of this barrier) takes the next tile's copies
    __syncthreads();
    if (s_bail) break;
    if (tid == 0 && tile + (int)gridDim.x < a.n_tiles) {
      fence_proxy_async();
      issue(tile + gridDim.x, b ^ 1);
    }
    if (a.c.data_term)
      for (int it = 0; it < a.iters; ++it) T.template iterate<true>(sm, a.c);
    else
      for (int it = 0; it < a.iters; ++it) T.template iterate<false>(sm, a.c);
    T.store(P, 1 - a.src, false);
  }
  // a CTA that stopped early waits once more (bounded) for the copies of the stage it
  // was waiting for, the only ones it can have in flight
  if (s_bail && tid == 0)
    for (unsigned n = 0; !mbar_done(wait_mb, wait_parity) && n < kStageSpin; ++n) {
    }
}

// ---------------------------------------------------------------- host side
bool encode_plane(CUtensorMap* m, const float* base, const Planes& P, int BW, int EH) {
  const uint64_t dims[2] = {(uint64_t)P.W, (uint64_t)P.H};
  const uint32_t box[2] = {(uint32_t)BW, (uint32_t)EH};
  return tma::encode_f32(m, base, 2, dims, (uint64_t)P.pitch * sizeof(float), 0, box);
}

template <int KX, int KY, int NTY>
bool tiles(const Planes& P, int R, int* tx, int* ty) {
  const int OW = 32 * KX - 2 * R, OH = NTY * KY - 2 * R;
  if (R < 1 || OW < R || OH < R) return false;
  *tx = (P.W + OW - 1) / OW;
  *ty = (P.H + OH - 1) / OH;
  return true;
}

template <int KX, int KY, int NTY>
int resident_ctas() {
  using SS = StageShape<KX, KY, NTY>;
  static int n = -1;
  if (n < 0) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_staged<KX, KY, NTY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS::SMEM) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_staged<KX, KY, NTY>, 32 * NTY,
                                                      SS::SMEM) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    n = sms * per;
  }
  return n;
}

template <int KX, int KY, int NTY>
int launch_t(const Planes& P, int R, int src, int iters, int pass, const SolveConsts& c,
             cudaStream_t st) {
  using SS = StageShape<KX, KY, NTY>;
  int tx, ty;
  if (P.storage != 0 || !tiles<KX, KY, NTY>(P, R, &tx, &ty) || iters < 1 || iters > R)
    return (int)cudaErrorInvalidValue;
  const int slots = resident_ctas<KX, KY, NTY>();
  if (slots < 1) return (int)cudaErrorInvalidConfiguration;
  StageMaps M;
  for (int b = 0; b < 2; ++b) {
    const float* q[4] = {P.u[b], P.p1[b], P.p2[b], P.p3[b]};
    for (int k = 0; k < 4; ++k)
      if (!encode_plane(&M.m[b][k], q[k], P, SS::BW, SS::EH)) return (int)cudaErrorInvalidValue;
  }
  if (!encode_plane(&M.tx, P.tx, P, SS::BW, SS::EH) ||
      !encode_plane(&M.ty, P.ty, P, SS::BW, SS::EH) ||
      !encode_plane(&M.f, P.f, P, SS::BW, SS::EH) ||
      !encode_plane(&M.iG, P.iG, P, SS::BW, SS::EH) ||
      !encode_plane(&M.sG, P.sG, P, SS::BW, SS::EH))
    return (int)cudaErrorInvalidValue;
  StageArgs a{P, c, src, iters, R, tx, tx * ty};
  const int n = tx * ty;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(n < slots ? n : slots);
  lc.blockDim = dim3(32, NTY);
  lc.dynamicSmemBytes = SS::SMEM;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&lc, k_staged<KX, KY, NTY>, M, a);
}

template <int KX, int KY, int NTY>
bool usable_t(const Planes& P, int R) {
  int tx, ty;
  return P.storage == 0 && tiles<KX, KY, NTY>(P, R, &tx, &ty) && tma::encode_fn() != nullptr &&
         resident_ctas<KX, KY, NTY>() > 0;
}

template <int KX, int KY, int NTY>
int ctas_t(const Planes& P, int R) {
  int tx = 0, ty = 0;
  if (!tiles<KX, KY, NTY>(P, R, &tx, &ty)) return 0;
  const int slots = resident_ctas<KX, KY, NTY>();
  return tx * ty < slots ? tx * ty : slots;
}

}  // namespace

#define EVR_STAGED_DISPATCH(FN, ...)          \
  switch (cfg.shape) {                        \
    case 0: return FN<1, 4, 8>(__VA_ARGS__);  \
    case 1: return FN<1, 2, 16>(__VA_ARGS__); \
    case 6: return FN<1, 4, 12>(__VA_ARGS__); \
    default: break;                           \
  }

int launch_staged(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
                  const SolveConsts& c, void* stream) {
  if (cfg.kind != 4) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  EVR_STAGED_DISPATCH(launch_t, P, cfg.R, src, iters, pass, c, st)
  return (int)cudaErrorInvalidValue;
}

bool staged_cfg_usable(const Planes& P, const SolverCfg& cfg) {
  if (cfg.kind != 4) return false;
  EVR_STAGED_DISPATCH(usable_t, P, cfg.R)
  return false;
}

int staged_cfg_ctas(const Planes& P, const SolverCfg& cfg) {
  if (cfg.kind != 4) return 0;
  EVR_STAGED_DISPATCH(ctas_t, P, cfg.R)
  return 0;
}

}  // namespace evr
