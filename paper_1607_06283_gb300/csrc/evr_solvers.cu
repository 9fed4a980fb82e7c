// evr_solvers.cu -- tiled primal-dual solvers (Eq. cont_iterates with Eq.
// update_rules) for sm_103a.
//
// Both solvers give every CTA an owned tile plus an R-pixel halo.  One iteration
// reads each pixel's neighbours within Chebyshev distance 1 (the divergence reads
// q = M^T p at x-1 and y-1, the forward differences read ubar at x+1 and y+1, and
// ubar(x+1, y) itself depends on q(x+1, y-1)), so after j local iterations the
// values are exact on the extended tile shrunk by j pixels, and after R on the
// owned tile.
//   kind 1 (k_tiled): one launch per R iterations; state in HBM/L2 between launches.
//   kind 2 (k_persist): one cooperative launch per packet; the tile stays in
//     registers for all iterations, and every R iterations each CTA publishes the
//     R-wide band along its owned border and reads its halo from the 8 neighbouring
//     CTAs' bands through L2, synchronised by per-CTA progress flags.  Every wait is
//     bounded; a wait that runs out sets an abort flag and EVR_ERR_TIMEOUT and the
//     kernel returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "evr_internal.cuh"
#include "evr_push.cuh"
#include "evr_tile.cuh"

namespace evr {

constexpr int kErrTimeout = -7;  // as in include/evr.h

const TileShape kTileShapes[kNumTileShapes] = {
    {32, 32, 8},   // 0: 256 threads, 4 px each
    {32, 32, 16},  // 1: 512 threads, 2 px each
    {32, 64, 16},  // 2: 512 threads, 4 px each
    {64, 32, 8},   // 3: 256 threads, 8 px each
    {64, 32, 16},  // 4: 512 threads, 4 px each
    {32, 16, 8},   // 5: 256 threads, 2 px each
    {32, 48, 12},  // 6: 384 threads, 4 px each
    {32, 64, 32},  // 7: 1024 threads, 2 px each
};

// {kind, shape, R}
const SolverCfg kSolverCfgs[kNumSolverCfgs] = {
    {1, 0, 2}, {1, 0, 4}, {1, 0, 6}, {1, 1, 2}, {1, 1, 4}, {1, 2, 4}, {1, 2, 6}, {1, 2, 8},
    {1, 3, 3}, {1, 4, 4},
    {2, 0, 1}, {2, 0, 2}, {2, 0, 3}, {2, 0, 4}, {2, 1, 1}, {2, 1, 2}, {2, 1, 3}, {2, 2, 2},
    {2, 2, 4}, {2, 3, 2}, {2, 4, 2}, {2, 5, 1}, {2, 5, 2}, {2, 5, 3},
    // more halo widths for the multi-launch solver: one pass fewer per packet where the
    // grid still fits one wave
    {1, 2, 9}, {1, 2, 10}, {1, 4, 8}, {1, 0, 5}, {1, 0, 7}, {1, 0, 8}, {1, 1, 6}, {1, 1, 8},
    {1, 4, 6}, {1, 3, 5},
    // the 384-thread tile, two resident CTAs per SM
    {1, 6, 3}, {1, 6, 4}, {1, 6, 5}, {1, 6, 6}, {1, 6, 7}, {1, 6, 8}, {1, 6, 9}, {1, 6, 10},
    // the 1024-thread tile (32 warps on one SM)
    {1, 7, 6}, {1, 7, 8}, {1, 7, 9}, {1, 7, 10},
    // kind 3, {3, shape, R, cx, cy}: one cluster over the whole sensor (R = 0) ...
    {3, 1, 0, 4, 4}, {3, 0, 0, 4, 4}, {3, 7, 0, 4, 2}, {3, 1, 0, 4, 2}, {3, 1, 0, 2, 4},
    {3, 5, 0, 4, 4}, {3, 1, 0, 8, 2}, {3, 1, 0, 2, 8},
    // ... or clusters as super-tiles with an R-pixel halo
    {3, 1, 6, 4, 4}, {3, 1, 8, 4, 4}, {3, 1, 4, 4, 2}, {3, 1, 6, 4, 2}, {3, 1, 4, 2, 2},
    {3, 1, 6, 2, 4}, {3, 7, 8, 4, 2}, {3, 6, 6, 4, 2},
    // kind 4: persistent passes with tensor-copy staging of each tile
    {4, 1, 4}, {4, 1, 6}, {4, 1, 8}, {4, 0, 4}, {4, 0, 6}, {4, 6, 4}, {4, 6, 5}, {4, 6, 6},
};

// ---------------------------------------------------------------- kind 1
// Launched with programmatic stream serialisation: a pass may start while the
// previous one drains.  Pass j > 0 of a packet first loads the packet constants
// (written by the prologue, which completed before pass j - 1 got past its own wait),
// then waits for the previous pass to complete before reading (u, p), and only then
// lets the next pass launch -- so no pass can run ahead of the prologue.  Pass 0
// loads everything after its wait.
// Resident CTAs per SM the register budget is sized for: tiles with two pixel pairs per
// thread get as many CTAs as fit at 80 registers (three of 256 threads, two of 384; no
// spills in FP32 and BF16, 4 bytes in FP16), tiles with one pair as many as fit at 64
// (four of 256 threads, two of 512, one of 1024; no spills), so that more warps hide
// latency and the next pass's CTAs can become resident while the current pass runs.
template <int KX, int KY, int NTY, typename ST>
constexpr int kTiledMinBlocks =
    (KX * KY == 4 && 65536 / (32 * NTY * 80) > 1)   ? 65536 / (32 * NTY * 80)
    : (KX * KY == 2 && 65536 / (32 * NTY * 64) > 1) ? 65536 / (32 * NTY * 64)
                                                    : 1;
// Tiles whose passes can take the packet's front (its computation needs the registers of
// an uncapped two-pair tile; one-pair tiles fit it in 64)
template <int KX, int KY, int NTY, typename ST>
constexpr bool kTiledFront = kTiledMinBlocks<KX, KY, NTY, ST> == 1 || KX * KY == 2;

// MODE 0: plain passes.  MODE 1 (FRONT): the packet's front launch is fused into the
// passes (instantiated for the tiles of kTiledFront).
// MODE 2 (tape, FP32 only): iteration it of this launch also writes the p it starts
// from, its v and its ubar into tape slot tape_first + it (5 planes, slot stride
// 5 tape_plane floats), for the reverse pass of the unrolled solve.
// The tape mode's tile is held to two resident CTAs per SM (64 registers), as the plain
// passes of the same tile reach without a cap.
// MODE 3 (FRONT and push, FP32 only): as MODE 1, and pass 0 integrates the packet
// itself.  Every CTA validates the whole packet (the same verdict everywhere; the
// stream's clock is read, never written, in pass 0), merges the events that fall into
// its extended tile plus one column and row into shared-memory maps (dynamic shared
// memory), forms the packet constants from the planes and the maps, and writes back its
// owned pixels' t_last (a pixel read as halo by another CTA gives that CTA the same
// value before or after the write: t_last only grows by the maximum).  CTA 0 records the
// packet's clock for pass 1, which commits it.
template <int KX, int KY, int NTY>
constexpr size_t tiled_push_smem() {
  return (size_t)(32 * KX + 1) * (NTY * KY + 1) * (sizeof(long long) + sizeof(int));
}

template <class TT>
__device__ __forceinline__ void push_front(TT& T, const Planes& P, const SolveConsts& c,
                                           const PrologueConsts& pc, const PushArgs& ev) {
  constexpr int MW = TT::EW + 1, MH = TT::EH + 1;
  const int NT = (int)(blockDim.x * blockDim.y);
  extern __shared__ __align__(16) unsigned char push_smem[];
  long long* mt = reinterpret_cast<long long*>(push_smem);
  int* mc = reinterpret_cast<int*>(mt + MW * MH);
  __shared__ int s_bad;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const long long clock0 = P.sc->clock;
  const int have = P.sc->t_init_set;
  const long long t_init0 = P.sc->t_init;
  if (tid == 0) s_bad = ev.n;
  for (int m = tid; m < MW * MH; m += NT) {
    mt[m] = kNeverFired;
    mc[m] = 0;
  }
  __syncthreads();
  for (int i = tid; i < ev.n; i += NT)
    if (event_code(ev.x, ev.y, ev.t, ev.pol, i, P.W, P.H, clock0, have) != 0)
      atomicMin(&s_bad, i);
  __syncthreads();
  const bool valid = s_bad >= ev.n;
  if (valid) {
    for (int i = tid; i < ev.n; i += NT) {
      const int lx = (int)ev.x[i] - T.gx0, ly = (int)ev.y[i] - T.gy0;
      if (lx >= 0 && lx < MW && ly >= 0 && ly < MH) {
        atomicMax(&mt[ly * MW + lx], ev.t[i]);
        atomicAdd(&mc[ly * MW + lx], ev.pol[i] > 0 ? 1 : (1 << 16));
      }
    }
  }
  __syncthreads();
  long long clock = clock0, t_init = have ? t_init0 : clock0;
  if (valid && ev.n > 0) {
    clock = max(clock0, ev.t[ev.n - 1]);
    t_init = have ? t_init0 : ev.t[0];
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (!valid) {
      atomicCAS(&P.sc->status, 0,
                event_code(ev.x, ev.y, ev.t, ev.pol, s_bad, P.W, P.H, clock0, have));
    } else if (ev.n > 0) {
      P.sc->clock_next = clock;
      P.sc->t_init_next = t_init;
      P.sc->commit_pending = 1;
    }
  }
  T.front_consts_push(P, c, pc, mt, mc, clock, t_init);
}

template <int KX, int KY, int NTY, typename ST, int MODE>
__global__ void __launch_bounds__(32 * NTY, (MODE == 2 ? 2 : kTiledMinBlocks<KX, KY, NTY, ST>))
    k_tiled(Planes P, int src, int iters, int R, SolveConsts c, int tiles_x, BatchRef B,
            int pass, PrologueConsts pc, float* tape, long long tape_plane, int tape_first,
            PushArgs ev) {
  constexpr bool FRONT = MODE == 1 || MODE == 3;
  __shared__ TileSmem<KX, KY, NTY, ST> sm;
  __shared__ Planes sP;  // this CTA's stream, staged once (no per-thread local copy)
  int tile = blockIdx.x;
  if (B.descs) {  // batch: this CTA's (stream, tile); one code path for both uses
    const int2 w = B.work[blockIdx.x];
    if (!B.active[w.x]) return;
    src = B.curs[w.x] ^ (pass & 1);
    tile = w.y;
    if (threadIdx.x == 0 && threadIdx.y == 0) sP = B.descs[w.x];
  } else if (threadIdx.x == 0 && threadIdx.y == 0) {
    sP = P;
  }
  __syncthreads();
  if (B.descs) tiles_x = (sP.W + (32 * KX - 2 * R) - 1) / (32 * KX - 2 * R);
  Tile<KX, KY, NTY, ST> T;
  T.setup(tile, tiles_x, R);
  Tile<KX, KY, NTY, ST>::zero_pads(sm);
  // The first pass of a packet follows the prologue, whose writes are only guaranteed
  // visible after the wait; later passes may read the constants before it.  With the
  // front fused (FRONT, single streams only) pass 0 computes the constants itself
  // after its wait (the push has then completed) and writes the owned ones; pass 1 reads
  // them after its own wait and clears the owned event counts.
  const bool early = pass > (FRONT ? 1 : 0);
  if (early) T.load_consts(sP, c);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
  if constexpr (MODE == 3) {
    T.load_state(sP, src);  // the front takes f from the current u
    if (pass == 0) {
      push_front(T, sP, c, pc, ev);
    } else if (!early) {
      T.load_consts(sP, c);
      T.clear_counts(sP);
      if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0 && sP.sc->commit_pending) {
        sP.sc->clock = sP.sc->clock_next;  // the packet integrated by pass 0
        sP.sc->t_init = sP.sc->t_init_next;
        sP.sc->t_init_set = 1;
        sP.sc->commit_pending = 0;
      }
    }
  } else if constexpr (FRONT) {
    T.load_state(sP, src);  // front_consts takes f from the current u
    if (pass == 0) {
      T.front_consts(sP, c, pc);
    } else if (!early) {
      T.load_consts(sP, c);
      T.clear_counts(sP);
    }
  } else {
    if (!early) T.load_consts(sP, c);
    T.load_state(sP, src);
  }
  if constexpr (MODE == 2) {
    // the owned pixels' tape indices, computed once (a tape plane holds < 2^31 floats)
    unsigned ti[Tile<KX, KY, NTY, ST>::K];
#pragma unroll
    for (int k = 0; k < Tile<KX, KY, NTY, ST>::K; ++k)
      ti[k] = (T.owned(k) && T.on(k, sP.W, sP.H)) ? (unsigned)T.gidx(sP, k) : ~0u;
    const unsigned pl = (unsigned)tape_plane;
    for (int it = 0; it < iters; ++it) {
      float* slot = tape + (long long)(tape_first + it) * 5 * tape_plane;
      T.store_tape_p(slot, pl, ti);
      if (c.data_term)
        T.template iterate<true, true>(sm, c);
      else
        T.template iterate<false, true>(sm, c);
      T.store_tape_vub(slot, pl, ti);
    }
  } else {
    if (c.data_term)
      for (int it = 0; it < iters; ++it) T.template iterate<true>(sm, c);
    else
      for (int it = 0; it < iters; ++it) T.template iterate<false>(sm, c);
  }
  T.store(sP, 1 - src, false);
}

// ---------------------------------------------------------------- kind 2
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr unsigned kSpinLimit = 1u << 18;  // polls (two L2 round trips each, no sleep: a
                                           // sleeping poll wakes late and delays every
                                           // exchange): a wait gives up well under a second

template <int KX, int KY, int NTY>
__global__ void __launch_bounds__(32 * NTY) k_persist(Planes P, int cur, int iters, int R,
                                                      SolveConsts c, int tiles_x, int tiles_y,
                                                      int base, int silent_cta) {
  __shared__ TileSmem<KX, KY, NTY> sm;
  __shared__ int s_bail;
  Tile<KX, KY, NTY> T;
  const int cta = blockIdx.x;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  T.setup(cta, tiles_x, R);
  Tile<KX, KY, NTY>::zero_pads(sm);
  T.load(P, cur, c);
  // progress flags count exchanges since the host last cleared them; `base` is the
  // count every CTA reached at the end of the previous launch
  const int passes = (iters + R - 1) / R;
  const int bx = cta % tiles_x, by = cta / tiles_x;
  for (int j = 0; j < passes; ++j) {
    const int r = min(R, iters - j * R);
    if (c.data_term)
      for (int it = 0; it < r; ++it) T.template iterate<true>(sm, c);
    else
      for (int it = 0; it < r; ++it) T.template iterate<false>(sm, c);
    const int buf = cur ^ ((j + 1) & 1);
    if (j == passes - 1) {
      T.store(P, buf, false);
      break;
    }
    T.store(P, buf, true);
    __syncthreads();
    if (tid == 0 && cta != silent_cta) {  // silent_cta >= 0 only in the wait self-test
      __threadfence();
      st_release(&P.flags[cta], base + j + 1);
    }
    if (tid < 32) {  // lanes 0..7 wait for one neighbour each
      bool ok = true;
      if (tid < 8) {
        const int d = tid < 4 ? tid : tid + 1;  // 3x3 neighbourhood without the centre
        const int nx = bx + d % 3 - 1, ny = by + d / 3 - 1;
        if (nx >= 0 && nx < tiles_x && ny >= 0 && ny < tiles_y) {
          const int* f = &P.flags[ny * tiles_x + nx];
          const volatile int* ab = &P.sc->abort;
          unsigned n = 0;
          while (ld_acquire(f) < base + j + 1) {
            if (*ab || ++n > kSpinLimit) {
              ok = false;
              break;
            }
          }
        }
      }
      ok = __all_sync(0xffffffffu, ok);
      if (tid == 0) {
        s_bail = ok ? 0 : 1;
        if (!ok) {
          atomicExch(&P.sc->abort, 1);
          atomicCAS(&P.sc->status, 0, kErrTimeout);
        }
      }
    }
    __syncthreads();
    if (s_bail) return;
    T.reload_halo(P, buf);
  }
}

// ---------------------------------------------------------------- launchers
template <int KX, int KY, int NTY>
static int tiles_of(const Planes& P, int R, int* tx, int* ty) {
  const int OW = 32 * KX - 2 * R, OH = NTY * KY - 2 * R;
  if (R < 1 || OW < R || OH < R) return 0;
  *tx = (P.W + OW - 1) / OW;
  *ty = (P.H + OH - 1) / OH;
  return 1;
}

// Whether the push can be fused into pass 0 for this tile (MODE 3 instantiated: FP32,
// no register cap); sets the kernel's dynamic shared-memory limit for its event maps.
template <int KX, int KY, int NTY>
static bool push_fusable_t() {
  if constexpr (kTiledMinBlocks<KX, KY, NTY, float> == 1) {
    static int ok = -1;
    if (ok < 0) {
      ok = cudaFuncSetAttribute((const void*)k_tiled<KX, KY, NTY, float, 3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tiled_push_smem<KX, KY, NTY>()) == cudaSuccess;
      if (!ok) cudaGetLastError();
    }
    return ok == 1;
  } else {
    return false;
  }
}

template <int KX, int KY, int NTY, typename ST>
static cudaError_t launch_k_tiled_st(cudaLaunchConfig_t* lc, const Planes& P, int src,
                                     int iters, int R, const SolveConsts& c, int tx,
                                     const BatchRef& B, int pass, const PrologueConsts* front,
                                     const PushArgs* push) {
  const PushArgs none{nullptr, nullptr, nullptr, nullptr, 0};
  if (front && push) {
    if constexpr (kTiledMinBlocks<KX, KY, NTY, ST> == 1 && sizeof(ST) == 4) {
      if (push->n < 0 || push->n > kTiledPushMax) return cudaErrorInvalidValue;
      lc->dynamicSmemBytes = tiled_push_smem<KX, KY, NTY>();
      return cudaLaunchKernelEx(lc, k_tiled<KX, KY, NTY, ST, 3>, P, src, iters, R, c, tx, B,
                                pass, *front, (float*)nullptr, 0LL, 0,
                                pass == 0 ? *push : none);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (front) {
    if constexpr (kTiledFront<KX, KY, NTY, ST>)
      return cudaLaunchKernelEx(lc, k_tiled<KX, KY, NTY, ST, 1>, P, src, iters, R, c, tx, B,
                                pass, *front, (float*)nullptr, 0LL, 0, none);
    else
      return cudaErrorInvalidValue;
  }
  return cudaLaunchKernelEx(lc, k_tiled<KX, KY, NTY, ST, 0>, P, src, iters, R, c, tx, B, pass,
                            PrologueConsts{}, (float*)nullptr, 0LL, 0, none);
}

template <int KX, int KY, int NTY>
static void tiled_config(cudaLaunchConfig_t* lc, cudaLaunchAttribute* at, int blocks,
                         cudaStream_t st) {
  *lc = cudaLaunchConfig_t{};
  lc->gridDim = dim3(blocks);
  lc->blockDim = dim3(32, NTY);
  lc->stream = st;
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc->attrs = at;
  lc->numAttrs = 1;
}

template <int KX, int KY, int NTY>
static int launch_k_tiled(int blocks, const Planes& P, int src, int iters, int R,
                          const SolveConsts& c, int tx, const BatchRef& B, int pass,
                          int storage, cudaStream_t st, const PrologueConsts* front,
                          const PushArgs* push = nullptr) {
  cudaLaunchConfig_t lc;
  cudaLaunchAttribute at[1];
  tiled_config<KX, KY, NTY>(&lc, at, blocks, st);
  switch (storage) {
    case 0:
      return (int)launch_k_tiled_st<KX, KY, NTY, float>(&lc, P, src, iters, R, c, tx, B, pass,
                                                        front, push);
    case 1:
      return (int)launch_k_tiled_st<KX, KY, NTY, __half>(&lc, P, src, iters, R, c, tx, B, pass,
                                                         front, push);
    case 2:
      return (int)launch_k_tiled_st<KX, KY, NTY, __nv_bfloat16>(&lc, P, src, iters, R, c, tx, B,
                                                                pass, front, push);
    default:
      return (int)cudaErrorInvalidValue;
  }
}

template <int KX, int KY, int NTY>
static bool front_fusable(int storage) {
  switch (storage) {
    case 0: return kTiledFront<KX, KY, NTY, float>;
    case 1: return kTiledFront<KX, KY, NTY, __half>;
    case 2: return kTiledFront<KX, KY, NTY, __nv_bfloat16>;
    default: return false;
  }
}

template <int KX, int KY, int NTY>
static int run_tiled(const Planes& P, int R, int src, int iters, int pass,
                     const SolveConsts& c, cudaStream_t st, const PrologueConsts* front,
                     const PushArgs* push) {
  int tx, ty;
  if (!tiles_of<KX, KY, NTY>(P, R, &tx, &ty) || iters > R || iters < 1)
    return (int)cudaErrorInvalidValue;
  return launch_k_tiled<KX, KY, NTY>(tx * ty, P, src, iters, R, c, tx,
                                     BatchRef{nullptr, nullptr, nullptr, nullptr}, pass,
                                     P.storage, st, front, push);
}

// The pass-0 node of a captured push-fused graph of a packet solve of `iters` iterations,
// given the next packet: the arguments launch_tiled_pass gave pass 0 (min(iters, R)
// iterations from buffer src), with this push.
template <int KX, int KY, int NTY>
static int set_push_node(cudaGraphExec_t exec, cudaGraphNode_t node, const Planes& P, int R,
                         int src, int iters, const SolveConsts& c, const PrologueConsts& front,
                         const PushArgs& push) {
  int tx, ty;
  if constexpr (kTiledMinBlocks<KX, KY, NTY, float> == 1) {
    if (!tiles_of<KX, KY, NTY>(P, R, &tx, &ty) || iters < 1 || push.n < 0 ||
        push.n > kTiledPushMax)
      return (int)cudaErrorInvalidValue;
    Planes Pc = P;
    SolveConsts cc = c;
    BatchRef B{nullptr, nullptr, nullptr, nullptr};
    PrologueConsts pc = front;
    PushArgs ev = push;
    int srcv = src, itv = iters < R ? iters : R, Rv = R, txv = tx, pass = 0;
    float* tape = nullptr;
    long long tp = 0;
    int tf = 0;
    void* args[] = {&Pc, &srcv, &itv, &Rv, &cc, &txv, &B, &pass, &pc, &tape, &tp, &tf, &ev};
    cudaKernelNodeParams kp;
    cudaError_t e = cudaGraphKernelNodeGetParams(node, &kp);
    if (e != cudaSuccess) return (int)e;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return (int)cudaGraphExecKernelNodeSetParams(exec, node, &kp);
  } else {
    return (int)cudaErrorInvalidValue;
  }
}

template <int KX, int KY, int NTY>
static int run_tiled_batch(const BatchRef& B, int n_work, int R, int pass, int iters,
                           const SolveConsts& c, int storage, cudaStream_t st) {
  const int OW = 32 * KX - 2 * R, OH = NTY * KY - 2 * R;
  if (R < 1 || OW < R || OH < R || iters > R || iters < 1) return (int)cudaErrorInvalidValue;
  if (n_work <= 0) return 0;
  Planes dummy{};
  return launch_k_tiled<KX, KY, NTY>(n_work, dummy, 0, iters, R, c, 0, B, pass, storage, st,
                                     nullptr);
}

template <int KX, int KY, int NTY>
static bool persist_fits(const Planes& P, int R, int* nctas) {
  int tx, ty;
  if (!tiles_of<KX, KY, NTY>(P, R, &tx, &ty)) return false;
  *nctas = tx * ty;
  if (tx * ty > kMaxCtas) return false;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<KX, KY, NTY>, 32 * NTY,
                                                    0) != cudaSuccess)
    return false;
  return tx * ty <= sms * per_sm;
}

template <int KX, int KY, int NTY>
static int run_persist(const Planes& P, int R, int cur, int iters, int base, int silent_cta,
                       const SolveConsts& c, cudaStream_t st) {
  int tx, ty, n;
  if (!tiles_of<KX, KY, NTY>(P, R, &tx, &ty) || iters < 1) return (int)cudaErrorInvalidValue;
  if (!persist_fits<KX, KY, NTY>(P, R, &n)) return (int)cudaErrorCooperativeLaunchTooLarge;
  Planes Pc = P;
  SolveConsts cc = c;
  void* args[] = {&Pc, &cur, &iters, &R, &cc, &tx, &ty, &base, &silent_cta};
  return (int)cudaLaunchCooperativeKernel((const void*)k_persist<KX, KY, NTY>, dim3(tx * ty),
                                          dim3(32, NTY), args, 0, st);
}

#define EVR_SHAPE_DISPATCH(FN, ...)                                  \
  switch (cfg.shape) {                                               \
    case 0: return FN<1, 4, 8>(__VA_ARGS__);                         \
    case 1: return FN<1, 2, 16>(__VA_ARGS__);                        \
    case 2: return FN<1, 4, 16>(__VA_ARGS__);                        \
    case 3: return FN<2, 4, 8>(__VA_ARGS__);                         \
    case 4: return FN<2, 2, 16>(__VA_ARGS__);                        \
    case 5: return FN<1, 2, 8>(__VA_ARGS__);                         \
    case 6: return FN<1, 4, 12>(__VA_ARGS__);                        \
    case 7: return FN<1, 2, 32>(__VA_ARGS__);                        \
    default: break;                                                  \
  }

int launch_tiled_pass(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
                      const SolveConsts& c, void* stream, const PrologueConsts* front,
                      const PushArgs* push) {
  cudaStream_t st = (cudaStream_t)stream;
  EVR_SHAPE_DISPATCH(run_tiled, P, cfg.R, src, iters, pass, c, st, front, push)
  return (int)cudaErrorInvalidValue;
}

bool tiled_push_fusable(const SolverCfg& cfg, int storage) {
  if (cfg.kind != 1 || storage != 0) return false;
  EVR_SHAPE_DISPATCH(push_fusable_t)
  return false;
}

int tiled_node_set_push(void* graph_exec, void* node, const Planes& P, const SolverCfg& cfg,
                        int src, int iters, const SolveConsts& c, const PrologueConsts& front,
                        const PushArgs& push) {
  if (cfg.kind != 1) return (int)cudaErrorInvalidValue;
  cudaGraphExec_t ex = (cudaGraphExec_t)graph_exec;
  cudaGraphNode_t nd = (cudaGraphNode_t)node;
  EVR_SHAPE_DISPATCH(set_push_node, ex, nd, P, cfg.R, src, iters, c, front, push)
  return (int)cudaErrorInvalidValue;
}

int launch_tiled_pass_batch(const BatchRef& B, int n_work, const SolverCfg& cfg, int pass,
                            int iters, const SolveConsts& c, int storage, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (cfg.kind != 1) return (int)cudaErrorInvalidValue;
  EVR_SHAPE_DISPATCH(run_tiled_batch, B, n_work, cfg.R, pass, iters, c, storage, st)
  return (int)cudaErrorInvalidValue;
}

int launch_tiled_tape(const Planes& P, int R, int src, int iters, int pass,
                      const SolveConsts& c, float* tape, long long tape_plane, int tape_first,
                      void* stream) {
  int tx, ty;
  if (!tiles_of<kTapeKX, kTapeKY, kTapeNTY>(P, R, &tx, &ty) || iters > R || iters < 1)
    return (int)cudaErrorInvalidValue;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(tx * ty);
  lc.blockDim = dim3(32, kTapeNTY);
  lc.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  if (tape)
    return (int)cudaLaunchKernelEx(&lc, k_tiled<kTapeKX, kTapeKY, kTapeNTY, float, 2>, P, src,
                                   iters, R, c, tx, BatchRef{nullptr, nullptr, nullptr, nullptr},
                                   pass, PrologueConsts{}, tape, tape_plane, tape_first,
                                   PushArgs{nullptr, nullptr, nullptr, nullptr, 0});
  return (int)cudaLaunchKernelEx(&lc, k_tiled<kTapeKX, kTapeKY, kTapeNTY, float, 0>, P, src,
                                 iters, R, c, tx, BatchRef{nullptr, nullptr, nullptr, nullptr},
                                 pass, PrologueConsts{}, (float*)nullptr, 0LL, 0,
                                 PushArgs{nullptr, nullptr, nullptr, nullptr, 0});
}

int tiled_front_fusable(const SolverCfg& cfg, int storage) {
  if (cfg.kind != 1) return 0;
  switch (cfg.shape) {
    case 0: return front_fusable<1, 4, 8>(storage);
    case 1: return front_fusable<1, 2, 16>(storage);
    case 2: return front_fusable<1, 4, 16>(storage);
    case 3: return front_fusable<2, 4, 8>(storage);
    case 4: return front_fusable<2, 2, 16>(storage);
    case 5: return front_fusable<1, 2, 8>(storage);
    case 6: return front_fusable<1, 4, 12>(storage);
    case 7: return front_fusable<1, 2, 32>(storage);
    default: return 0;
  }
}

int launch_persistent(const Planes& P, const SolverCfg& cfg, int cur, int iters, int base,
                      const SolveConsts& c, void* stream, int silent_cta) {
  cudaStream_t st = (cudaStream_t)stream;
  EVR_SHAPE_DISPATCH(run_persist, P, cfg.R, cur, iters, base, silent_cta, c, st)
  return (int)cudaErrorInvalidValue;
}

template <int KX, int KY, int NTY>
static bool usable(const Planes& P, const SolverCfg& cfg) {
  int tx, ty, n;
  if (cfg.kind == 1) return tiles_of<KX, KY, NTY>(P, cfg.R, &tx, &ty) != 0;
  if (cfg.kind == 2) return persist_fits<KX, KY, NTY>(P, cfg.R, &n);
  return false;
}

template <int KX, int KY, int NTY>
static int ctas(const Planes& P, const SolverCfg& cfg) {
  int tx = 0, ty = 0;
  tiles_of<KX, KY, NTY>(P, cfg.R, &tx, &ty);
  return tx * ty;
}

bool solver_cfg_usable(const Planes& P, const SolverCfg& cfg) {
  if (cfg.kind == 3) return cluster_cfg_usable(P, cfg);
  if (cfg.kind == 4) return staged_cfg_usable(P, cfg);
  EVR_SHAPE_DISPATCH(usable, P, cfg)
  return false;
}

int solver_cfg_ctas(const Planes& P, const SolverCfg& cfg) {
  if (cfg.kind == 3) return cluster_cfg_ctas(P, cfg);
  if (cfg.kind == 4) return staged_cfg_ctas(P, cfg);
  EVR_SHAPE_DISPATCH(ctas, P, cfg)
  return 0;
}

}  // namespace evr
