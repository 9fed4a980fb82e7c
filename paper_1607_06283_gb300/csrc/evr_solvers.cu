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
//   kind 5 (k_resident): as kind 2 with the exchange behind one grid-wide barrier (an
//     arrival counter), the packet's front -- and its push -- at the start of the same
//     launch, and the launch captured in the packet's graph: one launch per packet.
#include <cuda_bf16.h>
#include <algorithm>
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
    // kind 5: one resident cooperative launch per packet, grid barrier every R iterations
    {5, 7, 6}, {5, 7, 8}, {5, 7, 9}, {5, 7, 10}, {5, 1, 4}, {5, 1, 6}, {5, 1, 8}, {5, 0, 4},
    {5, 0, 6}, {5, 6, 5},
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
// Tiles whose pass 0 can also take the packet's push (FP32; the event maps in dynamic
// shared memory): the front's tiles
template <int KX, int KY, int NTY>
constexpr bool kTiledPush = kTiledFront<KX, KY, NTY, float>;

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
// memory) that start from the planes' t_last, forms the packet constants from the maps
// and the planes' counts, and writes back the t_last of its owned pixels that events hit
// (a pixel read as halo by another CTA gives that CTA the same value before or after the
// write: t_last only grows by the maximum).  CTA 0 records the packet's clock for pass 1,
// which commits it.
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
  // Every global read the front needs that does not depend on the packet's verdict, in
  // one round: the stream's clock, this thread's first event (and the timestamp before
  // it), the packet's first and last timestamps, the counts of the thread's pixels, and
  // the t_last of the map's pixels (the map starts from them, so the merged surface
  // needs no second read).
  const bool mine = tid < ev.n;
  int x0 = 0, y0 = 0, p0 = 1;
  long long t0 = 0, tp0 = 0;
  if (mine) {
    x0 = ev.x[tid];
    y0 = ev.y[tid];
    t0 = ev.t[tid];
    p0 = ev.pol[tid];
    if (tid > 0) tp0 = ev.t[tid - 1];
  }
  const long long clock0 = P.sc->clock;
  const int have = P.sc->t_init_set;
  const long long t_init0 = P.sc->t_init;
  const long long t_first = ev.n > 0 ? ev.t[0] : 0, t_end = ev.n > 0 ? ev.t[ev.n - 1] : 0;
  int np[TT::K], nn[TT::K];
  T.load_counts(P, np, nn);
  if (tid == 0) s_bad = ev.n;
  for (int m = tid; m < MW * MH; m += NT) {
    const int gx = T.gx0 + m % MW, gy = T.gy0 + m / MW;
    mt[m] = (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H) ? P.t_last[(size_t)gy * P.pitch + gx]
                                                          : kNeverFired;
    mc[m] = 0;
  }
  __syncthreads();
  if (mine && event_code_of(x0, y0, t0, tp0, p0, tid == 0, P.W, P.H, clock0, have) != 0)
    atomicMin(&s_bad, tid);
  for (int i = tid + NT; i < ev.n; i += NT)
    if (event_code(ev.x, ev.y, ev.t, ev.pol, i, P.W, P.H, clock0, have) != 0)
      atomicMin(&s_bad, i);
  __syncthreads();
  const bool valid = s_bad >= ev.n;
  if (valid) {
    auto merge = [&](int xe, int ye, long long te, int pe) {
      const int lx = xe - T.gx0, ly = ye - T.gy0;
      if (lx >= 0 && lx < MW && ly >= 0 && ly < MH) {
        atomicMax(&mt[ly * MW + lx], te);
        atomicAdd(&mc[ly * MW + lx], pe > 0 ? 1 : (1 << 16));
      }
    };
    if (mine) merge(x0, y0, t0, p0);
    for (int i = tid + NT; i < ev.n; i += NT) merge(ev.x[i], ev.y[i], ev.t[i], ev.pol[i]);
  }
  __syncthreads();
  long long clock = clock0, t_init = have ? t_init0 : clock0;
  if (valid && ev.n > 0) {
    clock = max(clock0, t_end);
    t_init = have ? t_init0 : t_first;
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
  T.front_consts_push(P, c, pc, mt, mc, np, nn, clock, t_init);
}

template <int KX, int KY, int NTY, typename ST, int MODE>
__global__ void __launch_bounds__(32 * NTY, (MODE == 2 ? 2 : kTiledMinBlocks<KX, KY, NTY, ST>))
    k_tiled(const __grid_constant__ Planes P, int src, int iters, int R, SolveConsts c,
            int tiles_x, BatchRef B,
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
    if (threadIdx.y == 0) stage_planes(&sP, &B.descs[w.x], threadIdx.x);
  } else if (threadIdx.y == 0) {
    stage_planes(&sP, &P, threadIdx.x);
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

// ---------------------------------------------------------------- kind 5
// Grid-wide barrier of a cooperative launch: the CTA's earlier global writes (issued
// before the call by any of its threads) are visible to every CTA after it.  `arrive`
// counts arrivals from 0 within the launch; the j-th barrier (j = 1, 2, ...) waits for
// j * ctas of them.  The wait is bounded: it gives up when the stream's abort flag is set
// or after kSpinLimit polls (then it sets the flag and EVR_ERR_TIMEOUT).  Returns false
// (in every thread of the CTA) if it gave up.
__device__ __forceinline__ bool grid_barrier(int* arrive, int target, DevScalars* sc, int tid,
                                             int* s_bail) {
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(arrive), "r"(1) : "memory");
    bool ok = true;
    unsigned n = 0;
    while (ld_acquire(arrive) < target) {
      if ((++n & 31) == 0 && (*(volatile int*)&sc->abort || n > kSpinLimit)) {
        ok = false;
        break;
      }
    }
    if (!ok) {
      atomicExch(&sc->abort, 1);
      atomicCAS(&sc->status, 0, kErrTimeout);
    }
    *s_bail = ok ? 0 : 1;
  }
  __syncthreads();
  return *s_bail == 0;
}

// One packet's solve in one cooperative launch of one CTA per tile (all resident).
// FM (the front): 0 -- the packet constants come from the planes (the prologue ran
// before); 1 -- computed here as the prologue computes them; 3 -- as 1 after validating
// and integrating the packet `ev` here (the same code as pass 0 of the push-fused
// passes: every CTA scans the packet into shared-memory maps of its extended tile).
// Then `iters` iterations from buffer `cur`: after every R of them (and after the first R
// only if FM > 0 and they are all) the CTA writes its band into buffer cur ^ (j + 1 & 1),
// passes a grid barrier and reads its halo back; after the first barrier the owned event
// counts are cleared and CTA 0 commits the packet's stream clock (FM 3).  The last pass
// writes every owned pixel into buffer cur ^ (passes & 1).  The barrier words live after
// the persistent solver's flags: an arrival count and a leave count; the last CTA to
// leave resets both, so every launch starts from 0.  One-pair tiles take the
// multi-launch tile's register budget (64: several CTAs per SM where the block size
// allows them); two-pair tiles, whose front needs more, are not capped.
template <int KX, int KY, int NTY>
constexpr int kResidentMinBlocks = KX * KY == 2 ? kTiledMinBlocks<KX, KY, NTY, float> : 1;

template <int KX, int KY, int NTY, int FM>
__global__ void __launch_bounds__(32 * NTY, (kResidentMinBlocks<KX, KY, NTY>))
    k_resident(const __grid_constant__ Planes P, int cur, int iters, int R, SolveConsts c,
               int tiles_x, int tiles_y, PrologueConsts pc, PushArgs ev) {
  using TT = Tile<KX, KY, NTY>;
  __shared__ TileSmem<KX, KY, NTY> sm;
  __shared__ Planes sP;
  __shared__ int s_bail;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int nct = tiles_x * tiles_y;
  if (threadIdx.y == 0) stage_planes(&sP, &P, threadIdx.x);
  if (tid == 0) s_bail = 0;
  __syncthreads();
  TT T;
  T.setup(blockIdx.x, tiles_x, R);
  TT::zero_pads(sm);
  if constexpr (FM == 3) {
    T.load_state(sP, cur);  // the front takes f from the current u
    push_front(T, sP, c, pc, ev);
  } else if constexpr (FM == 1) {
    T.load_state(sP, cur);
    T.front_consts(sP, c, pc);
  } else {
    T.load_consts(sP, c);
    T.load_state(sP, cur);
  }
  int* arrive = sP.flags + kMaxCtas;
  int* leave = arrive + 1;
  const int passes = (iters + R - 1) / R;
  bool settled = FM == 0;  // event counts cleared and clock committed
  int bars = 0;
  for (int j = 0; j < passes; ++j) {
    const int r = min(R, iters - j * R);
    if (c.data_term)
      for (int it = 0; it < r; ++it) T.template iterate<true>(sm, c);
    else
      for (int it = 0; it < r; ++it) T.template iterate<false>(sm, c);
    const int buf = cur ^ ((j + 1) & 1);
    const bool last = j == passes - 1;
    T.store(sP, buf, !last);
    if (last && settled) break;
    if (!grid_barrier(arrive, ++bars * nct, sP.sc, tid, &s_bail)) return;
    if (!settled) {  // every CTA's front has read the counts and the clock
      T.clear_counts(sP);
      if (blockIdx.x == 0 && tid == 0 && sP.sc->commit_pending) {
        sP.sc->clock = sP.sc->clock_next;
        sP.sc->t_init = sP.sc->t_init_next;
        sP.sc->t_init_set = 1;
        sP.sc->commit_pending = 0;
      }
      settled = true;
    }
    if (last) break;
    T.reload_halo(sP, buf);
  }
  if (tid == 0 && atomicAdd(leave, 1) == nct - 1) {  // every CTA has left every barrier
    *arrive = 0;
    *leave = 0;
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
// a tile that takes the front); sets the kernel's dynamic shared-memory limit for its
// event maps.
template <int KX, int KY, int NTY>
static bool push_fusable_t() {
  if constexpr (kTiledPush<KX, KY, NTY>) {
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
    if constexpr (kTiledPush<KX, KY, NTY> && sizeof(ST) == 4) {
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
  if constexpr (kTiledPush<KX, KY, NTY>) {
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

template <int KX, int KY, int NTY, int FM>
static int resident_per_sm() {
  static int per = -1;
  if (per < 0) {
    const size_t dyn = FM == 3 ? tiled_push_smem<KX, KY, NTY>() : 0;
    if (FM == 3 && cudaFuncSetAttribute((const void*)k_resident<KX, KY, NTY, 3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dyn) != cudaSuccess) {
      cudaGetLastError();
      return per = 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_resident<KX, KY, NTY, FM>, 32 * NTY,
                                                      dyn) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    per = n;
  }
  return per;
}

// Whether all tiles of the resident solver are co-resident (in every front form).
template <int KX, int KY, int NTY>
static bool resident_fits(const Planes& P, int R, int* nctas) {
  int tx, ty;
  if (!P.flags || P.storage != 0 || !tiles_of<KX, KY, NTY>(P, R, &tx, &ty)) return false;
  *nctas = tx * ty;
  if (tx * ty > kMaxCtas) return false;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  const int per = std::min(resident_per_sm<KX, KY, NTY, 0>(),
                           std::min(resident_per_sm<KX, KY, NTY, 1>(),
                                    resident_per_sm<KX, KY, NTY, 3>()));
  return tx * ty <= sms * per;
}

template <int KX, int KY, int NTY>
static int run_resident(const Planes& P, int R, int cur, int iters, const SolveConsts& c,
                        cudaStream_t st, const PrologueConsts* front, const PushArgs* push) {
  int tx, ty, n;
  if (!tiles_of<KX, KY, NTY>(P, R, &tx, &ty) || iters < 1) return (int)cudaErrorInvalidValue;
  if (!resident_fits<KX, KY, NTY>(P, R, &n)) return (int)cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(tx * ty);
  lc.blockDim = dim3(32, NTY);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  const PushArgs none{nullptr, nullptr, nullptr, nullptr, 0};
  if (front && push) {
    if (push->n < 0 || push->n > kTiledPushMax) return (int)cudaErrorInvalidValue;
    lc.dynamicSmemBytes = tiled_push_smem<KX, KY, NTY>();
    return (int)cudaLaunchKernelEx(&lc, k_resident<KX, KY, NTY, 3>, P, cur, iters, R, c, tx, ty,
                                   *front, *push);
  }
  if (front)
    return (int)cudaLaunchKernelEx(&lc, k_resident<KX, KY, NTY, 1>, P, cur, iters, R, c, tx, ty,
                                   *front, none);
  return (int)cudaLaunchKernelEx(&lc, k_resident<KX, KY, NTY, 0>, P, cur, iters, R, c, tx, ty,
                                 PrologueConsts{}, none);
}

// The resident launch node of a captured push-fused graph, given the next packet.
template <int KX, int KY, int NTY>
static int set_resident_push_node(cudaGraphExec_t exec, cudaGraphNode_t node, const Planes& P,
                                  int R, int cur, int iters, const SolveConsts& c,
                                  const PrologueConsts& front, const PushArgs& push) {
  int tx, ty;
  if (!tiles_of<KX, KY, NTY>(P, R, &tx, &ty) || iters < 1 || push.n < 0 ||
      push.n > kTiledPushMax)
    return (int)cudaErrorInvalidValue;
  Planes Pc = P;
  SolveConsts cc = c;
  PrologueConsts pc = front;
  PushArgs ev = push;
  int curv = cur, itv = iters, Rv = R, txv = tx, tyv = ty;
  void* args[] = {&Pc, &curv, &itv, &Rv, &cc, &txv, &tyv, &pc, &ev};
  cudaKernelNodeParams kp;
  cudaError_t e = cudaGraphKernelNodeGetParams(node, &kp);
  if (e != cudaSuccess) return (int)e;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return (int)cudaGraphExecKernelNodeSetParams(exec, node, &kp);
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

int launch_resident(const Planes& P, const SolverCfg& cfg, int cur, int iters,
                    const SolveConsts& c, void* stream, const PrologueConsts* front,
                    const PushArgs* push) {
  if (cfg.kind != 5) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  EVR_SHAPE_DISPATCH(run_resident, P, cfg.R, cur, iters, c, st, front, push)
  return (int)cudaErrorInvalidValue;
}

int resident_node_set_push(void* graph_exec, void* node, const Planes& P, const SolverCfg& cfg,
                           int cur, int iters, const SolveConsts& c, const PrologueConsts& front,
                           const PushArgs& push) {
  if (cfg.kind != 5) return (int)cudaErrorInvalidValue;
  cudaGraphExec_t ex = (cudaGraphExec_t)graph_exec;
  cudaGraphNode_t nd = (cudaGraphNode_t)node;
  EVR_SHAPE_DISPATCH(set_resident_push_node, ex, nd, P, cfg.R, cur, iters, c, front, push)
  return (int)cudaErrorInvalidValue;
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
  if (cfg.kind == 5) return resident_fits<KX, KY, NTY>(P, cfg.R, &n);
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
