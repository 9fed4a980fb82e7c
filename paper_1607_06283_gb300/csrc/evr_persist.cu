// evr_persist.cu -- a batch step as one persistent launch (the batching form of the
// primal-dual solve: Eq. cont_iterates with Eq. update_rules over many independent
// event streams).
//
// The host lists the step's work items in order: per window of streams (streams in
// index order whose pass working set fits a budget, so that it stays in L2 across the
// passes) each stream's push (validation and scatter of its packet, Sec. 3 and Sec.
// 3.1), the bands of its packet prologue (time surface, metric of Eq. 2 / Eq. 3, data
// image of Eq. intensity_update), then pass after pass the tiles of every stream of the
// window (R iterations of the tiled solver's Tile, evr_tile.cuh).  The grid holds as many
// CTAs as are resident at once; each CTA takes the next item from a queue counter,
// waits until its stream has completed the items the item depends on (the push for the
// prologue, the prologue and every earlier pass for a pass: a per-stream count), runs
// it and adds one to its stream's count.  Items are taken in list order and depend only
// on earlier items, so the earliest unfinished item can always run: the queue cannot
// deadlock.  Streams are independent, so while one stream's pass drains the other
// streams' tiles keep the SMs busy.
//
// Each pass tile runs exactly the arithmetic of the multi-launch tiled pass (the same
// Tile instantiation, the same packet constants) and the prologue exactly that of the
// prologue kernel (the shared per-pixel functions of evr_internal.cuh), so every
// stream's result is bit-identical to the graph of launches and to a single stream with
// the same tile.  Data another CTA wrote during the launch is read from L2 (ld.global.cg):
// an SM's L1 is not kept coherent with other SMs' writes.
//
// Every wait is bounded (a count of polls and 0.2 s of the global timer); a wait that
// runs out sets the step's abort flag and status and the stream's status to
// EVR_ERR_TIMEOUT, every CTA then leaves at its next item or poll, and the last CTA to
// leave resets the control words, so the next launch starts clean.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "evr_internal.cuh"
#include "evr_persist.cuh"
#include "evr_push.cuh"
#include "evr_tile.cuh"

namespace evr {

namespace {

constexpr int kErrTimeoutCode = -7;     // EVR_ERR_TIMEOUT in include/evr.h
constexpr int kErrInvalidArgCode = -1;  // EVR_ERR_INVALID_ARG
constexpr int kMaxPacket = 32768;       // per-stream packet limit of a batch step
constexpr unsigned kPolls = 1u << 22;
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;

__device__ __forceinline__ int acquire_load(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int relaxed_load(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Release of the item's writes: the CTA's barrier orders every thread's writes before
// this thread's release add (the arrive of a GPU-scope barrier).
__device__ __forceinline__ void release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// 16-byte copy global -> shared that completes asynchronously (L2 only)
__device__ __forceinline__ void copy16_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void copy_async_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0: wait until *cnt >= need.  1: go; 0: another CTA aborted the step; -1: this
// wait ran out (the abort flag is then set).
__device__ int wait_count(const int* cnt, int need, int* ctrl) {
  if (acquire_load(cnt) >= need) return 1;
  const unsigned long long t0 = global_ns();
  for (unsigned k = 1; k < kPolls; ++k) {
    __nanosleep(32);
    if (acquire_load(cnt) >= need) return 1;
    if ((k & 15) == 0) {
      if (relaxed_load(ctrl + kCtrlAbort)) return 0;
      if (global_ns() - t0 > kWaitNs) break;
    }
  }
  atomicExch(ctrl + kCtrlAbort, 1);
  atomicCAS(ctrl + kCtrlStatus, 0, kErrTimeoutCode);
  return -1;
}

// One band of kPersistProRows rows of a stream's packet prologue: per pixel the time
// surface's forward differences, the metric, 1/G, sqrt G, the data image and the
// cleared counts, with the per-pixel functions the prologue kernel uses.  A thread takes
// kBandBatch pixels at a time and issues all their loads before any arithmetic, so that
// they are in flight together (the band's planes come from HBM after the last step).
constexpr int kBandBatch = 3;
__device__ __forceinline__ void prologue_band(const Planes& P, int cur, const PrologueConsts& c,
                                              int band, int tid, int nthr) {
  const long long clock = __ldcg(&P.sc->clock);
  const long long t_init = __ldcg(&P.sc->t_init_set) ? __ldcg(&P.sc->t_init) : clock;
  const int y0 = band * kPersistProRows;
  const int rows = min(kPersistProRows, P.H - y0);
  const int n = rows * P.W;
  const float* base_plane = (c.data_mode == 0) ? P.u[cur] : P.f;
  for (int q0 = tid; q0 < n; q0 += kBandBatch * nthr) {
    long long t0[kBandBatch], t1[kBandBatch], t2[kBandBatch];
    float base[kBandBatch];
    int np[kBandBatch], nn[kBandBatch], xs[kBandBatch], ys[kBandBatch];
#pragma unroll
    for (int k = 0; k < kBandBatch; ++k) {
      const int q = q0 + k * nthr;
      xs[k] = -1;
      ys[k] = 0;
      t0[k] = t1[k] = t2[k] = 0;
      base[k] = 0.0f;
      np[k] = nn[k] = 0;
      if (q < n) {
        const int y = y0 + q / P.W, x = q % P.W;
        const size_t i = (size_t)y * P.pitch + x;
        xs[k] = x;
        ys[k] = y;
        t0[k] = __ldcg(P.t_last + i);
        if (x < P.W - 1) t1[k] = __ldcg(P.t_last + i + 1);
        if (y < P.H - 1) t2[k] = __ldcg(P.t_last + i + P.pitch);
        base[k] = __ldcg(base_plane + i);
        np[k] = __ldcg(P.npos + i);
        nn[k] = __ldcg(P.nneg + i);
      }
    }
#pragma unroll
    for (int k = 0; k < kBandBatch; ++k) {
      if (xs[k] < 0) continue;
      const int x = xs[k], y = ys[k];
      const size_t i = (size_t)y * P.pitch + x;
      const float s0 = time_surface(t0[k], clock, t_init, c);
      const float a =
          (x < P.W - 1) ? surface_diff(time_surface(t1[k], clock, t_init, c), s0) : 0.0f;
      const float b =
          (y < P.H - 1) ? surface_diff(time_surface(t2[k], clock, t_init, c), s0) : 0.0f;
      const float G = metric_G(a, b);
      P.tx[i] = a;
      P.ty[i] = b;
      P.iG[i] = 1.0f / G;
      P.sG[i] = sqrtf(G);
      P.f[i] = data_image(base[k], np[k], nn[k], c);
      P.npos[i] = 0;
      P.nneg[i] = 0;
    }
  }
}

// A pass tile's packet constants and (u, p) from buffer buf, as Tile::load does, read
// from L2.
template <class TT, typename ST>
__device__ __forceinline__ void load_tile_l2(TT& T, const Planes& P, int buf,
                                             const SolveConsts& c) {
  const float tl = c.tau * c.lambda;
#pragma unroll
  for (int k = 0; k < TT::K; ++k) {
    float a = 0.0f, b = 0.0f, ig = 1.0f, sg = 1.0f, f = 1.0f, mx = 0.0f, my = 0.0f;
    if (T.on(k, P.W, P.H)) {
      const size_t i = T.gidx(P, k);
      a = __ldcg(P.tx + i);
      b = __ldcg(P.ty + i);
      ig = __ldcg(P.iG + i);
      sg = __ldcg(P.sG + i);
      f = __ldcg(P.f + i);
      mx = (T.gx0 + T.lx(k) < P.W - 1) ? 1.0f : 0.0f;
      const int gy = T.gy0 + T.ly(k);
      my = ((P.Hm == P.H ? gy : gy % P.Hm) < P.Hm - 1) ? 1.0f : 0.0f;
    }
    T.set_consts(k, a, b, ig, sg, f, mx, my, tl, c);
  }
  const float* U = P.u[buf];
  const ST *P1 = (const ST*)P.p1[buf], *P2 = (const ST*)P.p2[buf], *P3 = (const ST*)P.p3[buf];
  using S = Stor<ST>;
#pragma unroll
  for (int k = 0; k < TT::K; ++k) {
    const int j = k >> 1, h = k & 1;
    if (T.on(k, P.W, P.H)) {
      const size_t i = T.gidx(P, k);
      el(T.u[j], h) = __ldcg(U + i);
      el(T.p1[j], h) = S::ldcg(P1, i);
      el(T.p2[j], h) = S::ldcg(P2, i);
      el(T.p3[j], h) = S::ldcg(P3, i);
    } else {
      el(T.u[j], h) = 1.0f;
      el(T.p1[j], h) = el(T.p2[j], h) = el(T.p3[j], h) = 0.0f;
    }
  }
}

// Resident CTAs per SM the register budget is sized for, as for the multi-launch passes
// of the same tile: two-pixel-pair tiles at 80 registers, one-pair tiles at 64.
template <int KX, int KY, int NTY>
constexpr int kPersistMinBlocks =
    (KX * KY == 4 && 65536 / (32 * NTY * 80) > 1)   ? 65536 / (32 * NTY * 80)
    : (KX * KY == 2 && 65536 / (32 * NTY * 64) > 1) ? 65536 / (32 * NTY * 64)
                                                    : 1;

template <int KX, int KY, int NTY, typename ST>
__global__ void __launch_bounds__(32 * NTY, (kPersistMinBlocks<KX, KY, NTY>))
    k_batch_persist(const __grid_constant__ PersistArgs a) {
  using TT = Tile<KX, KY, NTY, ST>;
  __shared__ TileSmem<KX, KY, NTY, ST> sm;
  __shared__ Planes sP;  // the current item's stream
  // the current and the next work item (x < 0: none left); the next one is fetched while
  // the current one runs: its index when the current one starts, the item itself by an
  // asynchronous copy that is complete before the current item's last barrier
  __shared__ __align__(16) int4 s_w[2];
  __shared__ int s_go;
  const int tid = threadIdx.y * 32 + threadIdx.x, nthr = 32 * NTY;
  int* const counts = a.ctrl + kCtrlCount;
  const int passes = (a.iters + a.R - 1) / a.R;
  TT::zero_pads(sm);  // the iterations never write the pads
  if (tid == 0) {
    const int first = atomicAdd(a.ctrl + kCtrlHead, 1);
    s_w[0] = first < a.n_items ? a.items[first] : make_int4(-1, 0, 0, 0);
  }
  __syncthreads();
  int par = 0, cur_s = -1;
  for (;;) {
    const int4 w = s_w[par];
    if (w.x < 0) break;
    const int s = w.x, j = w.y;
    if (s != cur_s && threadIdx.y == 0) stage_planes(&sP, &a.descs[s], threadIdx.x);
    cur_s = s;
    if (tid == 0) {
      const int nxt = atomicAdd(a.ctrl + kCtrlHead, 1);  // returns during the wait
      s_go = w.w > 0 ? wait_count(counts + s * kCtrlStride, w.w, a.ctrl) : 1;
      if (nxt < a.n_items)
        copy16_async(&s_w[par ^ 1], a.items + nxt);
      else
        s_w[par ^ 1] = make_int4(-1, 0, 0, 0);
    }
    __syncthreads();
    if (s_go <= 0) {
      if (tid == 0) {
        copy_async_wait();
        if (s_go < 0 && !a.timing) atomicCAS(&sP.sc->status, 0, kErrTimeoutCode);
      }
      break;
    }
    if (j == kItemPush) {
      const long long e0 = a.offsets[s], e1 = a.offsets[s + 1];
      if (tid == 0) a.active[s] = e1 > e0 ? 1 : 0;
      if (e1 - e0 > kMaxPacket) {
        if (tid == 0) atomicCAS(&sP.sc->status, 0, kErrInvalidArgCode);
      } else if (e1 > e0) {
        push_cta(sP, a.x + e0, a.y + e0, a.t + e0, a.pol + e0, (int)(e1 - e0), tid, nthr);
      }
    } else if (a.timing || __ldcg(a.active + s)) {
      const int cur = __ldcg(a.curs + s);
      if (j == kItemPrologue) {
        prologue_band(sP, cur, a.pc, w.z, tid, nthr);
      } else {
        const int src = cur ^ (a.timing ? 0 : (j & 1));
        const int its = min(a.R, a.iters - j * a.R);
        const int tiles_x = (sP.W + (TT::EW - 2 * a.R) - 1) / (TT::EW - 2 * a.R);
        TT T;
        T.setup(w.z, tiles_x, a.R);
        load_tile_l2<TT, ST>(T, sP, src, a.c);
        if (a.c.data_term)
          for (int it = 0; it < its; ++it) T.template iterate<true>(sm, a.c);
        else
          for (int it = 0; it < its; ++it) T.template iterate<false>(sm, a.c);
        T.store(sP, 1 - src, false);
      }
    }
    if (tid == 0) copy_async_wait();  // the next item is in shared memory
    __syncthreads();                  // every write of the item is issued
    if (tid == 0) {
      if (!a.timing && j == passes - 1) {
        // a last-pass item: the stream's last item flips its buffer after an odd number
        // of passes
        __threadfence();
        const int done = atomicAdd(counts + s * kCtrlStride, 1) + 1;
        if (done == a.totals[s] && __ldcg(a.active + s) && (passes & 1)) atomicXor(a.curs + s, 1);
      } else {
        release_add(counts + s * kCtrlStride, 1);
      }
    }
    par ^= 1;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_go = atomicAdd(a.ctrl + kCtrlLeft, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (s_go) {  // every other CTA has left: clear the words for the next launch
    for (int q = tid; q < a.n_streams; q += nthr) counts[q * kCtrlStride] = 0;
    if (tid == 0) {
      a.ctrl[kCtrlHead] = 0;
      a.ctrl[kCtrlAbort] = 0;
      a.ctrl[kCtrlLeft] = 0;
    }
    __threadfence();
  }
}

template <int KX, int KY, int NTY, typename ST>
int grid_of() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persist<KX, KY, NTY, ST>,
                                                    32 * NTY, 0) != cudaSuccess)
    return 0;
  return sms * per_sm;
}

template <int KX, int KY, int NTY>
int grid_st(int storage) {
  switch (storage) {
    case 0: return grid_of<KX, KY, NTY, float>();
    case 1: return grid_of<KX, KY, NTY, __half>();
    case 2: return grid_of<KX, KY, NTY, __nv_bfloat16>();
    default: return 0;
  }
}

template <int KX, int KY, int NTY>
cudaError_t launch_st(int storage, const PersistArgs& a, int grid, cudaStream_t st) {
  const dim3 blk(32, NTY);
  switch (storage) {
    case 0: k_batch_persist<KX, KY, NTY, float><<<grid, blk, 0, st>>>(a); break;
    case 1: k_batch_persist<KX, KY, NTY, __half><<<grid, blk, 0, st>>>(a); break;
    case 2: k_batch_persist<KX, KY, NTY, __nv_bfloat16><<<grid, blk, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// The tiles the persistent step is instantiated for (kTileShapes): 32 x 32 with 256
// threads (0) and with 512 (1), 32 x 48 with 384 (6).
bool persist_supported(const SolverCfg& cfg, int storage) {
  return cfg.kind == 1 && (cfg.shape == 0 || cfg.shape == 1 || cfg.shape == 6) && storage >= 0 &&
         storage <= 2;
}

int persist_grid(const SolverCfg& cfg, int storage) {
  if (!persist_supported(cfg, storage)) return 0;
  switch (cfg.shape) {
    case 0: return grid_st<1, 4, 8>(storage);
    case 1: return grid_st<1, 2, 16>(storage);
    case 6: return grid_st<1, 4, 12>(storage);
    default: return 0;
  }
}

int launch_batch_persist(const SolverCfg& cfg, int storage, const PersistArgs& a, int grid,
                         cudaStream_t st) {
  if (!persist_supported(cfg, storage) || grid <= 0) return (int)cudaErrorInvalidValue;
  const TileShape& t = kTileShapes[cfg.shape];
  if (a.n_items > 0 && (t.EW - 2 * a.R < a.R || t.EH - 2 * a.R < a.R || a.R < 1))
    return (int)cudaErrorInvalidValue;
  switch (cfg.shape) {
    case 0: return (int)launch_st<1, 4, 8>(storage, a, grid, st);
    case 1: return (int)launch_st<1, 2, 16>(storage, a, grid, st);
    case 6: return (int)launch_st<1, 4, 12>(storage, a, grid, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int persist_node_set(cudaGraphExec_t exec, cudaGraphNode_t node, const PersistArgs& a) {
  cudaKernelNodeParams kp;
  cudaError_t e = cudaGraphKernelNodeGetParams(node, &kp);
  if (e != cudaSuccess) return (int)e;
  PersistArgs copy = a;
  void* args[] = {&copy};
  kp.kernelParams = args;
  kp.extra = nullptr;
  return (int)cudaGraphExecKernelNodeSetParams(exec, node, &kp);
}

}  // namespace evr
