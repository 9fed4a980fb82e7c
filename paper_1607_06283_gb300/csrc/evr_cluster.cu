// evr_cluster.cu -- cluster solver (kind 3) for sm_103a: the primal-dual iterations
// (Eq. cont_iterates with Eq. update_rules) on thread-block clusters whose CTAs
// exchange their tile edges through distributed shared memory every iteration.
//
// A cluster of CX x CY CTAs holds one super-tile: CTA (rx, ry) keeps the tile at
// (rx EW, ry EH) of it, with the same register-resident state and paired FP32
// arithmetic as the multi-launch solver (evr_tile.cuh).  An iteration reads q = M^T p
// at x-1 and y-1 (primal step) and ubar at x+1 and y+1 (dual step, Eq. 3 forward
// differences), so each CTA needs exactly one column and one row of each from its
// neighbours: after forming q it stores its last column to the right neighbour's pad
// and its last row to the lower neighbour's, and after the primal step it stores the
// first column and row of ubar to the left and upper neighbours.  The stores are
// st.async into the neighbour's shared memory, each completing a byte count on the
// neighbour's mbarrier (one for q, one for ubar); a CTA waits on its own mbarriers
// only for the bytes its neighbours owe it.  No cluster-wide barrier runs inside the
// iteration loop.
//
// The pad a neighbour writes for iteration k + 1 cannot overtake the reads of
// iteration k: to send q of iteration k + 1 a CTA must have finished its dual step of
// iteration k, which waited for ubar of iteration k from the receiver, which the
// receiver sent after reading its q pad of iteration k (and symmetrically for ubar).
// For the same reason no bytes of phase k + 1 can reach an mbarrier before phase k has
// completed.  The expected byte count of phase k + 1 is posted only after a CTA
// barrier that every thread reaches after polling phase k, so no thread can miss a
// phase.
//
// Only the super-tile carries a halo: with R > 0, each launch runs at most R
// iterations and the owned region is exact after them (as for the multi-launch
// solver, whose tiles each carry their own halo).  R = 0: one cluster covers the
// sensor, and one launch runs the packet's push, prologue and every iteration.
//
// Every wait is bounded.  A wait that runs out sets EVR_ERR_TIMEOUT in the stream's
// status and a flag that makes this CTA's later waits return at once; the launch
// then finishes its iterations on whatever its pads hold and reports the timeout.
// A final cluster barrier keeps every CTA alive until no neighbour can still store
// into its shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "evr_internal.cuh"
#include "evr_push.cuh"
#include "evr_tile.cuh"

namespace evr {

namespace {

constexpr int kErrTimeoutCl = -7;        // EVR_ERR_TIMEOUT
constexpr unsigned kClusterSpin = 1u << 22;  // polls of an mbarrier (shared-memory reads, a
                                             // few tens of ns each): a wait gives up well
                                             // under a second
constexpr int kMaxClusterPacket = 32768;  // events a single-launch packet may push

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// shared::cluster address of the variable at shared::cta address `a` in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival (the barrier's only one per phase) that also raises the phase's
// transaction count by `bytes`
__device__ __forceinline__ void mbar_expect(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
               "r"(bytes)
               : "memory");
}
// non-blocking test of the phase with the given parity: a suspended wait (try_wait)
// wakes late and delays every exchange
__device__ __forceinline__ bool mbar_test(uint32_t mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mb), "r"(parity)
      : "memory");
  return ok != 0;
}
// stores into another CTA's shared memory that complete their size in bytes on that
// CTA's mbarrier
__device__ __forceinline__ void st_async_f32(uint32_t a, float v, uint32_t mb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(a),
               "f"(v), "r"(mb)
               : "memory");
}
__device__ __forceinline__ void st_async_f32x2(uint32_t a, float2 v, uint32_t mb) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
          a),
      "f"(v.x), "f"(v.y), "r"(mb)
      : "memory");
}

// ---------------------------------------------------------------- edge exchange
// The tile's pads (TileSmem): q1[r][0] holds q1 at x = -1 (from the left neighbour),
// ub[r][EW] ubar at x = EW (right neighbour), q2last[0][x] q2 at y = -1 (upper
// neighbour), ubfirst[NTY][x] ubar at y = EH (lower neighbour).  Pads without a
// neighbour stay zero, as in the multi-launch solver.
template <int KX, int KY, int NTY>
struct ClusterX {
  static constexpr bool kOn = true;
  static constexpr int EW = 32 * KX, EH = NTY * KY;
  uint32_t mbq, mbu;        // this CTA's mbarriers: q pads, ubar pads
  uint32_t r_q1, r_mb;      // right neighbour: its q1 pad column, its q mbarrier
  uint32_t d_q2, d_mb;      // lower neighbour: its q2 pad row, its q mbarrier
  uint32_t l_ub, l_mb;      // left neighbour: its ubar pad column, its ubar mbarrier
  uint32_t u_ub, u_mb;      // upper neighbour: its ubar pad row, its ubar mbarrier
  uint32_t exp_q, exp_u;    // bytes the neighbours owe this CTA per iteration
  uint32_t ph_q, ph_u;      // parity of the phase to wait for
  int sends;                // bit 0 right, 1 lower, 2 left, 3 upper
  bool own_q, own_u;        // the thread that posts each mbarrier's expected bytes
  int it;                   // iterations completed
  volatile int* abort_s;    // shared: set once a wait of this CTA ran out
  int* status;              // the stream's status word

  __device__ __forceinline__ void setup(TileSmem<KX, KY, NTY, float>& sm,
                                        unsigned long long* mb, int rank, int rx, int ry,
                                        int CX, int CY, bool silent, volatile int* ab, int* st) {
    mbq = smem_addr(&mb[0]);
    mbu = smem_addr(&mb[1]);
    const bool hl = rx > 0, hr = rx < CX - 1, hu = ry > 0, hd = ry < CY - 1;
    exp_q = (hl ? (EH / 2) * 8u : 0u) + (hu ? EW * 4u : 0u);
    exp_u = (hr ? (EH / 2) * 8u : 0u) + (hd ? EW * 4u : 0u);
    sends = silent ? 0 : ((hr ? 1 : 0) | (hd ? 2 : 0) | (hl ? 4 : 0) | (hu ? 8 : 0));
    r_q1 = r_mb = d_q2 = d_mb = l_ub = l_mb = u_ub = u_mb = 0;
    if (hr) {
      r_q1 = map_rank(smem_addr(&sm.q1[0][0]), rank + 1);
      r_mb = map_rank(mbq, rank + 1);
    }
    if (hd) {
      d_q2 = map_rank(smem_addr(&sm.q2last[0][0]), rank + CX);
      d_mb = map_rank(mbq, rank + CX);
    }
    if (hl) {
      l_ub = map_rank(smem_addr(&sm.ub[0][EW]), rank - 1);
      l_mb = map_rank(mbu, rank - 1);
    }
    if (hu) {
      u_ub = map_rank(smem_addr(&sm.ubfirst[NTY][0]), rank - CX);
      u_mb = map_rank(mbu, rank - CX);
    }
    ph_q = ph_u = 0;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    own_q = tid == 0;
    own_u = tid == 32 * NTY - 1;
    it = 0;
    abort_s = ab;
    status = st;
  }

  // after the mbarriers are initialised: the expected bytes of iteration 0
  __device__ __forceinline__ void post_first() {
    if (own_q && exp_q) mbar_expect(mbq, exp_q);
    if (own_u && exp_u) mbar_expect(mbu, exp_u);
  }

  __device__ __forceinline__ void wait(uint32_t mb, uint32_t parity) {
    if (*abort_s) return;
    for (unsigned n = 0;; ++n) {
      if (mbar_test(mb, parity)) return;
      if (*abort_s) return;
      if (n >= kClusterSpin) {
        *abort_s = 1;
        atomicCAS(status, 0, kErrTimeoutCl);
        return;
      }
    }
  }

  // q of pixel pair (x, row pair row2): the last column to the right neighbour; q2 of a
  // strip's last pixel (column x1) of the last strip row to the lower neighbour
  __device__ __forceinline__ void send_q(int x, int row2, float2 q1, bool strip_last, int x1,
                                         float q2) {
    if ((sends & 1) && x == EW - 1) st_async_f32x2(r_q1 + (uint32_t)(row2 * (EW + 1)) * 8u, q1, r_mb);
    if ((sends & 2) && threadIdx.y == NTY - 1 && strip_last)
      st_async_f32(d_q2 + (uint32_t)x1 * 4u, q2, d_mb);
  }
  // ubar of pixel pair (x, row2): the first column to the left neighbour; ubar of a
  // strip's first pixel of the first strip row to the upper neighbour
  __device__ __forceinline__ void send_u(int x, int row2, float2 ub, bool strip_first) {
    if ((sends & 4) && x == 0) st_async_f32x2(l_ub + (uint32_t)(row2 * (EW + 1)) * 8u, ub, l_mb);
    if ((sends & 8) && threadIdx.y == 0 && strip_first)
      st_async_f32(u_ub + (uint32_t)x * 4u, ub.x, u_mb);
  }
  // after the barrier that ends the q phase of iteration `it`: every thread polled the
  // ubar phase of iteration it - 1 before it, so the ubar phase of this iteration can be
  // armed; then wait for this iteration's q pads
  __device__ __forceinline__ void after_bar1() {
    if (it > 0 && own_u && exp_u && !*abort_s) mbar_expect(mbu, exp_u);
    if (exp_q) {
      wait(mbq, ph_q);
      ph_q ^= 1u;
    }
  }
  // after the barrier that ends the primal step: arm the q phase of the next iteration
  // (every thread polled this one before the barrier), then wait for the ubar pads
  __device__ __forceinline__ void after_bar2() {
    if (own_q && exp_q && !*abort_s) mbar_expect(mbq, exp_q);
    if (exp_u) {
      wait(mbu, ph_u);
      ph_u ^= 1u;
    }
    ++it;
  }
};

// ---------------------------------------------------------------- kernel
struct ClusterArgs {
  Planes P;
  SolveConsts c;
  PrologueConsts pc;
  PushArgs push;  // n > 0 (R = 0 only): integrate this packet first
  int src, iters, pass;
  int front;      // 1: the packet's front is fused (see launch_cluster)
  int R, CX, CY, sup_x;
  int silent;     // wait self-test: this rank sends nothing (-1: none)
};

template <int KX, int KY, int NTY>
__global__ void __launch_bounds__(32 * NTY, 1) k_cluster(const __grid_constant__ ClusterArgs a) {
  using TT = Tile<KX, KY, NTY, float>;
  __shared__ TileSmem<KX, KY, NTY, float> sm;
  __shared__ __align__(8) unsigned long long s_mb[2];
  __shared__ int s_abort;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int rank = (int)cluster_rank();
  const int rx = rank % a.CX, ry = rank / a.CX;
  const Planes& P = a.P;
  TT T;
  T.setup_cluster((int)cluster_index(), a.sup_x, a.CX, a.CY, rx, ry, a.R);
  TT::zero_pads(sm);
  ClusterX<KX, KY, NTY> X;
  X.setup(sm, s_mb, rank, rx, ry, a.CX, a.CY, rank == a.silent, &s_abort, &P.sc->status);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(X.mbq, 1);
    mbar_init(X.mbu, 1);
    mbar_init_fence();
  }
  __syncthreads();
  X.post_first();
  // As the multi-launch passes: a pass after the one that wrote the packet constants
  // may load them before the previous pass has completed; everything else waits.
  const bool front = a.front != 0;
  const bool early = a.pass > (front ? 1 : 0);
  if (early) T.load_consts(P, a.c);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
  if (a.push.n > 0 && rank == 0)
    push_cta(P, a.push.x, a.push.y, a.push.t, a.push.pol, a.push.n, tid, 32 * NTY);
  // every CTA's mbarriers initialised and pads cleared before any neighbour stores into
  // them; the pushed packet visible to the whole cluster
  cluster_barrier();
  if (front) {
    T.load_state(P, a.src);  // f is formed from the current u
    if (a.pass == 0) {
      T.front_consts(P, a.c, a.pc);
      // one super-tile over the sensor: every pixel read its own counts above and no
      // other CTA reads them
      if (a.R == 0) T.clear_counts(P);
    } else if (!early) {
      T.load_consts(P, a.c);
      T.clear_counts(P);
    }
  } else {
    if (!early) T.load_consts(P, a.c);
    T.load_state(P, a.src);
  }
  if (a.c.data_term)
    for (int it = 0; it < a.iters; ++it) T.template iterate<true, false>(sm, a.c, &X);
  else
    for (int it = 0; it < a.iters; ++it) T.template iterate<false, false>(sm, a.c, &X);
  T.store(P, 1 - a.src, false);
  cluster_barrier();
}

// ---------------------------------------------------------------- launchers
template <int KX, int KY, int NTY>
bool geometry(const Planes& P, const SolverCfg& cfg, int* sup_x, int* sup_y) {
  if (cfg.cx < 1 || cfg.cy < 1 || cfg.cx * cfg.cy > 16 || cfg.R < 0) return false;
  const int SW = cfg.cx * 32 * KX, SH = cfg.cy * NTY * KY;
  if (cfg.R == 0) {
    *sup_x = *sup_y = 1;
    return SW >= P.W && SH >= P.H;
  }
  const int SOW = SW - 2 * cfg.R, SOH = SH - 2 * cfg.R;
  if (SOW < cfg.R || SOH < cfg.R) return false;
  *sup_x = (P.W + SOW - 1) / SOW;
  *sup_y = (P.H + SOH - 1) / SOH;
  return true;
}

template <int KX, int KY, int NTY>
void fill_config(cudaLaunchConfig_t* lc, cudaLaunchAttribute* at, const SolverCfg& cfg,
                 int n_clusters, cudaStream_t st) {
  *lc = cudaLaunchConfig_t{};
  lc->gridDim = dim3(n_clusters * cfg.cx * cfg.cy);
  lc->blockDim = dim3(32, NTY);
  lc->stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cfg.cx * cfg.cy;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  lc->attrs = at;
  lc->numAttrs = 2;
}

template <int KX, int KY, int NTY>
bool usable_t(const Planes& P, const SolverCfg& cfg) {
  int sx, sy;
  if (P.storage != 0 || !geometry<KX, KY, NTY>(P, cfg, &sx, &sy)) return false;
  // clusters of more than 8 CTAs are a non-portable size; the attribute is set here,
  // before any launch of the kernel (the autotuner and evr_create ask first)
  if (cudaFuncSetAttribute((const void*)k_cluster<KX, KY, NTY>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t lc;
  cudaLaunchAttribute at[2];
  fill_config<KX, KY, NTY>(&lc, at, cfg, sx * sy, nullptr);
  lc.numAttrs = 1;  // the cluster shape only
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_cluster<KX, KY, NTY>, &lc) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

ClusterArgs make_args(const Planes& P, const SolverCfg& cfg, int sup_x, int src, int iters,
                      int pass, const SolveConsts& c, const PrologueConsts* front,
                      const PushArgs* push, int silent) {
  ClusterArgs a{};
  a.P = P;
  a.c = c;
  a.pc = front ? *front : PrologueConsts{};
  a.push = push ? *push : PushArgs{nullptr, nullptr, nullptr, nullptr, 0};
  a.src = src;
  a.iters = iters;
  a.pass = pass;
  a.front = front ? 1 : 0;
  a.R = cfg.R;
  a.CX = cfg.cx;
  a.CY = cfg.cy;
  a.sup_x = sup_x;
  a.silent = silent;
  return a;
}

bool args_valid(const SolverCfg& cfg, int iters, const PushArgs* push) {
  if (iters < 1 || (cfg.R > 0 && iters > cfg.R)) return false;
  if (push && (cfg.R != 0 || push->n < 0 || push->n > kMaxClusterPacket)) return false;
  return true;
}

template <int KX, int KY, int NTY>
int launch_t(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
             const SolveConsts& c, cudaStream_t st, const PrologueConsts* front,
             const PushArgs* push, int silent) {
  int sx, sy;
  if (!geometry<KX, KY, NTY>(P, cfg, &sx, &sy) || !args_valid(cfg, iters, push))
    return (int)cudaErrorInvalidValue;
  const ClusterArgs a = make_args(P, cfg, sx, src, iters, pass, c, front, push, silent);
  cudaLaunchConfig_t lc;
  cudaLaunchAttribute at[2];
  fill_config<KX, KY, NTY>(&lc, at, cfg, sx * sy, st);
  return (int)cudaLaunchKernelEx(&lc, k_cluster<KX, KY, NTY>, a);
}

template <int KX, int KY, int NTY>
int set_push_t(cudaGraphExec_t exec, cudaGraphNode_t node, const Planes& P, const SolverCfg& cfg,
               int src, int iters, const SolveConsts& c, const PrologueConsts& front,
               const PushArgs& push) {
  int sx, sy;
  if (!geometry<KX, KY, NTY>(P, cfg, &sx, &sy) || !args_valid(cfg, iters, &push))
    return (int)cudaErrorInvalidValue;
  ClusterArgs a = make_args(P, cfg, sx, src, iters, 0, c, &front, &push, -1);
  cudaKernelNodeParams kp;
  cudaError_t e = cudaGraphKernelNodeGetParams(node, &kp);
  if (e != cudaSuccess) return (int)e;
  void* args[1] = {(void*)&a};
  kp.kernelParams = args;
  kp.extra = nullptr;
  return (int)cudaGraphExecKernelNodeSetParams(exec, node, &kp);
}

template <int KX, int KY, int NTY>
int ctas_t(const Planes& P, const SolverCfg& cfg) {
  int sx = 0, sy = 0;
  if (!geometry<KX, KY, NTY>(P, cfg, &sx, &sy)) return 0;
  return sx * sy * cfg.cx * cfg.cy;
}

}  // namespace

// FP32 storage only: the pads are exchanged as 32-bit values.
#define EVR_CLUSTER_DISPATCH(FN, ...)                \
  switch (cfg.shape) {                               \
    case 0: return FN<1, 4, 8>(__VA_ARGS__);         \
    case 1: return FN<1, 2, 16>(__VA_ARGS__);        \
    case 5: return FN<1, 2, 8>(__VA_ARGS__);         \
    case 6: return FN<1, 4, 12>(__VA_ARGS__);        \
    case 7: return FN<1, 2, 32>(__VA_ARGS__);        \
    default: break;                                  \
  }

int launch_cluster(const Planes& P, const SolverCfg& cfg, int src, int iters, int pass,
                   const SolveConsts& c, void* stream, const PrologueConsts* front,
                   const PushArgs* push, int silent_rank) {
  if (cfg.kind != 3 || P.storage != 0) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  EVR_CLUSTER_DISPATCH(launch_t, P, cfg, src, iters, pass, c, st, front, push, silent_rank)
  return (int)cudaErrorInvalidValue;
}

int cluster_node_set_push(void* graph_exec, void* node, const Planes& P, const SolverCfg& cfg,
                          int src, int iters, const SolveConsts& c, const PrologueConsts& front,
                          const PushArgs& push) {
  if (cfg.kind != 3) return (int)cudaErrorInvalidValue;
  cudaGraphExec_t ex = (cudaGraphExec_t)graph_exec;
  cudaGraphNode_t nd = (cudaGraphNode_t)node;
  EVR_CLUSTER_DISPATCH(set_push_t, ex, nd, P, cfg, src, iters, c, front, push)
  return (int)cudaErrorInvalidValue;
}

bool cluster_cfg_usable(const Planes& P, const SolverCfg& cfg) {
  if (cfg.kind != 3) return false;
  EVR_CLUSTER_DISPATCH(usable_t, P, cfg)
  return false;
}

int cluster_cfg_ctas(const Planes& P, const SolverCfg& cfg) {
  if (cfg.kind != 3) return 0;
  EVR_CLUSTER_DISPATCH(ctas_t, P, cfg)
  return 0;
}

}  // namespace evr
