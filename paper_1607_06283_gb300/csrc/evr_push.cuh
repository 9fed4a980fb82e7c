// evr_push.cuh -- event validation and scatter (Sec. 3, Sec. 3.1), shared by the push
// kernels (evr_kernels.cu) and the cluster solver, whose single-launch form pushes the
// packet itself (evr_cluster.cu).
#pragma once
#include <cstdint>

#include "evr_internal.cuh"

namespace evr {

// codes as in include/evr.h
constexpr int kErrOutOfRange = -2;
constexpr int kErrBadPolarity = -3;
constexpr int kErrNonmonotonic = -4;

// ---------------------------------------------------------------- event scatter
// Code of an event (x, y, t, polarity; tprev = t of the event before it) when all events
// before it are valid (then the running clock is tprev, or the stream clock for the
// first event): range, then polarity, then time.
__device__ __forceinline__ int event_code_of(int xi, int yi, long long ti, long long tprev,
                                             int pi, bool first, int W, int H, long long clock,
                                             int have_clock) {
  if (xi >= W || yi >= H) return kErrOutOfRange;
  if (pi == 0) return kErrBadPolarity;
  if (!first) {
    if (ti < tprev) return kErrNonmonotonic;
  } else if (have_clock && ti < clock) {
    return kErrNonmonotonic;
  }
  return 0;
}

__device__ __forceinline__ int event_code(const uint16_t* x, const uint16_t* y,
                                          const long long* t, const int8_t* pol, int i, int W,
                                          int H, long long clock, int have_clock) {
  return event_code_of((int)x[i], (int)y[i], t[i], i > 0 ? t[i - 1] : 0, (int)pol[i], i == 0,
                       W, H, clock, have_clock);
}

// Warp-aggregated commit of events [base, n) with stride `stride`: lanes holding
// the same pixel elect the highest lane (it carries the latest timestamp because
// the packet is sorted), which issues one atomicMax on t_last and one atomicAdd per
// polarity.  max and + commute, so the result is independent of scheduling.
__device__ __forceinline__ void commit_events(const Planes& P, const uint16_t* x, const uint16_t* y,
                                              const long long* t, const int8_t* pol, int n,
                                              int first, int stride) {
  const int lane = first & 31;  // first = the thread's linear index (a multiple of 32 per warp)
  for (int base = first - lane; base < n; base += stride) {
    int i = base + lane;
    bool ok = i < n;
    unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!ok) continue;
    int idx = (int)y[i] * P.pitch + (int)x[i];
    unsigned peers = __match_any_sync(act, idx);
    unsigned posm = __ballot_sync(act, pol[i] > 0);
    int leader = 31 - __clz(peers);
    if (lane == leader) {
      atomicMax(&P.t_last[idx], t[i]);
      int np = __popc(peers & posm);
      int nn = __popc(peers & ~posm);
      if (np) atomicAdd(&P.npos[idx], np);
      if (nn) atomicAdd(&P.nneg[idx], nn);
    }
  }
}

// One CTA validates the whole packet, then commits it: a rejected packet changes
// nothing (Sec. 3 requires theta in {-1,1}, pixels on the sensor, increasing t).
// tid: the thread's linear index in the CTA (lane = tid % 32), nthr: the CTA's threads.
__device__ __forceinline__ void push_cta(const Planes& P, const uint16_t* __restrict__ x,
                                         const uint16_t* __restrict__ y,
                                         const long long* __restrict__ t,
                                         const int8_t* __restrict__ pol, int n, int tid,
                                         int nthr) {
  __shared__ int s_bad;
  __shared__ long long s_clock;
  __shared__ int s_have;
  // each thread's first event is loaded while thread 0 fetches the stream's clock
  const int i0 = tid;
  int x0 = 0, y0 = 0, p0 = 1;
  long long t0 = 0, tp0 = 0;
  if (i0 < n) {
    x0 = x[i0];
    y0 = y[i0];
    t0 = t[i0];
    p0 = pol[i0];
    if (i0 > 0) tp0 = t[i0 - 1];
  }
  if (tid == 0) {
    s_bad = n;
    s_clock = P.sc->clock;
    s_have = P.sc->t_init_set;
  }
  __syncthreads();
  if (i0 < n &&
      event_code_of(x0, y0, t0, tp0, p0, i0 == 0, P.W, P.H, s_clock, s_have) != 0)
    atomicMin(&s_bad, i0);
  for (int i = i0 + nthr; i < n; i += nthr)
    if (event_code(x, y, t, pol, i, P.W, P.H, s_clock, s_have) != 0) atomicMin(&s_bad, i);
  __syncthreads();
  int bad = s_bad;
  if (bad < n) {
    if (tid == 0)
      atomicCAS(&P.sc->status, 0, event_code(x, y, t, pol, bad, P.W, P.H, s_clock, s_have));
    return;
  }
  commit_events(P, x, y, t, pol, n, tid, nthr);
  if (tid == 0) {
    if (!s_have) {
      P.sc->t_init = t[0];
      P.sc->t_init_set = 1;
    }
    P.sc->clock = t[n - 1] > s_clock ? t[n - 1] : s_clock;
  }
}

}  // namespace evr
