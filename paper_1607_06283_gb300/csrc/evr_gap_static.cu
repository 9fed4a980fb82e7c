// evr_gap_static.cu -- evr_gap_static: the FP64 primal-dual gap of caller-provided
// planes, with its reduction scratch in a fixed device array instead of memory from
// cudaMalloc.
//
// Who needs this: code that must not allocate device memory once it is running --
// a real-time event-camera loop that cannot afford cudaMalloc's implicit device
// synchronisation and latency, or a host application that owns every byte of
// device memory through its own pool and forbids other allocations.  Such a caller
// passes its own input planes and a 2-double output buffer; this file allocates
// nothing.
//
// The scratch is `g_gap_partials`, one 3-double partial per chunk of 4096 pixels,
// at most kStaticChunks chunks, so the entry point accepts at most
// EVR_GAP_STATIC_MAX_PIXELS pixels.  Every GPU that loads the library holds the
// array (24 KiB) until the process exits.  All calls share it: each call overwrites
// every partial it uses before reading it, and calls that overlap on the GPU (on
// different streams, or from different host threads without ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/evr.h"

namespace {

constexpr int kChunk = 4096;         // pixels reduced by one CTA
constexpr int kStaticChunks = 1024;  // partials held by the array
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;
static_assert((long long)kChunk * kStaticChunks == EVR_GAP_STATIC_MAX_PIXELS,
              "the header's limit is the array's capacity");

static __device__ __align__(256) double g_gap_partials[3 * kStaticChunks];

// Host-side device address of g_gap_partials for each device (the symbol's name in
// host code is only a stand-in and must never be passed to a kernel), looked up by the
// first call on that device.  A device reset (cudaDeviceReset) unloads the module, so
// the address cached here is stale afterwards: the entry point must not be called on
// a device after it was reset.
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

int scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gap_partials) != cudaSuccess || !p) return EVR_ERR_CUDA;
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return EVR_OK;
}

// Per pixel, in FP64 from FP32 planes (Eq. 5 and the dual of Eq. primal_dual_energy):
// the g-tensor norm term sqrt(G)|L_g u|, and with a = lambda sqrt(G), w = -div_g p
//   KL data term (data_term 0): sqrt(G)(u - f log u) and the dual term
//     min over the box of a (u - f log u) + w u;
//   L2 data term of Eq. 7 (data_term 1, no box): sqrt(G)(u - f)^2 / 2 and the dual
//     term min over u of (a/2)(u - f)^2 + w u = w f - w^2 / (2a).
// These are the terms evr_gap reduces for a stream with the same data term.
struct GapIn {
  const float *u, *p1, *p2, *p3, *f, *tx, *ty;
  int W, H, pitch, data_term;
  double lambda, u_min, u_max;
};

__device__ __forceinline__ void mtp(const GapIn& g, size_t i, double& q1, double& q2) {
  double a = g.tx[i], b = g.ty[i];
  double G = 1.0 + a * a + b * b;
  double p1 = g.p1[i], p2 = g.p2[i], p3 = g.p3[i];
  q1 = ((1.0 + b * b) * p1 - a * b * p2 + a * p3) / G;
  q2 = (-a * b * p1 + (1.0 + a * a) * p2 + b * p3) / G;
}

__global__ void __launch_bounds__(kThreads) k_gap_static_partial(GapIn g, double* partials) {
  __shared__ double s[3][kThreads];
  double reg = 0.0, dat = 0.0, dua = 0.0;
  const int n = g.W * g.H;
  const int end = min(n, (int)(blockIdx.x + 1) * kChunk);
  for (int k = blockIdx.x * kChunk + threadIdx.x; k < end; k += kThreads) {
    const int x = k % g.W, y = k / g.W;
    const size_t i = (size_t)y * g.pitch + x;
    double a = g.tx[i], b = g.ty[i];
    double G = 1.0 + a * a + b * b, sG = sqrt(G);
    double u = g.u[i], f = g.f[i];
    double ux = (x < g.W - 1) ? (double)g.u[i + 1] - u : 0.0;
    double uy = (y < g.H - 1) ? (double)g.u[i + g.pitch] - u : 0.0;
    double g1 = ((1.0 + b * b) * ux - a * b * uy) / G;
    double g2 = ((1.0 + a * a) * uy - a * b * ux) / G;
    double g3 = (a * ux + b * uy) / G;
    reg += sqrt(G * (g1 * g1 + g2 * g2 + g3 * g3));
    if (g.data_term)
      dat += 0.5 * (u - f) * (u - f) * sG;
    else
      dat += (u - (f == 0.0 ? 0.0 : f * log(u))) * sG;
    double q1, q2, q1m = 0.0, q2m = 0.0, d;
    mtp(g, i, q1, q2);
    if (x > 0) mtp(g, i - 1, q1m, d);
    if (y > 0) mtp(g, i - g.pitch, d, q2m);
    double div = ((x < g.W - 1) ? q1 : 0.0) - q1m + ((y < g.H - 1) ? q2 : 0.0) - q2m;
    double aa = g.lambda * sG, w = -div;
    if (g.data_term) {
      dua += w * f - w * w / (2.0 * aa);
    } else {
      double us = (aa + w > 0.0) ? aa * f / (aa + w) : g.u_max;
      us = fmin(fmax(us, g.u_min), g.u_max);
      dua += aa * (us - (f == 0.0 ? 0.0 : f * log(us))) + w * us;
    }
  }
  s[0][threadIdx.x] = reg;
  s[1][threadIdx.x] = dat;
  s[2][threadIdx.x] = dua;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 3; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) partials[3 * blockIdx.x + j] = s[j][0];
}

// Fixed-order reduction of the `chunks` partials: out[0] = primal, out[1] = dual.
__global__ void __launch_bounds__(kStaticChunks) k_gap_static_final(const double* partials,
                                                                    int chunks, double lambda,
                                                                    double* out) {
  __shared__ double s[3][kStaticChunks];
  for (int j = 0; j < 3; ++j)
    s[j][threadIdx.x] = (threadIdx.x < chunks) ? partials[3 * threadIdx.x + j] : 0.0;
  __syncthreads();
  for (int h = kStaticChunks / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 3; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[0][0] + lambda * s[1][0];
    out[1] = s[2][0];
  }
}

}  // namespace

extern "C" int evr_gap_static(const float* u, const float* p1, const float* p2, const float* p3,
                              const float* f, const float* tx, const float* ty, int W, int H,
                              int pitch, float lambda, float u_min, float u_max, int data_term,
                              double* out_dev, void* cuda_stream) {
  if (!u || !p1 || !p2 || !p3 || !f || !tx || !ty || !out_dev) return EVR_ERR_INVALID_ARG;
  if (data_term != 0 && data_term != 1) return EVR_ERR_INVALID_ARG;
  if (W <= 0 || H <= 0 || pitch < W) return EVR_ERR_INVALID_ARG;
  if ((long long)W * H > EVR_GAP_STATIC_MAX_PIXELS) return EVR_ERR_INVALID_ARG;
  if (!(lambda > 0.f) || !(u_min > 0.f) || !(u_min < u_max)) return EVR_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EVR_ERR_CUDA;
  double* partials = nullptr;
  int rc = scratch_address(dev, &partials);
  if (rc) return rc;
  GapIn g{u, p1, p2, p3, f, tx, ty, W, H, pitch, data_term, (double)lambda, (double)u_min,
          (double)u_max};
  const int chunks = (int)(((long long)W * H + kChunk - 1) / kChunk);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_gap_static_partial<<<chunks, kThreads, 0, st>>>(g, partials);
  k_gap_static_final<<<1, kStaticChunks, 0, st>>>(partials, chunks, (double)lambda, out_dev);
  return cudaGetLastError() == cudaSuccess ? EVR_OK : EVR_ERR_CUDA;
}
