// dg_peak_probe: measured arithmetic peaks of this GPU (the denominators of
// the roofline fractions that are bound by the FP64 or FP32 pipe).
//
// Each thread runs CH independent fused multiply-add chains for a fixed
// number of iterations; the grid holds a whole number of resident blocks per
// SM.  FLOP/s = 2 x FMAs / the CUDA-event time of the launch (best of four
// launches after a warm-up), and the best of a few shapes (chains per
// thread, threads per block) is reported.  The chains' results feed a
// store that never happens but cannot be removed.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/dg.h"

namespace {

template <typename T, int CH, int NT>
__global__ void __launch_bounds__(NT) fma_chains(int iters, T b, T c, T* sink) {
  T a[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) a[j] = (T)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int j = 0; j < CH; ++j) a[j] = fma(a[j], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < CH; ++j) s += a[j];
  if (s == (T)-1.2345) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

// One shape (CH chains per thread, NT threads per block): FLOP/s of the best
// of four timed launches after a warm-up, in TFLOP/s; 0 on error.
template <typename T, int CH, int NT>
double time_shape(int sms, int target_fmas_per_thread, void* sink, cudaEvent_t e0, cudaEvent_t e1) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<T, CH, NT>, NT, 0) != cudaSuccess) return 0.0;
  const int blocks = sms * std::max(1, per_sm);
  const int iters = std::max(1, target_fmas_per_thread / (16 * CH));
  double best_ms = 1e30;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0, 0);
    fma_chains<T, CH, NT><<<blocks, NT>>>(iters, (T)0.999999, (T)1e-7, static_cast<T*>(sink));
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) return 0.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best_ms = std::min(best_ms, (double)ms);  // the first launch is the warm-up
  }
  const double fmas = (double)blocks * NT * CH * 16.0 * iters;
  return 2.0 * fmas / (best_ms * 1e-3) / 1e12;
}

}  // namespace

extern "C" dg_status dg_peak_probe(int kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return DG_ERR_ARG;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DG_ERR_CUDA;
  void* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * sms * 64) != cudaSuccess) return DG_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 0.0;
  dg_status st = DG_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = DG_ERR_CUDA;
  } else if (kind == 0) {
    // about 30-60 ms per launch at the nominal 1.25 TFLOP/s
    const int f = 1 << 17;
    best = std::max(best, time_shape<double, 4, 256>(sms, f, sink, e0, e1));
    best = std::max(best, time_shape<double, 8, 256>(sms, f, sink, e0, e1));
    best = std::max(best, time_shape<double, 16, 128>(sms, f, sink, e0, e1));
    best = std::max(best, time_shape<double, 8, 512>(sms, f, sink, e0, e1));
  } else {
    const int f = 1 << 21;
    best = std::max(best, time_shape<float, 8, 256>(sms, f, sink, e0, e1));
    best = std::max(best, time_shape<float, 16, 128>(sms, f, sink, e0, e1));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (st != DG_OK) return st;
  if (!(best > 0.0)) return DG_ERR_CUDA;
  *tflops = best;
  return DG_OK;
}
