// dg_apply_dot_noalloc: operator apply plus the FP64 product src . dst, for
// callers that cannot allocate device memory.
//
// The apply kernel's dot-product epilogue needs one partial sum per CUDA
// block (scratch beyond the caller's inputs and outputs).  dg_cg_solve keeps
// that scratch in handle memory obtained with cudaMalloc on first use.  This
// entry point instead uses a fixed file-scope device array, so it never
// allocates: it suits code that runs where allocation is forbidden or unsafe,
// e.g. inside a memory pool owned by another framework, in a real-time loop
// that must not hit the allocator, or after start-up in a process whose
// device memory budget is already fully handed out.
//
// The array is part of the library's device image: every GPU on which the
// library's kernels are loaded holds it (kNoAllocPartials + 8 doubles,
// about 512 KiB) until the process exits.  All calls share it, so calls that
// overlap on the GPU (different streams or threads, no ordering between
// them) race on it and must be serialized by the caller.  Each call writes
// exactly the slots it reads back, so no slot needs clearing between calls.
//
// The array and reduce_dot sit in this translation unit, which the CUDA
// runtime loads as a module of its own; with lazy module loading (the default
// since CUDA 12.2) the array's device memory would be allocated when the
// module is first touched.  dg_setup, which allocates anyway, therefore calls
// dg_internal_noalloc_preload on its device: the module is loaded and the
// array's device address looked up there, once per device, so that
// dg_apply_dot_noalloc itself triggers neither a module load nor an
// allocation.  The first dg_setup on a device must come before any stream
// capture that records dg_apply_dot_noalloc.
#include <mutex>
#include <string>

#include "../../include/dg.h"
#include "dg_internal.cuh"

namespace {

constexpr int kNoAllocPartials = 65536;  // maximum number of apply blocks
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dot_scratch[kNoAllocPartials + 8];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_dot_scratch for the current device (host code only
// sees a host-side stand-in under that name).  Looked up once per device.
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Sum the n per-block partials in a fixed order and store the result.
__global__ void reduce_dot(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

// Load this module on the current device (the array and reduce_dot) and
// cache the array's device address.  Called by dg_setup.
cudaError_t dg_internal_noalloc_preload() {
  double* p = nullptr;
  cudaError_t e = scratch_address(&p);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes attr;
  return cudaFuncGetAttributes(&attr, reduce_dot);
}

// Defined in dg_api.cu: the apply launch with an optional per-block partial
// buffer, and the handle's sizes and stream.
dg_status dg_internal_apply_with_partials(dg_handle* h, const void* src, void* dst, double* partials,
                                          int64_t* n_blocks, cudaStream_t* stream);
dg_status dg_internal_fail(dg_handle* h, dg_status s, const char* msg);

extern "C" dg_status dg_apply_dot_noalloc(dg_handle* h, const void* src, void* dst, double* dot) {
  if (!h) return DG_ERR_ARG;
  if (!dot) return dg_internal_fail(h, DG_ERR_ARG, "dot is NULL");
  dg_info_t info;
  dg_info(h, &info);
  if (info.blocks > kNoAllocPartials) {
    std::string msg = "dg_apply_dot_noalloc: the operator needs " + std::to_string(info.blocks) +
                      " apply blocks, more than the fixed scratch of " + std::to_string(kNoAllocPartials) +
                      " partial sums; use dg_apply on a smaller mesh or dg_cg_solve's allocating path";
    return dg_internal_fail(h, DG_ERR_ARG, msg.c_str());
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    std::string msg = std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") + cudaGetErrorString(e);
    return dg_internal_fail(h, DG_ERR_CUDA, msg.c_str());
  }
  int64_t nblk = 0;
  cudaStream_t stream = nullptr;
  dg_status st = dg_internal_apply_with_partials(h, src, dst, scratch, &nblk, &stream);
  if (st != DG_OK) return st;
  reduce_dot<<<1, 256, 0, stream>>>(scratch, (int)nblk, dot);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::string msg = std::string("reduce_dot launch: ") + cudaGetErrorString(e);
    return dg_internal_fail(h, DG_ERR_CUDA, msg.c_str());
  }
  return DG_OK;
}
