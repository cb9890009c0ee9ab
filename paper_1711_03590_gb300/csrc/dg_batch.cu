// Batched operator evaluation: many set-up operators (different meshes,
// degrees, precisions) applied by one CUDA graph launch.
//
// The graph is captured once: the applies are sorted by estimated cost and
// dealt round-robin to a few capture streams forked from one origin stream,
// so the graph has that many independent branches and the device overlaps
// applies of different sizes; every apply uses its handle's cells-per-block
// tile shape (optionally chosen by dg_autotune first).  A launch replays all
// applies with the source/destination pointers given at creation.
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/dg.h"

dg_status dg_internal_apply_on_stream(dg_handle* h, const void* src, void* dst, void* stream);
dg_status dg_internal_fail(dg_handle* h, dg_status s, const char* msg);

struct dg_batch {
  std::vector<dg_handle*> handles;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

dg_status batch_fail(dg_status s, const std::string& msg) {
  g_batch_error = msg;
  return s;
}

}  // namespace

extern "C" {

dg_status dg_batch_create(dg_handle* const* handles, const void* const* srcs, void* const* dsts, int count,
                          int autotune, int branches, void* stream, dg_batch** out) {
  if (!out) return batch_fail(DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!handles || !srcs || !dsts || count < 1) return batch_fail(DG_ERR_ARG, "empty batch or NULL arrays");
  if (branches < 1) branches = 1;
  if (branches > 32) branches = 32;
  std::vector<std::pair<double, int>> order;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !srcs[i] || !dsts[i]) return batch_fail(DG_ERR_ARG, "NULL handle or vector in the batch");
    if (autotune) {
      dg_status st = dg_autotune(handles[i], nullptr, nullptr);
      if (st != DG_OK) return batch_fail(st, std::string("autotune: ") + dg_last_error(handles[i]));
    }
    dg_info_t info;
    dg_info(handles[i], &info);
    // cost estimate: dofs times the tensor-product work per dof (~k)
    order.push_back({(double)info.n_dofs * (info.degree + 1) * (info.prec == DG_FP32 ? 1.0 : 8.0), i});
  }
  std::sort(order.begin(), order.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first;
  });

  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return batch_fail(DG_ERR_OOM, "host allocation failed");
  b->handles.assign(handles, handles + count);
  b->stream = static_cast<cudaStream_t>(stream);

  std::vector<cudaStream_t> side(branches, nullptr);
  std::vector<cudaEvent_t> ev(branches + 1, nullptr);
  cudaStream_t origin = nullptr;
  cudaGraph_t graph = nullptr;
  dg_status st = DG_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  for (int i = 0; i < branches && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
  for (int i = 0; i <= branches && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  // one plain apply per operator first: validates the arguments and makes
  // every kernel's launch configuration known before the capture
  for (int i = 0; i < count && e == cudaSuccess && st == DG_OK; ++i)
    st = dg_internal_apply_on_stream(handles[i], srcs[i], dsts[i], origin);
  if (e == cudaSuccess && st == DG_OK) e = cudaStreamSynchronize(origin);
  if (e == cudaSuccess && st == DG_OK) e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess && st == DG_OK) {
    e = cudaEventRecord(ev[branches], origin);
    for (int i = 0; i < branches && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(side[i], ev[branches], 0);
    for (int j = 0; j < count && e == cudaSuccess && st == DG_OK; ++j) {
      const int i = order[j].second;
      st = dg_internal_apply_on_stream(handles[i], srcs[i], dsts[i], side[j % branches]);
    }
    for (int i = 0; i < branches && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ev[i], side[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && st == DG_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  for (auto s : side)
    if (s) cudaStreamDestroy(s);
  for (auto v : ev)
    if (v) cudaEventDestroy(v);
  if (origin) cudaStreamDestroy(origin);
  if (st == DG_OK && e != cudaSuccess) {
    st = batch_fail(DG_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  } else if (st != DG_OK) {
    g_batch_error = "batch apply failed (see the operators' dg_last_error)";
  }
  if (st != DG_OK) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
    cudaGetLastError();
    return st;
  }
  *out = b;
  return DG_OK;
}

dg_status dg_batch_launch(dg_batch* b) {
  if (!b) return batch_fail(DG_ERR_ARG, "batch is NULL");
  cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
  if (e != cudaSuccess) {
    b->err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
    g_batch_error = b->err;
    return DG_ERR_CUDA;
  }
  return DG_OK;
}

dg_status dg_batch_destroy(dg_batch* b) {
  if (!b) return DG_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
  return DG_OK;
}

const char* dg_batch_last_error(void) { return g_batch_error.c_str(); }

}  // extern "C"
