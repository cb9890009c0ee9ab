// Batched operator evaluation: many set-up operators (different meshes,
// degrees, precisions) applied by one CUDA graph launch of a few fused
// kernel launches.
//
// Operators are grouped by their kernel (degree, arithmetic, geometry
// variant, weak form, face mode); each group runs as batched launches whose
// grid holds the blocks of all its operators (up to kBatchOps per launch,
// larger operators first, so the small ones fill the last wave), pulling
// (operator, block) from a prefix table of block counts in the kernel
// parameters.  The group's tile shape (cells per block) is chosen by an
// autotuner that times the group's batched launch for every valid tile shape
// (CUDA events, warm-up first), or taken from the first operator.  The
// groups' launches are captured once into a CUDA graph, dealt to a few
// branches (largest groups first) so that groups of different degrees
// overlap; a launch replays everything with the vectors given at creation.
// Each cell's arithmetic is the same as in a single apply: results equal
// the single applies bit for bit.
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.cuh"

dg_status dg_internal_apply_on_stream(dg_handle* h, const void* src, void* dst, void* stream);
dg_status dg_internal_fail(dg_handle* h, dg_status s, const char* msg);
dg_status dg_internal_batch_desc(dg_handle* h, const void* src, void* dst, dg::BatchOp* op, int key[6],
                                 const void** tables);
cudaError_t dg_internal_batch_launch(const dg::BatchLaunch& L);

struct dg_batch {
  std::vector<dg_handle*> handles;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  int launches = 0;  // kernel launches per replay
  int groups = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

dg_status batch_fail(dg_status s, const std::string& msg) {
  g_batch_error = msg;
  return s;
}

struct Group {
  int key[5];                   // degree k, arithmetic, geometry, form, face mode
  int cpb = 0;                  // tile shape of the group's launches
  std::vector<int> members;     // operator indices, largest first
  std::vector<dg::BatchOp> ops; // in the same order
  const void* tables = nullptr;
  double cost = 0.0;
};

// The group's batched launches on a stream (chunks of kBatchOps operators).
cudaError_t launch_group(const Group& g, int cpb, cudaStream_t s, int* launches) {
  for (size_t first = 0; first < g.ops.size(); first += dg::kBatchOps) {
    dg::BatchLaunch L;
    L.k = g.key[0];
    L.prec = g.key[1];
    L.geo = g.key[2];
    L.op = g.key[3];
    L.face_mode = g.key[4];
    L.cpb = cpb;
    L.tables = g.tables;
    L.nops = (int)std::min<size_t>(dg::kBatchOps, g.ops.size() - first);
    L.ops = g.ops.data() + first;
    L.stream = s;
    const cudaError_t e = dg_internal_batch_launch(L);
    if (e != cudaSuccess) return e;
    if (launches) *launches += L.face_mode != 0 ? 2 : 1;
  }
  return cudaSuccess;
}

// Autotuner of a group: the fastest tile shape for the whole batched launch.
cudaError_t tune_group(Group& g, const std::vector<int>& choices, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 1e30;
  int best_c = g.cpb;
  for (size_t i = 0; i < choices.size() && e == cudaSuccess; ++i) {
    const int c = choices[i];
    e = launch_group(g, c, s, nullptr);  // warm-up
    if (e != cudaSuccess) break;
    e = cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_group(g, c, s, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      best_c = c;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  g.cpb = best_c;
  return e;
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
  for (int i = 0; i < count; ++i)
    if (!handles[i] || !srcs[i] || !dsts[i]) return batch_fail(DG_ERR_ARG, "NULL handle or vector in the batch");
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < i; ++j)
      if (dsts[i] == dsts[j]) return batch_fail(DG_ERR_ARG, "two operators of the batch write the same dst");

  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return batch_fail(DG_ERR_OOM, "host allocation failed");
  b->handles.assign(handles, handles + count);
  b->stream = static_cast<cudaStream_t>(stream);

  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> side(branches, nullptr);
  std::vector<cudaEvent_t> ev(branches + 1, nullptr);
  cudaGraph_t graph = nullptr;
  dg_status st = DG_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  for (int i = 0; i < branches && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
  for (int i = 0; i <= branches && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);

  // one plain apply per operator first: validates the arguments and sets up
  // every kernel's launch configuration before the capture
  for (int i = 0; i < count && e == cudaSuccess && st == DG_OK; ++i)
    st = dg_internal_apply_on_stream(handles[i], srcs[i], dsts[i], origin);
  if (e == cudaSuccess && st == DG_OK) e = cudaStreamSynchronize(origin);

  // groups by kernel; members largest first
  std::vector<Group> groups;
  if (e == cudaSuccess && st == DG_OK) {
    std::map<std::vector<int>, int> index;
    std::vector<std::pair<double, int>> order;
    for (int i = 0; i < count; ++i) {
      dg_info_t info;
      dg_info(handles[i], &info);
      // cost estimate: dofs times the tensor-product work per dof (~k)
      order.push_back({(double)info.n_dofs * (info.degree + 1) * (info.prec == DG_FP32 ? 1.0 : 8.0), i});
    }
    std::stable_sort(order.begin(), order.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
      return x.first > y.first;
    });
    for (const auto& oc : order) {
      const int i = oc.second;
      dg::BatchOp op;
      int key[6];
      const void* tables = nullptr;
      st = dg_internal_batch_desc(handles[i], srcs[i], dsts[i], &op, key, &tables);
      if (st != DG_OK) break;
      std::vector<int> kk(key, key + 5);
      auto it = index.find(kk);
      if (it == index.end()) {
        Group g;
        std::copy(key, key + 5, g.key);
        g.cpb = key[5];
        g.tables = tables;
        it = index.emplace(kk, (int)groups.size()).first;
        groups.push_back(g);
      }
      Group& g = groups[it->second];
      g.members.push_back(i);
      g.ops.push_back(op);
      g.cost += oc.first;
    }
  }
  // tile shape per group
  for (size_t gi = 0; gi < groups.size() && e == cudaSuccess && st == DG_OK; ++gi) {
    Group& g = groups[gi];
    if (autotune) {
      dg_info_t info;
      dg_info(handles[g.members[0]], &info);
      std::vector<int> choices;
      for (int c : info.tile_choices)
        if (c > 0) choices.push_back(c);
      e = tune_group(g, choices, origin);
    }
    // every member reports the group's tile shape (results do not depend on it)
    for (int i : g.members)
      if (st == DG_OK) st = dg_set_cells_per_block(handles[i], g.cpb);
  }
  std::sort(groups.begin(), groups.end(), [](const Group& x, const Group& y) { return x.cost > y.cost; });

  if (e == cudaSuccess && st == DG_OK) e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess && st == DG_OK) {
    e = cudaEventRecord(ev[branches], origin);
    for (int i = 0; i < branches && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(side[i], ev[branches], 0);
    for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi)
      e = launch_group(groups[gi], groups[gi].cpb, side[gi % branches], &b->launches);
    for (int i = 0; i < branches && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ev[i], side[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && st == DG_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
  b->groups = (int)groups.size();
  if (graph) cudaGraphDestroy(graph);
  for (auto s : side)
    if (s) cudaStreamDestroy(s);
  for (auto v : ev)
    if (v) cudaEventDestroy(v);
  if (origin) cudaStreamDestroy(origin);
  if (st == DG_OK && e != cudaSuccess) {
    st = batch_fail(DG_ERR_CUDA, std::string("batched launches: ") + cudaGetErrorString(e));
  } else if (st != DG_OK) {
    g_batch_error = "batch set-up failed (see the operators' dg_last_error)";
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

dg_status dg_batch_info(const dg_batch* b, int* groups, int* launches) {
  if (!b) return batch_fail(DG_ERR_ARG, "batch is NULL");
  if (groups) *groups = b->groups;
  if (launches) *launches = b->launches;
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
