// Solve server: continuous batching of Poisson solve requests on one GPU.
//
// Requests are queued in arrival order.  A fixed number of worker threads
// ("slots"), each with its own non-blocking CUDA stream, take a queued
// request as soon as a slot is free AND the request's estimated device
// memory fits into the remaining budget; so requests that arrive while
// others run are admitted as slots and memory free up, and the GPU work of
// all admitted requests overlaps on the device.  Which queued request a
// free slot takes is the admission policy (dg_server_set_policy): the
// oldest (FIFO, the default: a large request at the head makes the others
// wait), or the smallest estimated work (dofs x (p+1)) among those that fit
// the budget, except that requests queued longer than a given age go first,
// oldest first (shortest job first with aging: small requests are not stuck
// behind large ones, and no request waits forever).  Each request is solved
// end to end with device-resident state: FP64 and FP32 operators on its
// mesh, the manufactured right-hand side, the mixed-precision solve with a
// binary32 inner CG (dg_cg_solve_mixed), optional copy of the solution to
// the host.  A solve does not depend on what else runs: all reductions have
// a fixed order, so the result is the same alone and in the mix, bit for
// bit.
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dg.h"

namespace {

struct Entry {
  dg_request req;
  dg_result res;
  int64_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
};

}  // namespace

struct dg_server {
  int device = 0;
  int64_t budget = 0;
  int64_t in_use = 0;
  int policy = 0;          // 0 FIFO, 1 shortest job first with aging
  double max_age_s = 0.0;  // policy 1: requests queued longer than this go first
  bool stopping = false;
  int64_t next_ticket = 1;
  std::deque<int64_t> queue;
  std::map<int64_t, Entry> entries;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
};

namespace {

thread_local std::string g_server_error;

dg_status server_fail(dg_status s, const std::string& m) {
  g_server_error = m;
  return s;
}

double now_s(const dg_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int64_t request_dofs(const dg_request* r) {
  const int64_t k = r->degree + 1;
  return (int64_t)r->n[0] * r->n[1] * r->n[2] * k * k * k;
}

void solve_one(dg_server* srv, Entry& e, cudaStream_t stream) {
  dg_request& r = e.req;
  dg_result& out = e.res;
  dg_mesh mesh;
  for (int d = 0; d < 3; ++d) mesh.n[d] = r.n[d];
  mesh.periodic = r.periodic;
  mesh.mapping = r.mapping;
  mesh.amplitude = r.amplitude;
  dg_opts o64;
  o64.op = DG_OP_SIPG;
  o64.prec = DG_FP64;
  o64.velocity[0] = o64.velocity[1] = o64.velocity[2] = 0.0;
  o64.coeff = r.coeff;
  o64.penalty_scale = 1.0;
  o64.basis = DG_BASIS_LAGRANGE;
  dg_opts o32 = o64;
  o32.prec = DG_FP32;
  dg_handle *h64 = nullptr, *h32 = nullptr;
  double *rhs = nullptr, *x = nullptr;
  out.n_dofs = request_dofs(&r);
  dg_status st = dg_setup(&mesh, r.degree, r.geom, &o64, stream, &h64);
  if (st == DG_OK) st = dg_setup(&mesh, r.degree, r.geom, &o32, stream, &h32);
  const size_t bytes = sizeof(double) * (size_t)out.n_dofs;
  if (st == DG_OK && (cudaMallocAsync((void**)&rhs, bytes, stream) != cudaSuccess ||
                      cudaMallocAsync((void**)&x, bytes, stream) != cudaSuccess)) {
    cudaGetLastError();
    st = DG_ERR_OOM;
  }
  if (st == DG_OK) st = dg_rhs(h64, r.which_f, rhs);
  if (st == DG_OK && cudaMemsetAsync(x, 0, bytes, stream) != cudaSuccess) st = DG_ERR_CUDA;
  if (st == DG_OK) {
    // binary32 inner CG: on the served mix (tolerance 1e-8, up to 2e7 dofs)
    // building a third, double-float operator per request for the automatic
    // choice (dg_cg_solve_mixed_auto) lowered the saturated rate by 10%
    st = dg_cg_solve_mixed(h64, h32, rhs, x, r.rtol, r.max_outer, r.inner_rtol, r.max_inner, &out.outer_iters,
                           &out.inner_iters, &out.rel_res);
  }
  if (st == DG_OK && r.x_host) {
    if (cudaMemcpyAsync(r.x_host, x, bytes, cudaMemcpyDeviceToHost, stream) != cudaSuccess) st = DG_ERR_CUDA;
  }
  if (rhs) cudaFreeAsync(rhs, stream);
  if (x) cudaFreeAsync(x, stream);
  if (cudaStreamSynchronize(stream) != cudaSuccess && st == DG_OK) st = DG_ERR_CUDA;
  if (st != DG_OK) {
    const char* m = h64 ? dg_last_error(h64) : dg_last_error(nullptr);
    snprintf(out.message, sizeof(out.message), "%s%s%s", m, h32 ? " | " : "", h32 ? dg_last_error(h32) : "");
  }
  if (h64) dg_destroy(h64);
  if (h32) dg_destroy(h32);
  out.status = st;
  (void)srv;
}

// estimated work of a request: dofs x (p + 1) (the cost of one CG iteration)
double request_work(const dg_request& r) { return (double)request_dofs(&r) * (r.degree + 1); }

// Position in the queue of the request a free slot takes now, or -1 if none
// may start (FIFO: the head when it fits; shortest job first with aging:
// the oldest request queued longer than max_age_s if it fits, else the
// smallest estimated work among the requests that fit).  Called with the
// lock held.
long pick(dg_server* srv) {
  if (srv->queue.empty()) return -1;
  if (srv->policy == 0) {
    const Entry& head = srv->entries[srv->queue.front()];
    return srv->in_use + head.bytes <= srv->budget ? 0 : -1;
  }
  const double now = now_s(srv);
  long best = -1;
  double best_work = 0.0;
  for (size_t i = 0; i < srv->queue.size(); ++i) {
    const Entry& e = srv->entries[srv->queue[i]];
    const bool fits = srv->in_use + e.bytes <= srv->budget;
    if (now - e.res.t_submit > srv->max_age_s) {
      // aged: it goes first, oldest first (and blocks younger ones while it does not fit)
      return fits ? (long)i : -1;
    }
    if (!fits) continue;
    const double w = request_work(e.req);
    if (best < 0 || w < best_work) {
      best = (long)i;
      best_work = w;
    }
  }
  return best;
}

void worker_main(dg_server* srv) {
  cudaSetDevice(srv->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  std::unique_lock<std::mutex> lock(srv->mu);
  while (true) {
    // a queued request runs as soon as the policy picks one that fits into
    // the remaining budget (aging is rechecked at least every 10 ms)
    long pos = -1;
    while (true) {
      if (srv->queue.empty()) {
        if (srv->stopping) break;
        srv->cv_work.wait(lock);
        continue;
      }
      pos = pick(srv);
      if (pos >= 0) break;
      srv->cv_work.wait_for(lock, std::chrono::milliseconds(10));
    }
    if (pos < 0) break;
    const int64_t t = srv->queue[pos];
    srv->queue.erase(srv->queue.begin() + pos);
    Entry& e = srv->entries[t];
    e.state = 1;
    srv->in_use += e.bytes;
    e.res.t_admit = now_s(srv);
    lock.unlock();
    solve_one(srv, e, stream);
    lock.lock();
    e.res.t_done = now_s(srv);
    e.state = 2;
    srv->in_use -= e.bytes;
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  lock.unlock();
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int64_t dg_request_device_bytes(const dg_request* r) {
  if (!r || r->degree < 1 || r->degree > 8 || r->n[0] < 1 || r->n[1] < 1 || r->n[2] < 1) return -1;
  const double k = r->degree + 1;
  const double dofs = (double)request_dofs(r);
  double geo = 0.0;  // bytes per dof, FP64 + FP32 operators
  if (r->geom == DG_GEOM_FULL_JAC) geo = (10.0 + 21.0 / k) * (8 + 4);
  if (r->geom == DG_GEOM_MERGED) geo = (6.0 + 21.0 / k) * (8 + 4);
  if (r->geom == DG_GEOM_POSITIONS) geo = (4.0 + 21.0 / k) * (8 + 4);
  // vectors: rhs, x, three CG vectors per operator, two inner vectors (all
  // n doubles), plus set-up scratch of one double per point
  const double vec = 8.0 * (2 + 3 + 3 + 2) + 8.0;
  return (int64_t)(dofs * (geo + vec)) + ((int64_t)64 << 20);
}

dg_status dg_server_create(int device, int64_t budget_bytes, int slots, dg_server** out) {
  if (!out) return server_fail(DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (budget_bytes <= 0 || slots < 1 || slots > 256) return server_fail(DG_ERR_ARG, "need budget > 0, 1 <= slots <= 256");
  if (cudaSetDevice(device) != cudaSuccess) return server_fail(DG_ERR_CUDA, "cudaSetDevice failed");
  // freed device memory stays in the stream-ordered pool for the next request
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  dg_server* s = new (std::nothrow) dg_server();
  if (!s) return server_fail(DG_ERR_OOM, "host allocation failed");
  s->device = device;
  s->budget = budget_bytes;
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return DG_OK;
}

dg_status dg_server_submit(dg_server* s, const dg_request* r, int64_t* ticket) {
  if (!s || !r || !ticket) return server_fail(DG_ERR_ARG, "NULL argument");
  if (r->degree < 1 || r->degree > 8 || r->n[0] < 1 || r->n[1] < 1 || r->n[2] < 1 || !(r->rtol > 0))
    return server_fail(DG_ERR_ARG, "invalid request");
  const int64_t bytes = dg_request_device_bytes(r);
  std::lock_guard<std::mutex> lock(s->mu);
  if (bytes > s->budget) return server_fail(DG_ERR_ARG, "request needs more device memory than the whole budget");
  const int64_t t = s->next_ticket++;
  Entry& e = s->entries[t];
  e.req = *r;
  e.bytes = bytes;
  e.res = dg_result();
  e.res.t_submit = now_s(s);
  e.res.device_bytes = bytes;
  s->queue.push_back(t);
  *ticket = t;
  s->cv_work.notify_all();
  return DG_OK;
}

dg_status dg_server_wait(dg_server* s, int64_t ticket, dg_result* out) {
  if (!s || !out) return server_fail(DG_ERR_ARG, "NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->entries.find(ticket);
  if (it == s->entries.end()) return server_fail(DG_ERR_ARG, "unknown ticket");
  s->cv_done.wait(lock, [&] { return it->second.state == 2; });
  *out = it->second.res;
  s->entries.erase(it);
  return DG_OK;
}

dg_status dg_server_destroy(dg_server* s) {
  if (!s) return DG_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
    s->cv_work.notify_all();
  }
  for (auto& w : s->workers) w.join();
  delete s;
  return DG_OK;
}

dg_status dg_server_set_policy(dg_server* s, int policy, double max_age_s) {
  if (!s) return server_fail(DG_ERR_ARG, "server is NULL");
  if (policy != 0 && policy != 1) return server_fail(DG_ERR_ARG, "policy must be 0 (FIFO) or 1 (shortest job first)");
  if (!(max_age_s >= 0.0)) return server_fail(DG_ERR_ARG, "max_age_s must be >= 0");
  std::lock_guard<std::mutex> lock(s->mu);
  s->policy = policy;
  s->max_age_s = max_age_s;
  s->cv_work.notify_all();
  return DG_OK;
}

const char* dg_server_last_error(void) { return g_server_error.c_str(); }

}  // extern "C"
