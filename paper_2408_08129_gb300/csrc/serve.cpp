// Serving loop: simulation requests arrive at any time, are admitted by their
// device-memory footprint, and every admitted member advances one IMEX-RK2
// step per tick through dg_batch_step (continuous batching: a request that
// arrives while others run joins at the next tick, and finished members leave
// and free their memory at once).  One worker thread per server owns the
// device work, on its own context and stream.
//
// The paper has no serving layer; this is the deployment form of the same
// path (many independent atmosphere members on one GPU).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "dg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  dg_mesh_desc desc{};
  std::vector<uint8_t> level;
  std::vector<int32_t> ijk;
  int init_kind = 0;
  std::vector<double> init_params;
  double dt = 0.0;
  int steps = 0;
  dg_solver_opts solver{};
  size_t footprint = 0;
  int64_t n_dof = 0;
  int state = DG_REQ_QUEUED;
  int status = DG_OK;
  int steps_done = 0;
  long long gmres_iters = 0;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  dg_mesh* mesh = nullptr;
  dg_state* st = nullptr;
  std::vector<double> result;
};

inline int ipow(int b, int e) {
  int r = 1;
  while (e--) r *= b;
  return r;
}

}  // namespace

struct dg_server {
  dg_ctx* ctx = nullptr;
  dg_serve_opts opts{};
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Request*> active;
  size_t used = 0;
  bool cancel = false;
  uint64_t next_id = 1;
  Clock::time_point t0;
  cudaStream_t stream = nullptr;
  std::thread worker;
  int worker_status = DG_OK;
  long long ticks = 0;
};

namespace dg {

// Device bytes a request will hold while resident: mesh tables, geometry in
// FP64 and FP32, face and vector scratch, the state with its stage vectors
// and both GMRES bases.  Faces are estimated at 1.15 x dim per cell.
size_t request_footprint(const dg_mesh_desc& d, const dg_solver_opts& o) {
  const int n = d.degree + 1, dim = d.dim, V = dim + 2;
  const double K = (double)d.n_cells, Nn = K * ipow(n, dim), NF = ipow(n, dim - 1);
  const double nf = 1.15 * dim * K + 64.0;
  const double mesh = 4.0 * (5.0 * nf + 2.0 * dim * K + 2.0 * nf * NF) +
                      12.0 * (dim * dim * Nn + 4.0 * Nn + (dim + 1.0) * nf * NF + 256.0) +
                      8.0 * (V * nf * NF + dim * Nn + 1024.0);
  const double m = (double)std::max(1, std::min(o.restart, kMaxRestart));
  const double state = 8.0 * (7.0 * V + 4.0 * dim + 8.0) * Nn + 4.0 * 3.0 * Nn + (m + 2.0) * Nn * 12.0 + 65536.0;
  return (size_t)(1.1 * (mesh + state)) + ((size_t)1 << 20);
}

namespace {

double seconds_since(const Clock::time_point& t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

void release_member(Request* r) {
  if (r->st) dg_state_destroy(r->st);
  if (r->mesh) dg_mesh_destroy(r->mesh);
  r->st = nullptr;
  r->mesh = nullptr;
}

// create the member's mesh and state on the device and write its initial state
int admit(dg_server* sv, Request* r) {
  r->desc.level = r->level.data();
  r->desc.ijk = r->ijk.data();
  int rc = dg_mesh_create(sv->ctx, &r->desc, &r->mesh);
  if (rc != DG_OK) return rc;
  rc = dg_state_create(sv->ctx, r->mesh, &r->solver, &r->st);
  if (rc != DG_OK) return rc;
  return dg_init_state(sv->ctx, r->mesh, r->init_kind, r->init_params.data(), (int)r->init_params.size(),
                       dg_state_data(r->st), sv->stream);
}

bool same_solver(const dg_solver_opts& a, const dg_solver_opts& b) {
  return a.precision == b.precision && a.picard == b.picard && a.restart == b.restart && a.tol == b.tol &&
         a.inner_tol == b.inner_tol && a.max_iters == b.max_iters && a.fused == b.fused &&
         a.max_refine == b.max_refine;
}

void worker_main(dg_server* sv) {
  cudaSetDevice(sv->ctx->device);
  for (;;) {
    std::vector<Request*> to_admit;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (sv->cancel) break;
      // first come, first served: stop at the first request that does not fit
      while (!sv->queue.empty()) {
        Request* r = sv->reqs[sv->queue.front()].get();
        const int slots = sv->opts.max_members;
        if (slots > 0 && (int)(sv->active.size() + to_admit.size()) >= slots) break;
        if (sv->used + r->footprint > sv->opts.hbm_budget_bytes) break;
        sv->queue.pop_front();
        sv->used += r->footprint;
        to_admit.push_back(r);
      }
      if (to_admit.empty() && sv->active.empty()) {
        sv->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    for (Request* r : to_admit) {
      const int rc = admit(sv, r);
      std::lock_guard<std::mutex> lk(sv->mu);
      r->t_admit = seconds_since(sv->t0);
      if (rc != DG_OK) {
        release_member(r);
        r->state = DG_REQ_FAILED;
        r->status = rc;
        r->t_finish = r->t_admit;
        sv->used -= r->footprint;
        sv->cv.notify_all();
      } else {
        r->state = DG_REQ_RUNNING;
        sv->active.push_back(r);
      }
    }
    // one step of every resident member, one batched step per solver setting
    std::vector<Request*> act;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      act = sv->active;
    }
    std::vector<bool> grouped(act.size(), false);
    for (size_t g = 0; g < act.size(); ++g) {
      if (grouped[g]) continue;
      std::vector<Request*> grp;
      for (size_t j = g; j < act.size(); ++j)
        if (!grouped[j] && same_solver(act[j]->solver, act[g]->solver)) {
          grouped[j] = true;
          grp.push_back(act[j]);
        }
      const int n = (int)grp.size();
      std::vector<const dg_mesh*> meshes(n);
      std::vector<dg_state*> states(n);
      std::vector<double> dts(n);
      std::vector<dg_step_stats> stats(n);
      std::vector<int> statuses(n, DG_OK);
      for (int i = 0; i < n; ++i) {
        meshes[i] = grp[i]->mesh;
        states[i] = grp[i]->st;
        dts[i] = grp[i]->dt;
      }
      const int rc = dg_batch_step(sv->ctx, n, meshes.data(), states.data(), dts.data(), &grp[0]->solver,
                                   stats.data(), statuses.data(), sv->stream);
      for (int i = 0; i < n; ++i) {
        Request* r = grp[i];
        int st = statuses[i];
        if (rc == DG_ECUDA || rc == DG_ETIMEOUT || rc == DG_EINVAL) st = rc;  // the launch itself failed
        r->gmres_iters += stats[i].gmres_iters;
        if (st != DG_OK) {
          r->state = DG_REQ_FAILED;
          r->status = st;
        } else if (++r->steps_done >= r->steps) {
          r->result.assign((size_t)r->n_dof, 0.0);
          const int d = dg_state_download(r->st, r->result.data());
          r->state = d == DG_OK ? DG_REQ_DONE : DG_REQ_FAILED;
          r->status = d;
        }
      }
    }
    // retire finished members and free their memory
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      ++sv->ticks;
      std::vector<Request*> keep;
      for (Request* r : sv->active) {
        if (r->state == DG_REQ_RUNNING) {
          keep.push_back(r);
          continue;
        }
        release_member(r);
        sv->used -= r->footprint;
        r->t_finish = seconds_since(sv->t0);
      }
      sv->active.swap(keep);
      sv->cv.notify_all();
    }
  }
  // cancelled: free what is resident, mark the rest as cancelled
  std::lock_guard<std::mutex> lk(sv->mu);
  for (Request* r : sv->active) {
    release_member(r);
    r->state = DG_REQ_FAILED;
    r->status = DG_EINVAL;
  }
  sv->active.clear();
  for (uint64_t id : sv->queue) {
    sv->reqs[id]->state = DG_REQ_FAILED;
    sv->reqs[id]->status = DG_EINVAL;
  }
  sv->queue.clear();
  sv->cv.notify_all();
}

}  // namespace
}  // namespace dg

using namespace dg;

extern "C" int dg_serve_create(dg_ctx* ctx, const dg_serve_opts* opts, dg_server** out) {
  if (!ctx || !opts || !out) return fail(DG_EINVAL, "null argument");
  if (opts->hbm_budget_bytes == 0) return fail(DG_EINVAL, "zero memory budget");
  auto* sv = new (std::nothrow) dg_server();
  if (!sv) return fail(DG_ENOMEM, "host allocation failed");
  sv->opts = *opts;
  int rc = dg_ctx_create(ctx->device, &sv->ctx);
  if (rc != DG_OK) {
    delete sv;
    return rc;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    dg_ctx_destroy(sv->ctx);
    delete sv;
    return cuda_fail(e, "server stream");
  }
  sv->t0 = Clock::now();
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return DG_OK;
}

extern "C" int dg_serve_submit(dg_server* sv, const dg_request* req, uint64_t* id) {
  if (!sv || !req || !id) return fail(DG_EINVAL, "null argument");
  const dg_mesh_desc& d = req->mesh;
  if ((d.dim != 2 && d.dim != 3) || d.degree < 1 || d.degree > kMaxDegree || d.n_cells <= 0 || !d.level || !d.ijk)
    return fail(DG_EINVAL, "malformed request: bad mesh description");
  if (d.node_xyz || d.conforming || d.subfaces || d.walls)
    return fail(DG_EINVAL, "malformed request: serving builds meshes from the tree (no caller geometry or face tables)");
  if (!(req->dt > 0.0) || req->steps < 1) return fail(DG_EINVAL, "malformed request: dt and steps must be positive");
  if (req->init_kind < DG_INIT_REST || req->init_kind > DG_INIT_INFLOW || req->n_init_params < 0 ||
      req->n_init_params > 8)
    return fail(DG_EINVAL, "malformed request: bad initial state");
  if (req->solver.precision != DG_FP64 && req->solver.precision != DG_FP32)
    return fail(DG_EINVAL, "malformed request: bad precision");
  auto r = std::make_unique<Request>();
  r->desc = d;
  r->level.assign(d.level, d.level + d.n_cells);
  r->ijk.assign(d.ijk, d.ijk + d.n_cells * d.dim);
  r->init_kind = req->init_kind;
  r->init_params.assign(req->init_params, req->init_params + req->n_init_params);
  r->dt = req->dt;
  r->steps = req->steps;
  r->solver = req->solver;
  r->footprint = request_footprint(d, req->solver);
  r->n_dof = (int64_t)d.n_cells * ipow(d.degree + 1, d.dim) * (d.dim + 2);
  if (r->footprint > sv->opts.hbm_budget_bytes)
    return fail(DG_EBUDGET, "request footprint " + std::to_string(r->footprint) + " bytes exceeds the budget");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->cancel) return fail(DG_EINVAL, "server is shutting down");
  r->id = sv->next_id++;
  r->t_submit = seconds_since(sv->t0);
  *id = r->id;
  sv->queue.push_back(r->id);
  sv->reqs[r->id] = std::move(r);
  sv->cv.notify_all();
  return DG_OK;
}

extern "C" int dg_serve_poll(dg_server* sv, uint64_t id, dg_request_info* info, double* host_U) {
  if (!sv) return fail(DG_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return fail(DG_EINVAL, "unknown request id");
  const Request& r = *it->second;
  if (info) {
    info->state = r.state;
    info->status = r.status;
    info->steps_done = r.steps_done;
    info->gmres_iters = r.gmres_iters;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_finish = r.t_finish;
    info->footprint_bytes = r.footprint;
    info->n_dof = r.n_dof;
  }
  if (host_U && r.state == DG_REQ_DONE && !r.result.empty())
    std::memcpy(host_U, r.result.data(), r.result.size() * sizeof(double));
  return DG_OK;
}

extern "C" int dg_serve_wait(dg_server* sv, uint64_t id, double timeout_s) {
  if (!sv) return fail(DG_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return fail(DG_EINVAL, "unknown request id");
    const Request& r = *it->second;
    if ((r.state == DG_REQ_DONE || r.state == DG_REQ_FAILED) && !r.st) return DG_OK;
    if (Clock::now() >= deadline) return fail(DG_ETIMEOUT, "request still running at the deadline");
    sv->cv.wait_until(lk, deadline);
  }
}

extern "C" int dg_serve_release(dg_server* sv, uint64_t id) {
  if (!sv) return fail(DG_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return fail(DG_EINVAL, "unknown request id");
  if (it->second->state != DG_REQ_DONE && it->second->state != DG_REQ_FAILED)
    return fail(DG_EINVAL, "request still queued or running");
  sv->reqs.erase(it);
  return DG_OK;
}

extern "C" int dg_serve_stats(dg_server* sv, dg_serve_info* info) {
  if (!sv || !info) return fail(DG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  info->queued = (int)sv->queue.size();
  info->running = (int)sv->active.size();
  info->used_bytes = sv->used;
  info->ticks = sv->ticks;
  info->elapsed_s = seconds_since(sv->t0);
  return DG_OK;
}

extern "C" int dg_serve_destroy(dg_server* sv) {
  if (!sv) return DG_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->cancel = true;
    sv->cv.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  cudaStreamDestroy(sv->stream);
  dg_ctx_destroy(sv->ctx);
  delete sv;
  return DG_OK;
}
