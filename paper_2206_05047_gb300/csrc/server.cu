// Continuous-batching request server: light-field super-resolution requests
// arrive at any time; each is admitted in arrival order as soon as a slot
// and the device-memory budget allow, its state is created and loaded at
// the running batch's state parity, and all active light fields step
// through the ADMM iteration together (one launch per phase for all of
// them, see batch.cu).  A light field leaves exactly at its N-th iteration:
// its result is copied to host memory and its device state freed, which
// frees its slot and budget for the next request.
//
// Dry-run mode runs the same scheduling (admission order, slots, budget,
// stepping, retirement) without a device, for checking the host logic.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace lfsr;

namespace {

thread_local std::string t_server_err = "no error";

struct Request {
  lfsr_params prm{};
  std::vector<float> blur, disp, views, x0;   // owned copies until admission
  std::vector<float> proj_err;                // (paper weights, optional)
  std::vector<int32_t> view_list;             // the listed subset of the grid, if any
  int64_t bytes = 0;                          // state bytes (estimate, budgeted)
  int state = LFSR_REQ_QUEUED;
  int iters = 0;                              // ADMM iterations done
  int error = LFSR_OK;
  lfsr_handle* h = nullptr;
  std::vector<float> result;
};

}  // namespace

struct lfsr_server {
  lfsr_server_config cfg{};
  cudaStream_t stream = nullptr;
  lfsr_batch* batch = nullptr;                // launch structure over the active set
  bool have_solver = false;
  lfsr_params solver{};                       // constants every request must share
  std::map<int64_t, Request> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;
  bool changed = false;                       // active set differs from the batch's
  int64_t next_id = 0;
  int64_t bytes_in_use = 0, bytes_peak = 0;
  int64_t iterations = 0, rebuilds = 0, admitted = 0, retired = 0, dry_parity = 0, launches = 0;
  int64_t cancelled = 0;
  std::string err = "no error";
  mutable std::mutex mu;                      // every entry point holds it
};

namespace {

int sfail(lfsr_server* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  t_server_err = msg;
  set_thread_error(msg.c_str());
  return code;
}

bool dry(const lfsr_server* s) { return (s->cfg.flags & LFSR_SERVER_DRY_RUN) != 0; }

// Frees a request's host copies of its inputs (admitted or failed).
void release_inputs(Request& r) {
  for (std::vector<float>* v : {&r.blur, &r.disp, &r.views, &r.x0, &r.proj_err}) {
    v->clear();
    v->shrink_to_fit();
  }
  r.view_list.clear();
  r.view_list.shrink_to_fit();
}

// Frees a request's device state (its slot and budget).
void release(lfsr_server* s, Request& r) {
  if (r.h) lfsr_destroy(r.h);
  r.h = nullptr;
  s->bytes_in_use -= r.bytes;
  r.views.clear();
  r.views.shrink_to_fit();
  r.x0.clear();
  r.x0.shrink_to_fit();
}

// Admits queued requests in arrival order while a slot and the budget
// allow (the first one that does not fit waits: no overtaking).
int admit(lfsr_server* s) {
  while (!s->queue.empty() && (int)s->active.size() < s->cfg.max_active) {
    const int64_t id = s->queue.front();
    Request& r = s->reqs[id];
    if (r.bytes > s->cfg.hbm_budget_bytes) {   // can never fit
      s->queue.pop_front();
      r.state = LFSR_REQ_FAILED;
      r.error = LFSR_ENOMEM;
      release_inputs(r);
      continue;
    }
    if (s->bytes_in_use + r.bytes > s->cfg.hbm_budget_bytes) break;
    s->queue.pop_front();
    if (dry(s) && fault_alloc()) {   // an injected allocation failure at admission
      r.state = LFSR_REQ_FAILED;
      r.error = LFSR_ENOMEM;
      release_inputs(r);
      continue;
    }
    if (!dry(s)) {
      lfsr_params p = r.prm;
      p.blur = r.blur.data();
      p.disparity = r.disp.data();
      p.views = r.view_list.empty() ? nullptr : r.view_list.data();
      p.proj_err = r.proj_err.empty() ? nullptr : r.proj_err.data();
      lfsr_handle* h = nullptr;
      // (its operator units' costs are measured here: the batch splits its
      // launches with them at each rebuild)
      int rc = create_handle(&p, s->stream, &h, true);
      if (rc == LFSR_OK && (!h->op.fast || !h->nlf)) rc = LFSR_EUNSUPPORTED;
      const int parity = s->batch ? batch_parity(s->batch) : 0;
      if (rc == LFSR_OK)
        rc = load_state(h, r.views.data(), r.x0.data(), LFSR_MEM_HOST, parity);
      if (rc != LFSR_OK) {
        if (h) lfsr_destroy(h);
        r.state = LFSR_REQ_FAILED;
        r.error = rc;
        release_inputs(r);
        continue;
      }
      r.h = h;
    }
    // the handle holds what the solve needs: drop the host copies
    release_inputs(r);
    r.state = LFSR_REQ_ACTIVE;
    r.iters = 0;
    s->bytes_in_use += r.bytes;
    s->bytes_peak = std::max(s->bytes_peak, s->bytes_in_use);
    s->active.push_back(id);
    s->admitted += 1;
    s->changed = true;
  }
  return LFSR_OK;
}

}  // namespace

extern "C" {

int lfsr_server_create(const lfsr_server_config* cfg, void* cuda_stream, lfsr_server** out) {
  if (!out) return sfail(nullptr, LFSR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || cfg->struct_size != sizeof(lfsr_server_config))
    return sfail(nullptr, LFSR_EINVAL, "cfg->struct_size != sizeof(lfsr_server_config)");
  if (cfg->hbm_budget_bytes <= 0 || cfg->max_active < 1 || cfg->max_active > LFSR_BATCH_MAX ||
      cfg->iterations < 0 || cfg->iterations_per_step < 1)
    return sfail(nullptr, LFSR_EINVAL,
                 "budget must be > 0, max_active in [1, LFSR_BATCH_MAX], iterations >= 0, "
                 "iterations_per_step >= 1");
  lfsr_server* s = new (std::nothrow) lfsr_server();
  if (!s) return sfail(nullptr, LFSR_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->stream = (cudaStream_t)cuda_stream;
  *out = s;
  return LFSR_OK;
}

void lfsr_server_destroy(lfsr_server* s) {
  if (!s) return;
  if (!dry(s)) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs)
    if (kv.second.h) lfsr_destroy(kv.second.h);
  if (s->batch) lfsr_batch_destroy(s->batch);
  delete s;
}

const char* lfsr_server_last_error(const lfsr_server* s) {
  return s ? s->err.c_str() : t_server_err.c_str();
}

int lfsr_server_submit(lfsr_server* s, const lfsr_params* params, const float* lr_views,
                       const float* x0, int64_t* id) {
  if (!s) return sfail(nullptr, LFSR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (!params || !lr_views || !x0 || !id)
    return sfail(s, LFSR_EINVAL, "params, lr_views, x0 and id are required");
  const int64_t est = lfsr_estimate_state_bytes(params);
  if (est < 0) return sfail(s, LFSR_EINVAL, std::string("invalid request: ") + lfsr_last_error(nullptr));
  // served light fields run the batched (specialised) kernels, which take
  // one disparity map and the exact adjoint
  if (params->disparity_views || params->adjoint != LFSR_ADJOINT_EXACT)
    return sfail(s, LFSR_EUNSUPPORTED,
                 "served requests take one disparity map and the exact adjoint "
                 "(disparity_views and the backward warp run on the generic kernels)");
  if (s->have_solver && !same_solver(s->solver, *params))
    return sfail(s, LFSR_EINVAL,
                 "requests must share lambda1, lambda2, mu, the NLTV window, patch and h, "
                 "cg_iters, cg_tol, precision and the weight scheme with its sigmas");
  if (!s->have_solver) {
    s->solver = *params;
    s->have_solver = true;
  }
  Request r;
  r.prm = *params;
  const int64_t Hh = (int64_t)params->scale * params->H, Wh = (int64_t)params->scale * params->W;
  const int64_t sk = params->views ? (int64_t)params->n_views : (int64_t)params->U * params->V;
  if (params->views) r.view_list.assign(params->views, params->views + params->n_views);
  r.blur.assign(params->blur, params->blur + (size_t)params->kb * params->kb);
  r.disp.assign(params->disparity, params->disparity + (size_t)(Hh * Wh));
  if (params->weights == LFSR_WEIGHTS_PAPER && params->proj_err)
    r.proj_err.assign(params->proj_err, params->proj_err + (size_t)(Hh * Wh));
  r.views.assign(lr_views, lr_views + (size_t)(sk * params->H * params->W));
  r.x0.assign(x0, x0 + (size_t)(Hh * Wh));
  r.prm.blur = nullptr;
  r.prm.disparity = nullptr;
  r.prm.views = nullptr;
  r.prm.proj_err = nullptr;
  r.prm.disparity_views = nullptr;
  r.bytes = est;
  *id = s->next_id++;
  s->reqs.emplace(*id, std::move(r));
  s->queue.push_back(*id);
  return LFSR_OK;
}

int lfsr_server_step(lfsr_server* s) {
  NvtxRange range("lfsr_server_step (admit, step the active set, retire)");
  if (!s) return sfail(nullptr, LFSR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  admit(s);
  if (s->active.empty()) return 0;
  if (!dry(s) && s->changed) {
    if (!s->batch) s->batch = batch_new_shared(s->stream);
    if (!s->batch) return sfail(s, LFSR_ENOMEM, "host allocation failed");
    std::vector<lfsr_handle*> hs;
    for (int64_t id : s->active) hs.push_back(s->reqs[id].h);
    const cudaError_t e = batch_assign(s->batch, hs);
    if (e != cudaSuccess)
      return sfail(s, LFSR_ECUDA, std::string("rebuilding the batch: ") + cudaGetErrorString(e));
    s->rebuilds += 1;
  }
  s->changed = false;
  // iterations until the next light field is due (never past anyone's N)
  int k = s->cfg.iterations_per_step;
  for (int64_t id : s->active) k = std::min(k, s->cfg.iterations - s->reqs[id].iters);
  if (k > 0) {
    if (!dry(s)) {
      int rc = lfsr_batch_iterate(s->batch, k);
      if (rc != LFSR_OK) return sfail(s, rc, lfsr_batch_last_error(s->batch));
      s->launches += (int64_t)k * lfsr_batch_launches_per_iteration(s->batch);
      const cudaError_t e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) return sfail(s, LFSR_ECUDA, cudaGetErrorString(e));
    } else {
      s->dry_parity ^= (k & 1);
    }
    s->iterations += k;
    for (int64_t id : s->active) s->reqs[id].iters += k;
  }
  // retire the light fields that reached N: result to host, state freed
  std::vector<int64_t> keep;
  for (int64_t id : s->active) {
    Request& r = s->reqs[id];
    if (r.iters < s->cfg.iterations) {
      keep.push_back(id);
      continue;
    }
    const int64_t p = (int64_t)r.prm.scale * r.prm.H * r.prm.scale * r.prm.W;
    r.result.assign((size_t)p, 0.f);
    int rc = LFSR_OK;
    if (!dry(s)) rc = lfsr_get_x(r.h, r.result.data(), LFSR_MEM_HOST);
    r.state = rc == LFSR_OK ? LFSR_REQ_DONE : LFSR_REQ_FAILED;
    r.error = rc;
    release(s, r);
    s->retired += 1;
    s->changed = true;
  }
  s->active.swap(keep);
  return (int)s->active.size();
}

int lfsr_server_status(const lfsr_server* s, int64_t id, int* state, int* iterations) {
  if (!s) return sfail(nullptr, LFSR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LFSR_EINVAL;
  if (state) *state = it->second.state;
  if (iterations) *iterations = it->second.iters;
  return it->second.state == LFSR_REQ_FAILED ? it->second.error : LFSR_OK;
}

int lfsr_server_fetch(lfsr_server* s, int64_t id, float* x_out, int mem) {
  if (!s) return sfail(nullptr, LFSR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, LFSR_EINVAL, "unknown request");
  Request& r = it->second;
  if (r.state == LFSR_REQ_FAILED) return sfail(s, r.error, "the request failed");
  if (r.state != LFSR_REQ_DONE) return sfail(s, LFSR_EINVAL, "the request is not done");
  if (!x_out || (mem != LFSR_MEM_HOST && mem != LFSR_MEM_DEVICE))
    return sfail(s, LFSR_EINVAL, "x_out and a memory kind are required");
  if (mem == LFSR_MEM_HOST) {
    std::memcpy(x_out, r.result.data(), r.result.size() * sizeof(float));
  } else {
    const cudaError_t e = cudaMemcpyAsync(x_out, r.result.data(), r.result.size() * sizeof(float),
                                          cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return sfail(s, LFSR_ECUDA, cudaGetErrorString(e));
  }
  r.result.clear();
  r.result.shrink_to_fit();
  r.state = LFSR_REQ_FETCHED;
  return LFSR_OK;
}

int lfsr_server_stats(const lfsr_server* s, lfsr_server_stats_t* out) {
  if (!s) return sfail(nullptr, LFSR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (!out || out->struct_size != sizeof(lfsr_server_stats_t))
    return sfail(const_cast<lfsr_server*>(s), LFSR_EINVAL,
                 "out->struct_size != sizeof(lfsr_server_stats_t)");
  std::memset((char*)out + sizeof(uint32_t), 0, sizeof(lfsr_server_stats_t) - sizeof(uint32_t));
  out->queued = (int32_t)s->queue.size();
  out->active = (int32_t)s->active.size();
  for (const auto& kv : s->reqs) {
    if (kv.second.state == LFSR_REQ_DONE || kv.second.state == LFSR_REQ_FETCHED) out->done += 1;
    if (kv.second.state == LFSR_REQ_FAILED) out->failed += 1;
  }
  out->bytes_in_use = s->bytes_in_use;
  out->bytes_peak = s->bytes_peak;
  out->iterations = s->iterations;
  out->batch_rebuilds = s->rebuilds;
  out->admitted = s->admitted;
  out->retired = s->retired;
  out->launches = s->launches;
  out->cancelled = s->cancelled;
  return LFSR_OK;
}

int lfsr_server_cancel(lfsr_server* s, int64_t id) {
  if (!s) return sfail(nullptr, LFSR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, LFSR_EINVAL, "unknown request");
  Request& r = it->second;
  switch (r.state) {
    case LFSR_REQ_QUEUED:
      s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
      release_inputs(r);
      break;
    case LFSR_REQ_ACTIVE:
      // between steps no launch of the batch is in flight (a step ends with
      // a stream synchronisation): free the state, rebuild at the next step
      s->active.erase(std::find(s->active.begin(), s->active.end(), id));
      release(s, r);
      s->changed = true;
      break;
    case LFSR_REQ_DONE:
      r.result.clear();
      r.result.shrink_to_fit();
      break;
    default:
      return sfail(s, LFSR_EINVAL, "the request is already fetched, failed or cancelled");
  }
  r.state = LFSR_REQ_CANCELLED;
  s->cancelled += 1;
  return LFSR_OK;
}

}  // extern "C"
