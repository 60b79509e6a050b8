// Batches of light fields: many light fields of different sizes, angular
// grids, scales and blurs stepped through the ADMM iteration (Algorithm 1
// with the CG x-step of Algorithm 2) together.  Every phase of an iteration
// is one launch of a table-driven kernel over a work list that spans all
// light fields of the batch -- NLTV tiles, (tile, view pair) operator units,
// chunks of HR pixels -- with one launch per group of light fields sharing
// the scale and the blur for the operator phases (the operator kernel is
// compiled per (scale, blur size)).  Two iterations are captured as one CUDA
// graph.  Each light field keeps its own state (an lfsr_handle), so loading,
// reading and diagnostics reuse the single-light-field entry points.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace lfsr;

namespace {

thread_local std::string t_batch_err = "no error";

struct Group {
  Geom g{};                 // constants of the group; S = the largest shift bound
  OpPlan P{};
  int grid = 0;
  int units = 0;
  std::vector<int> members; // indices into lfsr_batch::jobs
  std::vector<int> unit0;   // first operator unit of each member
};

}  // namespace

struct lfsr_batch {
  std::vector<lfsr_handle*> jobs;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int sm_count = 0;
  int cg_iters = 0;
  Geom g{};                 // solver constants shared by all light fields
  std::vector<Group> groups;
  int nl_total = 0, vec_total = 0, vec_chunk = 0;
  std::vector<int> nl_unit0, vec_unit0, vec_units;
  // device memory: job tables of every launch, unit -> table-entry maps,
  // reduction slots (one region per launch kind), arrival counters
  JobArgs* tables = nullptr;
  int* maps = nullptr;
  double* partials = nullptr;
  size_t part_stride = 0;
  unsigned int* counters = nullptr;
  // table offsets (entries): all light fields for the NLTV / vector launches,
  // the members of each group for the operator launches
  int t_nlw[2] = {0, 0}, t_init[2] = {0, 0};
  int t_nla[2][2] = {{0, 0}, {0, 0}}, t_upd[2][2] = {{0, 0}, {0, 0}};
  std::vector<int> t_data[2], t_norm[2][2];
  int m_nl = 0, m_vec = 0;
  std::vector<int> m_op;    // map offsets (ints)
  int parity = 0;
  int64_t iters = 0;
  cudaGraphExec_t graph_pair = nullptr;
  cudaGraphExec_t graph_single[2] = {nullptr, nullptr};
  bool profiling = false;
  std::vector<ProfEvent> prof;
  double prof_ms[8] = {0};
  int64_t prof_n[8] = {0};
  std::string err = "no error";
};

namespace {

int bfail(lfsr_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  t_batch_err = msg;
  set_thread_error(msg.c_str());
  return code;
}

void drop_events(lfsr_batch* b) {
  for (auto& ev : b->prof) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  b->prof.clear();
}

void batch_free(lfsr_batch* b) {
  drop_events(b);
  if (b->graph_pair) cudaGraphExecDestroy(b->graph_pair);
  for (auto& gs : b->graph_single)
    if (gs) cudaGraphExecDestroy(gs);
  if (b->tables) cudaFree(b->tables);
  if (b->maps) cudaFree(b->maps);
  if (b->partials) cudaFree(b->partials);
  if (b->counters) cudaFree(b->counters);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (lfsr_handle* h : b->jobs) lfsr_destroy(h);
  b->jobs.clear();
}

// Parameters every light field of a batch must share.
bool same_solver(const lfsr_params& a, const lfsr_params& c) {
  return a.lambda1 == c.lambda1 && a.lambda2 == c.lambda2 && a.mu == c.mu &&
         a.nltv_window == c.nltv_window && a.nltv_patch == c.nltv_patch && a.nltv_h == c.nltv_h &&
         a.cg_iters == c.cg_iters && a.cg_tol == c.cg_tol && a.precision == c.precision;
}

// Same operator group: scale and blur taps equal.
bool same_operator(const Geom& a, const Geom& c) {
  return a.zeta == c.zeta && a.kb == c.kb &&
         std::memcmp(a.kv, c.kv, sizeof(a.kv)) == 0 && std::memcmp(a.kh, c.kh, sizeof(a.kh)) == 0;
}

TableArgs table(lfsr_batch* b, int offset, int n, int units, int map_offset, int kind, int counter,
                int check_done) {
  TableArgs t{};
  t.jobs = b->tables + offset;
  t.unit_job = b->maps + map_offset;
  t.n_jobs = n;
  t.total_units = units;
  t.check_done = check_done;
  t.partials = b->partials + (size_t)kind * b->part_stride;
  t.counter = b->counters + counter;
  return t;
}

// One ADMM iteration of every light field of the batch at parity pa; in
// profiling mode each launch is bracketed by events (class = launch kind).
cudaError_t batch_iteration(lfsr_batch* b, int pa, cudaStream_t s, bool prof) {
  const int n = (int)b->jobs.size();
  const int G = (int)b->groups.size();
  auto ctr = [&](int kind, int gi) { return kind * (G + 1) + gi; };
  auto run = [&](int cls, auto&& launch) -> cudaError_t {
    if (!prof) return launch();
    ProfEvent ev{cls, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev.a);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
    if (e != cudaSuccess) return e;
    cudaEventRecord(ev.a, s);
    e = launch();
    cudaEventRecord(ev.b, s);
    b->prof.push_back(ev);
    return e;
  };
  cudaError_t e = run(KD_NLW, [&] {
    return nlw2_launch(
        1, b->g, table(b, b->t_nlw[pa], n, b->nl_total, b->m_nl, KD_NLW, ctr(KD_NLW, G), 0), s);
  });
  for (int gi = 0; gi < G && e == cudaSuccess; ++gi) {
    const Group& gr = b->groups[gi];
    e = run(KD_DATA, [&] {
      return fast_launch(OP_DATA, gr.g, gr.P,
                         table(b, b->t_data[pa][gi], (int)gr.members.size(), gr.units,
                               b->m_op[gi], KD_DATA, ctr(KD_DATA, gi), 0),
                         gr.grid, s, nullptr);
    });
  }
  if (e == cudaSuccess)
    e = run(KD_INIT, [&] {
      return cg_init_nltv_launch(
          b->g, table(b, b->t_init[pa], n, b->vec_total, b->m_vec, KD_INIT, ctr(KD_INIT, G), 0),
          s);
    });
  for (int k = 0; k < b->cg_iters && e == cudaSuccess; ++k) {
    const int pb = k & 1;
    e = run(KD_NLA, [&] {
      return nla2_launch(
          b->g, table(b, b->t_nla[pa][pb], n, b->nl_total, b->m_nl, KD_NLA, ctr(KD_NLA, G), 1),
          s);
    });
    for (int gi = 0; gi < G && e == cudaSuccess; ++gi) {
      const Group& gr = b->groups[gi];
      e = run(KD_NORMAL, [&] {
        return fast_launch(OP_NORMAL, gr.g, gr.P,
                           table(b, b->t_norm[pa][pb][gi], (int)gr.members.size(), gr.units,
                                 b->m_op[gi], KD_NORMAL, ctr(KD_NORMAL, gi), 1),
                           gr.grid, s, nullptr);
      });
    }
    if (e == cudaSuccess)
      e = run(KD_UPDATE, [&] {
        return cg_update_launch(b->g,
                                table(b, b->t_upd[pa][pb], n, b->vec_total, b->m_vec, KD_UPDATE,
                                      ctr(KD_UPDATE, G), 0),
                                s);
      });
  }
  return e;
}

cudaError_t batch_graph(lfsr_batch* b, int first_parity, int n, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = cudaSuccess;
  for (int i = 0; i < n && el == cudaSuccess; ++i)
    el = batch_iteration(b, (first_parity + i) & 1, b->cap_stream, false);
  e = cudaStreamEndCapture(b->cap_stream, &graph);
  if (el != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return el;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

}  // namespace

extern "C" {

int lfsr_batch_create(const lfsr_params* params, int n, void* cuda_stream, lfsr_batch** out) {
  if (!out) return bfail(nullptr, LFSR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params || n < 1 || n > LFSR_BATCH_MAX)
    return bfail(nullptr, LFSR_EINVAL, "params is NULL or n is outside [1, LFSR_BATCH_MAX]");
  for (int j = 1; j < n; ++j)
    if (!same_solver(params[0], params[j]))
      return bfail(nullptr, LFSR_EINVAL,
                   "light fields of a batch must share lambda1, lambda2, mu, the NLTV window, "
                   "patch and h, cg_iters, cg_tol and precision");
  lfsr_batch* b = new (std::nothrow) lfsr_batch();
  if (!b) return bfail(nullptr, LFSR_ENOMEM, "host allocation failed");
  b->stream = (cudaStream_t)cuda_stream;
  b->cg_iters = params[0].cg_iters;
  for (int j = 0; j < n; ++j) {
    lfsr_handle* h = nullptr;
    const int rc = lfsr_create(&params[j], cuda_stream, &h);
    if (rc != LFSR_OK) {
      const std::string msg = std::string("light field ") + std::to_string(j) + ": " +
                              lfsr_last_error(nullptr);
      batch_free(b);
      delete b;
      return bfail(nullptr, rc, msg);
    }
    b->jobs.push_back(h);
    if (!h->op.fast || !h->nlf) {
      batch_free(b);
      delete b;
      return bfail(nullptr, LFSR_EUNSUPPORTED,
                   "light field " + std::to_string(j) +
                       ": batches need a separable blur of a specialised (scale, kb) and an "
                       "NLTV window of 3, 5 or 7 with a patch of 1, 3 or 5");
    }
  }
  b->g = b->jobs[0]->g;
  b->sm_count = b->jobs[0]->sm_count;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                         b->jobs[0]->device);
  // operator groups: shared scale and blur; the layout takes the group's
  // largest shift bound
  for (int j = 0; j < n && e == cudaSuccess; ++j) {
    const Geom& gj = b->jobs[j]->g;
    int gi = 0;
    while (gi < (int)b->groups.size() && !same_operator(b->groups[gi].g, gj)) ++gi;
    if (gi == (int)b->groups.size()) {
      b->groups.emplace_back();
      b->groups.back().g = gj;
    }
    Group& gr = b->groups[gi];
    if (gj.S > gr.g.S) gr.g.S = gj.S;
    gr.unit0.push_back(gr.units);
    gr.members.push_back(j);
    gr.units += b->jobs[j]->op_units;
  }
  for (Group& gr : b->groups) {
    if (e != cudaSuccess) break;
    if (fast_plan(gr.g, &gr.P, optin - 1024) != cudaSuccess) {
      batch_free(b);
      delete b;
      return bfail(nullptr, LFSR_EUNSUPPORTED,
                   "disparity * angular offset too large for the shared-memory tile");
    }
    gr.grid = op_grid(gr.P, gr.units, b->sm_count);
  }
  // vector kernels: one chunk size for the batch, about two CTAs per SM in
  // all (plus at most one partial chunk per light field)
  size_t total_p = 0;
  for (lfsr_handle* h : b->jobs) total_p += h->p;
  {
    size_t chunk = (total_p + 2 * (size_t)b->sm_count - 1) / (2 * (size_t)b->sm_count);
    chunk = (chunk + 31) / 32 * 32;
    if (chunk < 1024) chunk = 1024;
    b->vec_chunk = (int)chunk;
  }
  for (lfsr_handle* h : b->jobs) {
    b->nl_unit0.push_back(b->nl_total);
    b->nl_total += h->nl_units;
    const int vu = (int)((h->p + b->vec_chunk - 1) / b->vec_chunk);
    b->vec_unit0.push_back(b->vec_total);
    b->vec_units.push_back(vu);
    b->vec_total += vu;
  }
  // host tables and maps
  std::vector<JobArgs> tabs;
  auto vec_job = [&](int j, int kind, int pa, int pb) {
    JobArgs a = make_job(b->jobs[j], kind, pa, pb, b->vec_unit0[j]);
    a.chunk = b->vec_chunk;
    a.units = b->vec_units[j];
    return a;
  };
  for (int pa = 0; pa < 2; ++pa) {
    b->t_nlw[pa] = (int)tabs.size();
    for (int j = 0; j < n; ++j) tabs.push_back(make_job(b->jobs[j], KD_NLW, pa, 0, b->nl_unit0[j]));
    b->t_init[pa] = (int)tabs.size();
    for (int j = 0; j < n; ++j) tabs.push_back(vec_job(j, KD_INIT, pa, 0));
    for (int pb = 0; pb < 2; ++pb) {
      b->t_nla[pa][pb] = (int)tabs.size();
      for (int j = 0; j < n; ++j) tabs.push_back(make_job(b->jobs[j], KD_NLA, pa, pb, b->nl_unit0[j]));
      b->t_upd[pa][pb] = (int)tabs.size();
      for (int j = 0; j < n; ++j) tabs.push_back(vec_job(j, KD_UPDATE, pa, pb));
    }
    for (const Group& gr : b->groups) {
      b->t_data[pa].push_back((int)tabs.size());
      for (size_t m = 0; m < gr.members.size(); ++m)
        tabs.push_back(make_job(b->jobs[gr.members[m]], KD_DATA, pa, 0, gr.unit0[m]));
      for (int pb = 0; pb < 2; ++pb) {
        b->t_norm[pa][pb].push_back((int)tabs.size());
        for (size_t m = 0; m < gr.members.size(); ++m)
          tabs.push_back(make_job(b->jobs[gr.members[m]], KD_NORMAL, pa, pb, gr.unit0[m]));
      }
    }
  }
  std::vector<int> maps;
  b->m_nl = (int)maps.size();
  for (int j = 0; j < n; ++j) maps.insert(maps.end(), b->jobs[j]->nl_units, j);
  b->m_vec = (int)maps.size();
  for (int j = 0; j < n; ++j) maps.insert(maps.end(), b->vec_units[j], j);
  for (const Group& gr : b->groups) {
    b->m_op.push_back((int)maps.size());
    for (size_t m = 0; m < gr.members.size(); ++m)
      maps.insert(maps.end(), b->jobs[gr.members[m]]->op_units, (int)m);
  }
  // reduction slots: operator launches n_members x grid, the others one per unit
  size_t stride = (size_t)b->nl_total;
  if ((size_t)b->vec_total > stride) stride = b->vec_total;
  for (const Group& gr : b->groups)
    if (gr.members.size() * (size_t)gr.grid > stride) stride = gr.members.size() * (size_t)gr.grid;
  b->part_stride = stride;
  const size_t n_counters = (size_t)KD_NUM * (b->groups.size() + 1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->tables, tabs.size() * sizeof(JobArgs));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->maps, maps.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->partials, KD_NUM * stride * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->counters, n_counters * sizeof(unsigned int));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->tables, tabs.data(), tabs.size() * sizeof(JobArgs),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->counters, 0, n_counters * sizeof(unsigned int), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    const std::string msg = std::string("lfsr_batch_create: ") + cudaGetErrorString(e);
    batch_free(b);
    delete b;
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? LFSR_ENOMEM : LFSR_ECUDA, msg);
  }
  *out = b;
  return LFSR_OK;
}

void lfsr_batch_destroy(lfsr_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
}

const char* lfsr_batch_last_error(const lfsr_batch* b) {
  return b ? b->err.c_str() : t_batch_err.c_str();
}

int lfsr_batch_size(const lfsr_batch* b) { return b ? (int)b->jobs.size() : 0; }

int lfsr_batch_load(lfsr_batch* b, int job, const float* lr_views, const float* x0, int mem) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (job < 0 || job >= (int)b->jobs.size()) return bfail(b, LFSR_EINVAL, "job out of range");
  const int rc = load_state(b->jobs[job], lr_views, x0, mem, b->parity);
  if (rc != LFSR_OK) return bfail(b, rc, lfsr_last_error(b->jobs[job]));
  return LFSR_OK;
}

int lfsr_batch_iterate(lfsr_batch* b, int iterations) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (iterations < 0) return bfail(b, LFSR_EINVAL, "iterations must be >= 0");
  int left = iterations;
  cudaError_t e = cudaSuccess;
  if (b->profiling) {
    for (; left > 0 && e == cudaSuccess; --left) {
      e = batch_iteration(b, b->parity, b->stream, true);
      b->parity ^= 1;
    }
  }
  while (left > 0 && e == cudaSuccess) {
    if (b->parity == 0 && left >= 2) {
      if (!b->graph_pair) e = batch_graph(b, 0, 2, &b->graph_pair);
      if (e == cudaSuccess) e = cudaGraphLaunch(b->graph_pair, b->stream);
      left -= 2;
    } else {
      cudaGraphExec_t& gs = b->graph_single[b->parity];
      if (!gs) e = batch_graph(b, b->parity, 1, &gs);
      if (e == cudaSuccess) e = cudaGraphLaunch(gs, b->stream);
      b->parity ^= 1;
      left -= 1;
    }
  }
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("batch iteration: ") + cudaGetErrorString(e));
  b->iters += iterations;
  for (lfsr_handle* h : b->jobs) {
    h->parity = b->parity;
    h->iters += iterations;
    h->launches = 0;
  }
  return LFSR_OK;
}

int lfsr_batch_get_x(lfsr_batch* b, int job, float* x_out, int mem) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (job < 0 || job >= (int)b->jobs.size()) return bfail(b, LFSR_EINVAL, "job out of range");
  const int rc = lfsr_get_x(b->jobs[job], x_out, mem);
  if (rc != LFSR_OK) return bfail(b, rc, lfsr_last_error(b->jobs[job]));
  return LFSR_OK;
}

int lfsr_batch_stats(const lfsr_batch* bc, int job, lfsr_stats_t* out) {
  lfsr_batch* b = const_cast<lfsr_batch*>(bc);
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (job < 0 || job >= (int)b->jobs.size()) return bfail(b, LFSR_EINVAL, "job out of range");
  const int rc = lfsr_stats(b->jobs[job], out);
  if (rc != LFSR_OK) return bfail(b, rc, lfsr_last_error(b->jobs[job]));
  out->launches = 0;
  return LFSR_OK;
}

int lfsr_batch_set_profiling(lfsr_batch* b, int on) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  cudaStreamSynchronize(b->stream);
  drop_events(b);
  b->profiling = on != 0;
  for (int c = 0; c < 8; ++c) {
    b->prof_ms[c] = 0.0;
    b->prof_n[c] = 0;
  }
  return LFSR_OK;
}

int lfsr_batch_kernel_times(lfsr_batch* b, double* ms, int64_t* launches) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (!ms || !launches) return bfail(b, LFSR_EINVAL, "ms and launches are required");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  for (auto& ev : b->prof) {
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev.a, ev.b);
    b->prof_ms[ev.cls] += t;
    b->prof_n[ev.cls] += 1;
  }
  drop_events(b);
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("kernel times: ") + cudaGetErrorString(e));
  for (int c = 0; c < 8; ++c) {
    ms[c] = b->prof_ms[c];
    launches[c] = b->prof_n[c];
  }
  return LFSR_OK;
}

int lfsr_batch_launches_per_iteration(const lfsr_batch* b) {
  if (!b) return 0;
  const int G = (int)b->groups.size();
  return 2 + G + b->cg_iters * (2 + G);
}

}  // extern "C"
