// Batches of light fields: many light fields of different sizes, angular
// grids, scales and blurs stepped through the ADMM iteration (Algorithm 1
// with the CG x-step of Algorithm 2) together.  Every phase of an iteration
// is one launch of a table-driven kernel over a work list that spans all
// light fields of the batch -- NLTV tiles, (tile, view pair) operator units,
// chunks of HR pixels -- with one launch per group of light fields sharing
// the scale and the blur for the operator phases (the operator kernel is
// compiled per (scale, blur size)).  Two iterations are captured as one CUDA
// graph.  The persistent form runs the same phases as one cooperative launch
// per iteration (batch_persist.cuh) where a compiled instance fits.  Each
// light field keeps its own state (an lfsr_handle), so loading, reading and
// diagnostics reuse the single-light-field entry points.  An autotuner picks,
// on the batch's own data, the operator tile side of each group, the
// NLTV-apply direction chunk and the launch form (lfsr_batch_autotune).
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
  OpPlan P{};               // plan of the chosen tile side (P.TH)
  int tile = FAST_TILE;     // operator tile side (autotuned: 64 or 32)
  int grid = 0;
  int units = 0;
  std::vector<int> members; // indices into lfsr_batch::jobs
  std::vector<int> unit0;   // first operator unit of each member
  std::vector<int> units_m; // operator units of each member at this tile side
  std::vector<int> tiles_x; // tile columns of each member at this tile side
  int* cta_unit0 = nullptr; // cost-balanced CTA ranges of the operator launches (grid + 1), or NULL
  double split[2] = {0.0, 0.0};   // slowest CTA over the mean: even split, balanced
};

}  // namespace

struct lfsr_batch {
  std::vector<lfsr_handle*> jobs;
  bool owns_jobs = true;      // false: the light fields belong to a server
  std::vector<std::pair<Geom, int>> tuned_tiles;   // operator tile chosen per (scale, blur)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int sm_count = 0;
  int smem_limit = 0;
  int cg_iters = 0;
  int nla_chunk = NLA_CHUNK; // NLTV-apply direction chunk (autotuned: 6 or 3)
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
  size_t cap_tables = 0, cap_maps = 0, cap_partials = 0, cap_counters = 0;  // allocated entries
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
  // the persistent form (one cooperative launch per iteration): whether a
  // compiled instance fits the current groups, the group of each slot, its
  // launch shape, the arguments of both iteration parities (device) and the
  // grid-barrier arrival counter
  int form = LFSR_BATCH_PHASES;
  bool persist_ok = false;
  int persist_order[PERSIST_MAX_GROUPS] = {0, 0};
  size_t persist_smem = 0;
  int persist_grid = 0;
  PersistArgs* persist_args = nullptr;
  unsigned long long* bar = nullptr;
  unsigned long long wait_ns = LFSR_DEFAULT_WAIT_NS;   // device wait limit of its barriers
  int wait_unreachable = 0;
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

// Drops the balanced operator ranges (they belong to one table layout).
void free_ranges(lfsr_batch* b) {
  for (Group& gr : b->groups) {
    if (gr.cta_unit0) cudaFree(gr.cta_unit0);
    gr.cta_unit0 = nullptr;
    gr.split[0] = gr.split[1] = 0.0;
  }
}

void drop_graphs(lfsr_batch* b) {
  if (b->graph_pair) cudaGraphExecDestroy(b->graph_pair);
  b->graph_pair = nullptr;
  for (auto& gs : b->graph_single) {
    if (gs) cudaGraphExecDestroy(gs);
    gs = nullptr;
  }
}

void batch_free(lfsr_batch* b) {
  drop_events(b);
  free_ranges(b);
  drop_graphs(b);
  if (b->persist_args) cudaFree(b->persist_args);
  if (b->bar) cudaFree(b->bar);
  if (b->tables) cudaFree(b->tables);
  if (b->maps) cudaFree(b->maps);
  if (b->partials) cudaFree(b->partials);
  if (b->counters) cudaFree(b->counters);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->owns_jobs)
    for (lfsr_handle* h : b->jobs) lfsr_destroy(h);
  b->jobs.clear();
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

// One ADMM iteration of every light field of the batch at parity pa.  With
// a sink, each launch is bracketed by events (class = launch kind, grp =
// operator group).
cudaError_t batch_iteration(lfsr_batch* b, int pa, cudaStream_t s, std::vector<ProfEvent>* sink) {
  const int n = (int)b->jobs.size();
  const int G = (int)b->groups.size();
  auto ctr = [&](int kind, int gi) { return kind * (G + 1) + gi; };
  auto run = [&](int cls, int grp, auto&& launch) -> cudaError_t {
    if (!sink) return launch();
    ProfEvent ev{cls, nullptr, nullptr, grp};
    cudaError_t e = cudaEventCreate(&ev.a);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
    if (e != cudaSuccess) return e;
    cudaEventRecord(ev.a, s);
    e = launch();
    cudaEventRecord(ev.b, s);
    sink->push_back(ev);
    return e;
  };
  cudaError_t e = run(KD_NLW, 0, [&] {
    return nlw2_launch(
        1, b->g, table(b, b->t_nlw[pa], n, b->nl_total, b->m_nl, KD_NLW, ctr(KD_NLW, G), 0), s);
  });
  for (int gi = 0; gi < G && e == cudaSuccess; ++gi) {
    const Group& gr = b->groups[gi];
    e = run(KD_DATA, gi, [&] {
      TableArgs t = table(b, b->t_data[pa][gi], (int)gr.members.size(), gr.units, b->m_op[gi],
                          KD_DATA, ctr(KD_DATA, gi), 0);
      t.cta_unit0 = gr.cta_unit0;
      return fast_launch(OP_DATA, gr.g, gr.P, t, gr.grid, s, nullptr);
    });
  }
  if (e == cudaSuccess)
    e = run(KD_INIT, 0, [&] {
      return cg_init_acc_launch(
          b->g, table(b, b->t_init[pa], n, b->vec_total, b->m_vec, KD_INIT, ctr(KD_INIT, G), 0),
          s);
    });
  for (int k = 0; k < b->cg_iters && e == cudaSuccess; ++k) {
    const int pb = k & 1;
    e = run(KD_NLA, 0, [&] {
      return nla2_launch(
          b->g, table(b, b->t_nla[pa][pb], n, b->nl_total, b->m_nl, KD_NLA, ctr(KD_NLA, G), 1),
          s, b->nla_chunk);
    });
    for (int gi = 0; gi < G && e == cudaSuccess; ++gi) {
      const Group& gr = b->groups[gi];
      e = run(KD_NORMAL, gi, [&] {
        TableArgs t = table(b, b->t_norm[pa][pb][gi], (int)gr.members.size(), gr.units,
                            b->m_op[gi], KD_NORMAL, ctr(KD_NORMAL, gi), 1);
        t.cta_unit0 = gr.cta_unit0;
        return fast_launch(OP_NORMAL, gr.g, gr.P, t, gr.grid, s, nullptr);
      });
    }
    if (e == cudaSuccess)
      e = run(KD_UPDATE, 0, [&] {
        return cg_update_launch(b->g,
                                table(b, b->t_upd[pa][pb], n, b->vec_total, b->m_vec, KD_UPDATE,
                                      ctr(KD_UPDATE, G), 0),
                                s);
      });
  }
  return e;
}

// One ADMM iteration of every light field at parity pa as one persistent
// launch (batch_persist.cuh).
cudaError_t persist_iteration(lfsr_batch* b, int pa, cudaStream_t s) {
  const int G = (int)b->groups.size();
  Geom gg[PERSIST_MAX_GROUPS];
  for (int gi = 0; gi < G && gi < PERSIST_MAX_GROUPS; ++gi) gg[gi] = b->groups[gi].g;
  return persist_launch(b->g, gg, b->persist_order, G, b->persist_args + pa, b->bar,
                        b->persist_smem, b->persist_grid, s);
}

// One iteration in the batch's current form.
cudaError_t form_iteration(lfsr_batch* b, int pa, cudaStream_t s) {
  if (b->form == LFSR_BATCH_PERSISTENT) return persist_iteration(b, pa, s);
  return batch_iteration(b, pa, s, nullptr);
}

cudaError_t batch_graph(lfsr_batch* b, int first_parity, int n, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = cudaSuccess;
  for (int i = 0; i < n && el == cudaSuccess; ++i)
    el = form_iteration(b, (first_parity + i) & 1, b->cap_stream);
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

// Operator tile side of group gr: plan, per-member tiling and units, grid.
cudaError_t set_tile(lfsr_batch* b, Group& gr, int tile) {
  OpPlan P{};
  cudaError_t e = fast_plan_table(gr.g, &P, b->smem_limit, tile);
  if (e != cudaSuccess) return e;
  if (gr.cta_unit0) {   // ranges of the old unit count: the even split until rebalanced
    cudaStreamSynchronize(b->stream);
    cudaFree(gr.cta_unit0);
    gr.cta_unit0 = nullptr;
    gr.split[0] = gr.split[1] = 0.0;
  }
  gr.P = P;
  gr.tile = tile;
  gr.units = 0;
  gr.unit0.clear();
  gr.units_m.clear();
  gr.tiles_x.clear();
  for (int j : gr.members) {
    const lfsr_handle* h = b->jobs[j];
    const int tx = (h->g.Wh + tile - 1) / tile, ty = (h->g.Hh + tile - 1) / tile;
    const int um = tx * ty * ((h->g.sk + FAST_VIEWS - 1) / FAST_VIEWS);
    gr.unit0.push_back(gr.units);
    gr.units_m.push_back(um);
    gr.tiles_x.push_back(tx);
    gr.units += um;
  }
  gr.grid = op_grid(gr.P, gr.units, b->sm_count);
  return cudaSuccess;
}

// Cost-balanced CTA ranges of each operator group (see lfsr::split_by_cost):
// two timing launches of the group's normal-matrix table (the second one
// measured; timing launches leave the light fields' scalars alone, and q is
// scratch between CG steps).  Groups with fewer than two units per CTA, or
// whose balanced split would not be faster, keep the even split.
cudaError_t balance_groups(lfsr_batch* b) {
  const int G = (int)b->groups.size();
  cudaError_t e = cudaSuccess;
  for (int gi = 0; gi < G && e == cudaSuccess; ++gi) {
    Group& gr = b->groups[gi];
    if (gr.units < 2 * gr.grid) continue;
    const size_t n = (size_t)gr.units + gr.grid;
    long long* clk = nullptr;
    e = fault_alloc() ? cudaErrorMemoryAllocation : cudaMalloc((void**)&clk, n * sizeof(long long));
    if (e != cudaSuccess) break;
    TableArgs t = table(b, b->t_norm[0][0][gi], (int)gr.members.size(), gr.units, b->m_op[gi],
                        KD_NORMAL, KD_NORMAL * (G + 1) + gi, 0);
    t.unit_clock = clk;
    e = fast_launch(OP_NORMAL, gr.g, gr.P, t, gr.grid, b->stream, nullptr);   // warm-up
    if (e == cudaSuccess) e = fast_launch(OP_NORMAL, gr.g, gr.P, t, gr.grid, b->stream, nullptr);
    std::vector<long long> c(n);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c.data(), clk, n * sizeof(long long), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(clk);
    if (e != cudaSuccess) break;
    // a tile starts every (views + 1) / 2 units of each member
    std::vector<char> tile_start(gr.units, 0);
    for (size_t m = 0; m < gr.members.size(); ++m) {
      const int pairs = (b->jobs[gr.members[m]]->g.sk + FAST_VIEWS - 1) / FAST_VIEWS;
      for (int u = 0; u < gr.units_m[m]; u += pairs) tile_start[gr.unit0[m] + u] = 1;
    }
    std::vector<int> r0;
    if (!split_by_cost(c, gr.units, gr.grid, tile_start, &r0, gr.split)) continue;
    e = fault_alloc() ? cudaErrorMemoryAllocation
                      : cudaMalloc((void**)&gr.cta_unit0, r0.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(gr.cta_unit0, r0.data(), r0.size() * sizeof(int), cudaMemcpyHostToDevice,
                          b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // r0 is a local buffer
  }
  return e;
}

// Cost-balanced CTA ranges of a batch that cannot time its own launches (a
// server's, rebuilt whenever a request joins or leaves): each member's unit
// costs as its handle measured them at creation (the single-light-field
// kernel runs the same units in the same order at 64 x 64 tiles), a member
// without them (too few units to time) at the measured members' mean cost
// per unit scaled by its views per unit; the split packs them over the
// group's CTAs (see lfsr::split_by_unit_costs).  A group without any
// measured member keeps the even split.
cudaError_t member_cost_ranges(lfsr_batch* b) {
  cudaError_t e = cudaSuccess;
  for (Group& gr : b->groups) {
    if (gr.tile != FAST_TILE || gr.units < 2 * gr.grid) continue;
    double sum = 0.0, sw = 0.0;
    long long n_meas = 0;
    int members_meas = 0;
    for (size_t m = 0; m < gr.members.size(); ++m) {
      const lfsr_handle* h = b->jobs[gr.members[m]];
      if ((int)h->unit_cost.size() != gr.units_m[m]) continue;
      for (double c : h->unit_cost) sum += c;
      n_meas += (long long)h->unit_cost.size();
      sw += h->unit_cost_tile;
      ++members_meas;
    }
    if (members_meas == 0) continue;
    const double mean = sum / (double)n_meas;
    sw /= members_meas;
    std::vector<double> base((size_t)gr.units);
    std::vector<char> tile_start((size_t)gr.units, 0);
    for (size_t m = 0; m < gr.members.size(); ++m) {
      const lfsr_handle* h = b->jobs[gr.members[m]];
      const int pairs = (h->g.sk + FAST_VIEWS - 1) / FAST_VIEWS;
      const bool meas = (int)h->unit_cost.size() == gr.units_m[m];
      for (int u = 0; u < gr.units_m[m]; ++u) {
        const int pr = u % pairs;
        const int nv = std::min(FAST_VIEWS, h->g.sk - FAST_VIEWS * pr);
        base[(size_t)gr.unit0[m] + u] = meas ? h->unit_cost[u] : mean * nv / FAST_VIEWS;
        if (pr == 0) tile_start[(size_t)gr.unit0[m] + u] = 1;
      }
    }
    std::vector<int> r0;
    double mx = 0.0, mn = 0.0;
    if (!split_by_unit_costs(base, sw, tile_start, gr.grid, &r0, &mx, &mn)) continue;
    gr.split[1] = mx / mn;
    e = fault_alloc() ? cudaErrorMemoryAllocation
                      : cudaMalloc((void**)&gr.cta_unit0, r0.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(gr.cta_unit0, r0.data(), r0.size() * sizeof(int), cudaMemcpyHostToDevice,
                          b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // r0 is a local buffer
    if (e != cudaSuccess) break;
  }
  return e;
}

// The persistent form for the current groups and tables: whether a compiled
// instance fits them (else the batch keeps the per-phase launches), its
// shared memory and grid, and the arguments of both iteration parities
// (the same tables, counters and CTA ranges as the per-phase launches).
cudaError_t persist_setup(lfsr_batch* b) {
  b->persist_ok = false;
  const int G = (int)b->groups.size();
  const int n = (int)b->jobs.size();
  if (G < 1 || G > PERSIST_MAX_GROUPS) {
    b->form = LFSR_BATCH_PHASES;
    return cudaSuccess;
  }
  Geom gg[PERSIST_MAX_GROUPS];
  int tile[PERSIST_MAX_GROUPS];
  for (int gi = 0; gi < G; ++gi) {
    gg[gi] = b->groups[gi].g;
    tile[gi] = b->groups[gi].tile;
  }
  int* order = b->persist_order;
  OpPlan P[PERSIST_MAX_GROUPS];
  int sx_off = 0;
  bool ok = persist_supported(b->g, gg, tile, G, order);
  if (ok) {
    for (int sl = 0; sl < G; ++sl) P[sl] = b->groups[order[sl]].P;
    b->persist_smem = persist_smem(b->g, P, G, &sx_off);
    ok = b->persist_smem <= (size_t)b->smem_limit &&
         persist_prepare(b->g, gg, order, G, b->smem_limit + 1024) == cudaSuccess &&
         persist_occupancy(b->g, gg, order, G, b->persist_smem) >= 1;
  }
  if (!ok) {
    cudaGetLastError();   // an attribute call that failed leaves no sticky error
    b->form = LFSR_BATCH_PHASES;
    return cudaSuccess;
  }
  b->persist_grid = b->sm_count;
  auto ctr = [&](int kind, int gi) { return kind * (G + 1) + gi; };
  PersistArgs pa_args[2];
  for (int pa = 0; pa < 2; ++pa) {
    PersistArgs& a = pa_args[pa];
    a = PersistArgs{};
    a.nlw = table(b, b->t_nlw[pa], n, b->nl_total, b->m_nl, KD_NLW, ctr(KD_NLW, G), 0);
    a.init = table(b, b->t_init[pa], n, b->vec_total, b->m_vec, KD_INIT, ctr(KD_INIT, G), 0);
    for (int pb = 0; pb < 2; ++pb) {
      a.nla[pb] = table(b, b->t_nla[pa][pb], n, b->nl_total, b->m_nl, KD_NLA, ctr(KD_NLA, G), 1);
      a.upd[pb] =
          table(b, b->t_upd[pa][pb], n, b->vec_total, b->m_vec, KD_UPDATE, ctr(KD_UPDATE, G), 0);
    }
    for (int sl = 0; sl < G; ++sl) {
      const int gi = order[sl];
      const Group& gr = b->groups[gi];
      const int m = (int)gr.members.size();
      // the balanced ranges split the units over gr.grid CTAs
      const int* ranges = gr.grid == b->persist_grid ? gr.cta_unit0 : nullptr;
      a.data[sl] = table(b, b->t_data[pa][gi], m, gr.units, b->m_op[gi], KD_DATA, ctr(KD_DATA, gi), 0);
      a.data[sl].cta_unit0 = ranges;
      for (int pb = 0; pb < 2; ++pb) {
        a.norm[pb][sl] = table(b, b->t_norm[pa][pb][gi], m, gr.units, b->m_op[gi], KD_NORMAL,
                               ctr(KD_NORMAL, gi), 1);
        a.norm[pb][sl].cta_unit0 = ranges;
      }
      a.P[sl] = gr.P;
    }
    a.cg_iters = b->cg_iters;
    a.sx_off = sx_off;
  }
  cudaError_t e = cudaSuccess;
  if (!b->persist_args)
    e = fault_alloc() ? cudaErrorMemoryAllocation
                      : cudaMalloc((void**)&b->persist_args, 2 * sizeof(PersistArgs));
  if (e == cudaSuccess && !b->bar) {
    e = fault_alloc() ? cudaErrorMemoryAllocation
                      : cudaMalloc((void**)&b->bar, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned long long), b->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->persist_args, pa_args, sizeof(pa_args), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // pa_args is a local buffer
  if (e == cudaSuccess) b->persist_ok = true;
  else b->form = LFSR_BATCH_PHASES;
  return e;
}

// Builds the job tables and unit maps of every launch for the current tile
// sides, uploads them (growing the device buffers when needed) and drops
// the captured graphs, which hold the old launch shapes.  A batch that owns
// its light fields then balances its operator groups' CTA ranges.
cudaError_t build_tables(lfsr_batch* b) {
  const int n = (int)b->jobs.size();
  std::vector<JobArgs> tabs;
  auto vec_job = [&](int j, int kind, int pa, int pb) {
    JobArgs a = make_job(b->jobs[j], kind, pa, pb, b->vec_unit0[j]);
    a.chunk = b->vec_chunk;
    a.units = b->vec_units[j];
    return a;
  };
  auto op_job = [&](const Group& gr, size_t m, int kind, int pa, int pb) {
    JobArgs a = make_job(b->jobs[gr.members[m]], kind, pa, pb, gr.unit0[m]);
    a.units = gr.units_m[m];
    a.tiles_x = gr.tiles_x[m];
    return a;
  };
  for (int pa = 0; pa < 2; ++pa) {
    b->t_data[pa].clear();
    for (int pb = 0; pb < 2; ++pb) b->t_norm[pa][pb].clear();
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
      for (size_t m = 0; m < gr.members.size(); ++m) tabs.push_back(op_job(gr, m, KD_DATA, pa, 0));
      for (int pb = 0; pb < 2; ++pb) {
        b->t_norm[pa][pb].push_back((int)tabs.size());
        for (size_t m = 0; m < gr.members.size(); ++m)
          tabs.push_back(op_job(gr, m, KD_NORMAL, pa, pb));
      }
    }
  }
  std::vector<int> maps;
  b->m_nl = (int)maps.size();
  for (int j = 0; j < n; ++j) maps.insert(maps.end(), b->jobs[j]->nl_units, j);
  b->m_vec = (int)maps.size();
  for (int j = 0; j < n; ++j) maps.insert(maps.end(), b->vec_units[j], j);
  b->m_op.clear();
  for (const Group& gr : b->groups) {
    b->m_op.push_back((int)maps.size());
    for (size_t m = 0; m < gr.members.size(); ++m) maps.insert(maps.end(), gr.units_m[m], (int)m);
  }
  // reduction slots: operator launches n_members x grid, the others one per unit
  size_t stride = (size_t)b->nl_total;
  if ((size_t)b->vec_total > stride) stride = b->vec_total;
  // (the persistent form runs the operator phases on sm_count CTAs)
  for (const Group& gr : b->groups) {
    const size_t grid = gr.grid > b->sm_count ? (size_t)gr.grid : (size_t)b->sm_count;
    if (gr.members.size() * grid > stride) stride = gr.members.size() * grid;
  }
  b->part_stride = stride;
  cudaError_t e = cudaStreamSynchronize(b->stream);   // no launch may still read the old tables
  free_ranges(b);                                    // (they belong to the old layout)
  auto grow = [&](auto** buf, size_t* cap, size_t need, size_t elem) {
    if (e != cudaSuccess || need <= *cap) return;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    e = fault_alloc() ? cudaErrorMemoryAllocation : cudaMalloc((void**)buf, need * elem);
    if (e == cudaSuccess) *cap = need;
  };
  grow(&b->tables, &b->cap_tables, tabs.size(), sizeof(JobArgs));
  grow(&b->maps, &b->cap_maps, maps.size(), sizeof(int));
  grow(&b->partials, &b->cap_partials, KD_NUM * stride, sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->tables, tabs.data(), tabs.size() * sizeof(JobArgs),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (e == cudaSuccess) e = b->owns_jobs ? balance_groups(b) : member_cost_ranges(b);
  if (e == cudaSuccess) e = persist_setup(b);
  return e;
}

// Device time of one iteration's launches that match (cls, grp) (grp < 0:
// any group); the iteration runs at the current parity and advances it.
cudaError_t time_iteration(lfsr_batch* b, int cls, int grp, double* ms) {
  std::vector<ProfEvent> ev;
  cudaError_t e = batch_iteration(b, b->parity, b->stream, &ev);
  b->parity ^= 1;
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  double t = 0.0;
  for (auto& x : ev) {
    float m = 0.f;
    if (e == cudaSuccess && x.cls == cls && (grp < 0 || x.grp == grp))
      e = cudaEventElapsedTime(&m, x.a, x.b);
    t += m;
    cudaEventDestroy(x.a);
    cudaEventDestroy(x.b);
  }
  *ms = t;
  return e;
}

// Device time of two iterations in the current form, after one warm-up
// iteration (all at the current parity, which advances).
cudaError_t time_form(lfsr_batch* b, double* ms) {
  cudaEvent_t a = nullptr, c = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&c);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    if (i == 1) e = cudaEventRecord(a, b->stream);
    if (e == cudaSuccess) e = form_iteration(b, b->parity, b->stream);
    b->parity ^= 1;
  }
  if (e == cudaSuccess) e = cudaEventRecord(c, b->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(c);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, c);
  *ms = t;
  if (a) cudaEventDestroy(a);
  if (c) cudaEventDestroy(c);
  return e;
}

}  // namespace

// (Re)builds the launch structure of the batch over `jobs` (all of them on
// the specialised path, sharing the solver constants): operator groups and
// their plans, unit offsets, vector chunking, job tables and maps.  The
// graphs are dropped.  An empty list leaves an empty batch.
cudaError_t lfsr::batch_assign(lfsr_batch* b, const std::vector<lfsr_handle*>& jobs) {
  // remember the tuned tile side of every group before regrouping
  for (const Group& gr : b->groups) {
    bool found = false;
    for (auto& tt : b->tuned_tiles)
      if (same_operator(tt.first, gr.g)) {
        tt.second = gr.tile;
        found = true;
      }
    if (!found) b->tuned_tiles.emplace_back(gr.g, gr.tile);
  }
  if (&jobs != &b->jobs) b->jobs = jobs;
  cudaStreamSynchronize(b->stream);
  free_ranges(b);
  b->groups.clear();
  b->nl_unit0.clear();
  b->vec_unit0.clear();
  b->vec_units.clear();
  b->nl_total = b->vec_total = 0;
  const int n = (int)b->jobs.size();
  if (n == 0) return cudaSuccess;
  b->g = b->jobs[0]->g;
  b->g.wait_ns = b->wait_ns;
  b->g.wait_unreachable = b->wait_unreachable;
  b->sm_count = b->jobs[0]->sm_count;
  b->cg_iters = b->jobs[0]->prm.cg_iters;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                         b->jobs[0]->device);
  b->smem_limit = optin - 1024;
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
    gr.members.push_back(j);
  }
  for (Group& gr : b->groups) {
    if (e != cudaSuccess) break;
    int tile = FAST_TILE;
    for (const auto& tt : b->tuned_tiles)
      if (same_operator(tt.first, gr.g)) tile = tt.second;
    if (set_tile(b, gr, tile) != cudaSuccess && set_tile(b, gr, FAST_TILE) != cudaSuccess)
      return cudaErrorInvalidValue;
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
  const size_t n_counters = (size_t)KD_NUM * (b->groups.size() + 1);
  if (e == cudaSuccess && !b->cap_stream)
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && n_counters > b->cap_counters) {
    if (b->counters) cudaFree(b->counters);
    b->counters = nullptr;
    b->cap_counters = 0;
    e = fault_alloc() ? cudaErrorMemoryAllocation
                      : cudaMalloc((void**)&b->counters, n_counters * sizeof(unsigned int));
    if (e == cudaSuccess) {
      b->cap_counters = n_counters;
      e = cudaMemsetAsync(b->counters, 0, n_counters * sizeof(unsigned int), b->stream);
    }
  }
  if (e == cudaSuccess) e = build_tables(b);
  return e;
}

lfsr_batch* lfsr::batch_new_shared(cudaStream_t stream) {
  lfsr_batch* b = new (std::nothrow) lfsr_batch();
  if (!b) return nullptr;
  b->owns_jobs = false;
  b->stream = stream;
  return b;
}

int lfsr::batch_parity(const lfsr_batch* b) { return b->parity; }

// Parameters every light field of a batch (and of a server) must share.
bool lfsr::same_solver(const lfsr_params& a, const lfsr_params& c) {
  if (a.weights != c.weights) return false;
  if (a.weights == LFSR_WEIGHTS_PAPER &&
      (a.sigma_s != c.sigma_s || a.sigma_e != c.sigma_e || a.sigma_o1 != c.sigma_o1 ||
       a.sigma_o2 != c.sigma_o2))
    return false;
  return a.lambda1 == c.lambda1 && a.lambda2 == c.lambda2 && a.mu == c.mu &&
         a.nltv_window == c.nltv_window && a.nltv_patch == c.nltv_patch && a.nltv_h == c.nltv_h &&
         a.cg_iters == c.cg_iters && a.cg_tol == c.cg_tol && a.precision == c.precision;
}

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
                   "patch and h, cg_iters, cg_tol, precision and the weight scheme with its "
                   "sigmas");
  lfsr_batch* b = new (std::nothrow) lfsr_batch();
  if (!b) return bfail(nullptr, LFSR_ENOMEM, "host allocation failed");
  b->stream = (cudaStream_t)cuda_stream;
  b->cg_iters = params[0].cg_iters;
  for (int j = 0; j < n; ++j) {
    lfsr_handle* h = nullptr;
    const int rc = create_handle(&params[j], cuda_stream, &h, false);
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
  const cudaError_t e = batch_assign(b, b->jobs);
  if (e != cudaSuccess) {
    const std::string msg = std::string("lfsr_batch_create: ") + cudaGetErrorString(e);
    const int code = e == cudaErrorMemoryAllocation ? LFSR_ENOMEM
                     : e == cudaErrorInvalidValue  ? LFSR_EUNSUPPORTED : LFSR_ECUDA;
    batch_free(b);
    delete b;
    return bfail(nullptr, code, e == cudaErrorInvalidValue
                                    ? std::string("disparity * angular offset too large for the "
                                                  "shared-memory tile")
                                    : msg);
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
  // Re-arm the batch's reduction counters and the persistent form's
  // barrier count.  Between launches they are zero (a multiple of the grid
  // for the barrier count) and this is a no-op; after an iteration whose
  // barrier wait ran out, CTAs that abandoned the work arrived at later
  // phases' counters while others were still in earlier ones, so a
  // counter's reset can have dropped an arrival.
  cudaError_t e = cudaSuccess;
  if (b->counters)
    e = cudaMemsetAsync(b->counters, 0, b->cap_counters * sizeof(unsigned int), b->stream);
  if (e == cudaSuccess && b->bar)
    e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned long long), b->stream);
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("batch load: ") + cudaGetErrorString(e));
  return LFSR_OK;
}

int lfsr_batch_iterate(lfsr_batch* b, int iterations) {
  NvtxRange range("lfsr_batch_iterate");
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (iterations < 0) return bfail(b, LFSR_EINVAL, "iterations must be >= 0");
  int left = iterations;
  cudaError_t e = cudaSuccess;
  if (b->profiling) {
    for (; left > 0 && e == cudaSuccess; --left) {
      e = batch_iteration(b, b->parity, b->stream, &b->prof);
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
  out->op_split_even = out->op_split_balanced = 0.0;   // the batch's ranges: its group's
  for (const Group& gr : b->groups)
    for (int m : gr.members)
      if (m == job) {
        out->op_split_even = gr.split[0];
        out->op_split_balanced = gr.split[1];
      }
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

int lfsr_batch_autotune(lfsr_batch* b) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  cudaError_t e = cudaSuccess;
  double t = 0.0;
  // operator tile side, group by group: the data block and the normal-matrix
  // launches of the group, timed on one iteration after one warm-up
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    Group& gr = b->groups[gi];
    int best = gr.tile;
    double best_ms = 1e300;
    for (int tile : {64, 32}) {
      if (set_tile(b, gr, tile) != cudaSuccess) continue;   // layout too large
      e = build_tables(b);
      double ms_data = 0.0, ms_norm = 0.0;
      if (e == cudaSuccess) e = time_iteration(b, KD_NORMAL, (int)gi, &t);
      if (e == cudaSuccess) e = time_iteration(b, KD_NORMAL, (int)gi, &ms_norm);
      if (e == cudaSuccess) e = time_iteration(b, KD_DATA, (int)gi, &ms_data);
      if (e == cudaSuccess && ms_norm + ms_data < best_ms) {   // per-iteration operator time
        best_ms = ms_norm + ms_data;
        best = tile;
      }
    }
    if (e == cudaSuccess && set_tile(b, gr, best) != cudaSuccess) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = build_tables(b);
  }
  // NLTV-apply direction chunk
  if (e == cudaSuccess) {
    int best = b->nla_chunk;
    double best_ms = 1e300;
    for (int chunk : {6, 3}) {
      b->nla_chunk = chunk;
      double ms = 0.0;
      e = time_iteration(b, KD_NLA, -1, &t);
      if (e == cudaSuccess) e = time_iteration(b, KD_NLA, -1, &ms);
      if (e != cudaSuccess) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = chunk;
      }
    }
    b->nla_chunk = best;
    if (e == cudaSuccess) e = build_tables(b);   // drops the graphs of the old shapes
  }
  // launch form: the per-phase launches against the persistent launch
  // (when a compiled instance fits the batch)
  if (e == cudaSuccess && b->persist_ok) {
    double ms[2] = {0.0, 0.0};
    for (int form : {LFSR_BATCH_PHASES, LFSR_BATCH_PERSISTENT}) {
      b->form = form;
      e = time_form(b, &ms[form]);
      if (e != cudaSuccess) break;
    }
    b->form = (e == cudaSuccess && ms[LFSR_BATCH_PERSISTENT] < ms[LFSR_BATCH_PHASES])
                  ? LFSR_BATCH_PERSISTENT
                  : LFSR_BATCH_PHASES;
    drop_graphs(b);
  }
  for (lfsr_handle* h : b->jobs) h->parity = b->parity;
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
  return LFSR_OK;
}

int lfsr_batch_tuning(const lfsr_batch* b, int* op_tile, int max_groups, int* nla_chunk) {
  if (!b) return 0;
  const int G = (int)b->groups.size();
  for (int gi = 0; gi < G && gi < max_groups && op_tile; ++gi) op_tile[gi] = b->groups[gi].tile;
  if (nla_chunk) *nla_chunk = b->nla_chunk;
  return G;
}

int lfsr_batch_set_tuning(lfsr_batch* b, const int* op_tile, int n_groups, int nla_chunk) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (nla_chunk != 6 && nla_chunk != 3) return bfail(b, LFSR_EINVAL, "nla_chunk must be 6 or 3");
  if (!op_tile || n_groups != (int)b->groups.size())
    return bfail(b, LFSR_EINVAL, "op_tile must hold one tile side per operator group");
  for (int gi = 0; gi < n_groups; ++gi)
    if (op_tile[gi] != 64 && op_tile[gi] != 32)
      return bfail(b, LFSR_EINVAL, "operator tile sides are 64 or 32");
  for (int gi = 0; gi < n_groups; ++gi) {   // every side fits before any group changes
    OpPlan P{};
    if (fast_plan_table(b->groups[gi].g, &P, b->smem_limit, op_tile[gi]) != cudaSuccess)
      return bfail(b, LFSR_EUNSUPPORTED, "tile side does not fit the shared memory");
  }
  for (int gi = 0; gi < n_groups; ++gi)
    if (set_tile(b, b->groups[gi], op_tile[gi]) != cudaSuccess)
      return bfail(b, LFSR_EUNSUPPORTED, "tile side does not fit the shared memory");
  b->nla_chunk = nla_chunk;
  const cudaError_t e = build_tables(b);
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("set tuning: ") + cudaGetErrorString(e));
  return LFSR_OK;
}

int lfsr_batch_launches_per_iteration(const lfsr_batch* b) {
  if (!b) return 0;
  if (b->form == LFSR_BATCH_PERSISTENT) return 1;
  const int G = (int)b->groups.size();
  return 2 + G + b->cg_iters * (2 + G);
}

int lfsr_batch_persistent_available(const lfsr_batch* b) { return b && b->persist_ok ? 1 : 0; }

int lfsr_batch_form(const lfsr_batch* b) { return b ? b->form : -1; }

int lfsr_batch_set_form(lfsr_batch* b, int form) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (form != LFSR_BATCH_PHASES && form != LFSR_BATCH_PERSISTENT)
    return bfail(b, LFSR_EINVAL, "form must be LFSR_BATCH_PHASES or LFSR_BATCH_PERSISTENT");
  if (form == LFSR_BATCH_PERSISTENT && !b->persist_ok)
    return bfail(b, LFSR_EUNSUPPORTED,
                 "no compiled persistent iteration fits this batch (operator groups, their tile "
                 "sides, the NLTV window and patch, the weight scheme or the storage kind)");
  const cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("set form: ") + cudaGetErrorString(e));
  b->form = form;
  drop_graphs(b);   // they hold the other form's launches
  return LFSR_OK;
}

int lfsr_batch_set_device_wait(lfsr_batch* b, int64_t limit_ns, int test_unreachable) {
  if (!b) return bfail(nullptr, LFSR_EINVAL, "batch is NULL");
  if (limit_ns < 0) return bfail(b, LFSR_EINVAL, "limit_ns must be >= 0");
  const cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess)
    return bfail(b, LFSR_ECUDA, std::string("set device wait: ") + cudaGetErrorString(e));
  b->wait_ns = (unsigned long long)limit_ns;
  b->wait_unreachable = test_unreachable ? 1 : 0;
  b->g.wait_ns = b->wait_ns;
  b->g.wait_unreachable = b->wait_unreachable;
  drop_graphs(b);   // the captured launches hold the old limit
  return LFSR_OK;
}

}  // extern "C"
