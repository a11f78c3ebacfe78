// Batch engine: many independent solves stepped together by persistent
// kernels over device-resident slot tables and work lists.
//
// Solves are grouped by (velocity set, N).  For each group the engine keeps a
// device table of the members' View structs and two work lists: element
// batches (slot, first element / EPB) for the element kernels and chunks of
// node groups (slot, chunk of kDssThreads) for the gather-scatter kernels.
// One time step of the whole batch is one replay of a CUDA graph in which each
// group is a branch of 14 persistent kernels (fixed grids sized by occupancy);
// the kernels read the member count from device memory, so members can join
// or leave between replays without re-capturing the graph (only a new group,
// a grown list or a new tile choice re-captures).  The kernels run the same
// body functions as the single-solve path, and their per-node arithmetic does
// not depend on how elements are batched into CTAs, so every solve gives the
// same bits alone and in any mix.
//
// Autotuning: elements per CTA (EPB) is chosen per group among up to three
// compiled tile shapes by timing a few real steps of each (every shape gives
// identical results, so tuning steps are ordinary steps of the solves).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "solver.cuh"

using namespace semlbm;

namespace {

struct GroupDev {
  const View* views;
  const WorkItem* elem;
  const WorkItem* node;
  const int* counts;   // [0] element items, [1] node items
};

struct GroupOps {
  int epb = 0, threads = 0;
  size_t sm_lap = 0, sm_force = 0, sm_rhs = 0;
  int grid_lap = 0, grid_force = 0, grid_rhs = 0, grid_node = 0;
  void (*step)(const GroupOps&, const GroupDev&, cudaStream_t, bool pdl) = nullptr;
};

template <class L, int NP, int EPB>
void group_step(const GroupOps& o, const GroupDev& d, cudaStream_t st, bool pdl) {
  constexpr int T = cta_threads<L::D, NP, EPB>();
  const int* ce = d.counts;
  const int* cn = d.counts + 1;
  // with pdl, every kernel after the first is a programmatic dependent launch
  // of the one before it on the group's stream
  launch(kb_lap<L, NP, EPB>, o.grid_lap, T, o.sm_lap, st, false, d.views, d.elem, ce);
  launch(kb_dss_mu<L>, o.grid_node, kDssThreads, 0, st, pdl, d.views, d.node, cn);
  launch(kb_force<L, NP, EPB>, o.grid_force, T, o.sm_force, st, pdl, d.views, d.elem, ce);
  launch(kb_dss_collide<L>, o.grid_node, kDssThreads, 0, st, pdl, d.views, d.node, cn);
  launch(kb_rhs<L, NP, EPB>, o.grid_rhs, T, o.sm_rhs, st, pdl, d.views, d.elem, ce, 1);
  launch(kb_dss_rk<L, 1>, o.grid_node, kDssThreads, 0, st, pdl, d.views, d.node, cn);
  for (int stage = 2; stage <= 3; ++stage) {
    launch(kb_lap<L, NP, EPB>, o.grid_lap, T, o.sm_lap, st, pdl, d.views, d.elem, ce);
    launch(kb_dss_mu<L>, o.grid_node, kDssThreads, 0, st, pdl, d.views, d.node, cn);
    launch(kb_rhs<L, NP, EPB>, o.grid_rhs, T, o.sm_rhs, st, pdl, d.views, d.elem, ce, 0);
    if (stage == 2)
      launch(kb_dss_rk<L, 2>, o.grid_node, kDssThreads, 0, st, pdl, d.views, d.node, cn);
    else
      launch(kb_dss_rk<L, 3>, o.grid_node, kDssThreads, 0, st, pdl, d.views, d.node, cn);
  }
}

template <class K>
int resident_grid(K kernel, int threads, size_t smem, int sms) {
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess)
    return 0;
  return nb * sms;
}

template <class L, int NP, int EPB>
void add_candidate(std::vector<GroupOps>& out, int sms) {
  for (const GroupOps& o : out)
    if (o.epb == EPB) return;
  constexpr int D = L::D, NL = ipow(NP, D), NT = EPB * NL;
  GroupOps o;
  o.epb = EPB;
  o.threads = cta_threads<D, NP, EPB>();
  o.sm_lap = (NP * NP + NT + D * NT) * sizeof(double);
  o.sm_force = (NP * NP + 2 * NT) * sizeof(double);
  o.sm_rhs = (NP * NP + 2 * NT + (L::Q - 1) * NT) * sizeof(double);
  if (o.sm_rhs > 227 * 1024) return;
  o.grid_lap = resident_grid(kb_lap<L, NP, EPB>, o.threads, o.sm_lap, sms);
  o.grid_force = resident_grid(kb_force<L, NP, EPB>, o.threads, o.sm_force, sms);
  o.grid_rhs = resident_grid(kb_rhs<L, NP, EPB>, o.threads, o.sm_rhs, sms);
  const int g1 = resident_grid(kb_dss_rk<L, 1>, kDssThreads, 0, sms);
  const int g2 = resident_grid(kb_dss_collide<L>, kDssThreads, 0, sms);
  o.grid_node = std::min(g1, g2);
  if (!o.grid_lap || !o.grid_force || !o.grid_rhs || !o.grid_node) return;
  o.step = group_step<L, NP, EPB>;
  out.push_back(o);
}

// tile candidates: half, the default and twice the default elements per CTA
template <class L, int NP>
std::vector<GroupOps> candidates(int sms) {
  constexpr int NL = ipow(NP, L::D);
  constexpr int base = NL >= 256 ? 1 : 256 / NL;
  constexpr int lo = base / 2 > 0 ? base / 2 : 1;
  constexpr int cap = 1024 / NL > 0 ? 1024 / NL : 1;
  constexpr int hi = 2 * base < cap ? 2 * base : cap;
  std::vector<GroupOps> out;
  add_candidate<L, NP, base>(out, sms);   // default first
  add_candidate<L, NP, lo>(out, sms);
  add_candidate<L, NP, hi>(out, sms);
  return out;
}

template <class L, int... Ns>
std::vector<GroupOps> pick_candidates(int N, int sms, std::integer_sequence<int, Ns...>) {
  std::vector<GroupOps> out;
  ((N + 1 == Ns + 3 ? (out = candidates<L, Ns + 3>(sms), 0) : 0), ...);
  return out;
}

constexpr int kBatchMaxN = 8;   // batched kernels are compiled for N = 2..8

std::vector<GroupOps> group_candidates(sem_lbm_lattice lat, int N, int sms) {
  switch (lat) {
    case SEMLBM_D2Q9: return pick_candidates<D2Q9>(N, sms, std::make_integer_sequence<int, 7>{});
    case SEMLBM_D3Q13: return pick_candidates<D3Q13>(N, sms, std::make_integer_sequence<int, 7>{});
    case SEMLBM_D3Q19: return pick_candidates<D3Q19>(N, sms, std::make_integer_sequence<int, 7>{});
    case SEMLBM_D3Q27: return pick_candidates<D3Q27>(N, sms, std::make_integer_sequence<int, 7>{});
  }
  return {};
}

// tuned choices of this process: (lattice, N, log2 of the group's element count) -> EPB
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, int> g_tuned;

int size_bucket(int64_t elems) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= elems) ++b;
  return b;
}

}  // namespace

struct BatchGroup {
  sem_lbm_lattice lat;
  int N;
  std::vector<GroupOps> cands;
  int choice = 0;
  double tuned_ms[4] = {0, 0, 0, 0};
  std::vector<int> members;          // batch slots, in device-table order
  std::vector<View> h_views;
  std::vector<WorkItem> h_elem, h_node;
  int h_counts[2] = {0, 0};
  View* d_views = nullptr;
  WorkItem* d_elem = nullptr;
  WorkItem* d_node = nullptr;
  int* d_counts = nullptr;
  size_t cap_views = 0, cap_elem = 0, cap_node = 0;
  cudaStream_t branch = nullptr;
  cudaEvent_t join = nullptr;
  int64_t elems = 0;
};

struct sem_lbm_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sms = 0;
  std::vector<sem_lbm*> slots;
  std::vector<BatchGroup*> groups;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t fork = nullptr;
  int capture_failures = 0;   // steps that ran as direct launches instead
};

namespace {

void free_group(BatchGroup* g) {
  if (g->d_views) cudaFree(g->d_views);
  if (g->d_elem) cudaFree(g->d_elem);
  if (g->d_node) cudaFree(g->d_node);
  if (g->d_counts) cudaFree(g->d_counts);
  if (g->branch) cudaStreamDestroy(g->branch);
  if (g->join) cudaEventDestroy(g->join);
  delete g;
}

template <class T>
int ensure(T** p, size_t* cap, size_t need, bool* moved) {
  if (need <= *cap && *p) return 0;
  size_t n = std::max<size_t>(need, 2 * *cap);
  n = std::max<size_t>(n, 16);
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    *cap = 0;
    return fail(SEMLBM_ENOMEM, "batch work-list allocation of %zu bytes failed", n * sizeof(T));
  }
  *cap = n;
  *moved = true;
  return 0;
}

// rebuild and upload a group's view table and work lists for its current EPB
int refresh_group(sem_lbm_batch* b, BatchGroup* g) {
  const GroupOps& o = g->cands[g->choice];
  g->h_views.clear();
  g->h_elem.clear();
  g->h_node.clear();
  g->elems = 0;
  for (size_t i = 0; i < g->members.size(); ++i) {
    const sem_lbm* s = b->slots[g->members[i]];
    g->h_views.push_back(s->view);
    for (int64_t e = 0; e * o.epb < s->E; ++e) g->h_elem.push_back({(int)i, (int)e});
    for (int64_t c = 0; c * kDssThreads < s->G; ++c) g->h_node.push_back({(int)i, (int)c});
    g->elems += s->E;
  }
  g->h_counts[0] = (int)g->h_elem.size();
  g->h_counts[1] = (int)g->h_node.size();
  bool moved = false;
  if (int rc = ensure(&g->d_views, &g->cap_views, g->h_views.size(), &moved)) return rc;
  if (int rc = ensure(&g->d_elem, &g->cap_elem, g->h_elem.size(), &moved)) return rc;
  if (int rc = ensure(&g->d_node, &g->cap_node, g->h_node.size(), &moved)) return rc;
  if (!g->d_counts) {
    if (cudaMalloc((void**)&g->d_counts, 2 * sizeof(int)) != cudaSuccess)
      return fail(SEMLBM_ENOMEM, "batch counter allocation failed");
    moved = true;
  }
  if (moved) b->dirty = true;
  cudaStream_t st = b->stream;
  if (!g->h_views.empty())
    CUDA_TRY(cudaMemcpyAsync(g->d_views, g->h_views.data(), g->h_views.size() * sizeof(View),
                             cudaMemcpyHostToDevice, st));
  if (!g->h_elem.empty())
    CUDA_TRY(cudaMemcpyAsync(g->d_elem, g->h_elem.data(), g->h_elem.size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, st));
  if (!g->h_node.empty())
    CUDA_TRY(cudaMemcpyAsync(g->d_node, g->h_node.data(), g->h_node.size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(g->d_counts, g->h_counts, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
  // the host vectors are pageable (the CUDA runtime stages them), but keep ordering simple:
  CUDA_TRY(cudaStreamSynchronize(st));
  return 0;
}

GroupDev dev_of(const BatchGroup* g) { return GroupDev{g->d_views, g->d_elem, g->d_node, g->d_counts}; }

int capture(sem_lbm_batch* b, bool pdl) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t gr;
  // relaxed: other host threads (e.g. a server building the next solves) may
  // allocate or launch on their own streams meanwhile
  CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (BatchGroup* g : b->groups) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->branch, b->fork, 0);
    if (e == cudaSuccess) g->cands[g->choice].step(g->cands[g->choice], dev_of(g), g->branch, pdl);
    if (e == cudaSuccess) e = cudaEventRecord(g->join, g->branch);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, g->join, 0);
  }
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
  if (e != cudaSuccess) return fail(SEMLBM_ECUDA, "batch capture: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(SEMLBM_ECUDA, "batch capture: %s", cudaGetErrorString(e2));
  const cudaError_t e3 = cudaGraphInstantiate(&b->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e3 != cudaSuccess) {
    b->graph = nullptr;
    return fail(SEMLBM_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e3));
  }
  b->dirty = false;
  return 0;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int sem_lbm_batch_create(void* stream, sem_lbm_batch_t** out) {
  if (!out) return fail(SEMLBM_EINVAL, "out is NULL");
  *out = nullptr;
  sem_lbm_batch* b = new (std::nothrow) sem_lbm_batch();
  if (!b) return fail(SEMLBM_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    delete b;
    return fail(SEMLBM_ECUDA, "no CUDA device");
  }
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(SEMLBM_ECUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    sem_lbm_batch_destroy(b);
    return fail(SEMLBM_ECUDA, "cudaEventCreate failed");
  }
  *out = b;
  return 0;
}

int sem_lbm_batch_add(sem_lbm_batch_t* b, sem_lbm_t* s, int* slot) {
  if (!b || !s) return fail(SEMLBM_EINVAL, "NULL argument");
  if (s->batch) return fail(SEMLBM_EINVAL, "solver already belongs to a batch");
  if (!s->state_ready) return fail(SEMLBM_EINVAL, "solver state not set");
  if (s->device != b->device) return fail(SEMLBM_EINVAL, "solver and batch are on different devices");
  DeviceGuard dg(b->device);
  if (s->N > kBatchMaxN) return fail(SEMLBM_EUNSUPPORTED, "batched kernels are built for N <= %d", kBatchMaxN);
  BatchGroup* g = nullptr;
  for (BatchGroup* x : b->groups)
    if (x->lat == s->lat && x->N == s->N) g = x;
  if (!g) {
    g = new (std::nothrow) BatchGroup();
    if (!g) return fail(SEMLBM_ENOMEM, "host allocation failed");
    g->lat = s->lat;
    g->N = s->N;
    g->cands = group_candidates(s->lat, s->N, b->sms);
    if (g->cands.empty()) {
      delete g;
      return fail(SEMLBM_EUNSUPPORTED, "no launchable tile for N = %d", s->N);
    }
    if (cudaStreamCreateWithFlags(&g->branch, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->join, cudaEventDisableTiming) != cudaSuccess) {
      free_group(g);
      return fail(SEMLBM_ECUDA, "stream/event creation failed");
    }
    b->groups.push_back(g);
    b->dirty = true;
  }
  // the solver's pending work completes before the batch takes over
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  int id = -1;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i]) id = (int)i;
  if (id < 0) {
    id = (int)b->slots.size();
    b->slots.push_back(nullptr);
  }
  b->slots[id] = s;
  s->batch = b;
  s->home_stream = s->stream;
  s->stream = b->stream;
  g->members.push_back(id);
  {  // a tuned tile for groups of this shape, if one is known
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    int64_t elems = 0;
    for (int m : g->members) elems += b->slots[m]->E;
    auto it = g_tuned.find({(int)g->lat, g->N, size_bucket(elems)});
    if (it != g_tuned.end())
      for (size_t c = 0; c < g->cands.size(); ++c)
        if (g->cands[c].epb == it->second && (int)c != g->choice) {
          g->choice = (int)c;
          b->dirty = true;
        }
  }
  if (int rc = refresh_group(b, g)) return rc;
  if (slot) *slot = id;
  return 0;
}

int sem_lbm_batch_remove(sem_lbm_batch_t* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot])
    return fail(SEMLBM_EINVAL, "no solver in slot %d", slot);
  DeviceGuard dg(b->device);
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  sem_lbm* s = b->slots[slot];
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    BatchGroup* g = b->groups[gi];
    auto it = std::find(g->members.begin(), g->members.end(), slot);
    if (it == g->members.end()) continue;
    g->members.erase(it);
    if (g->members.empty()) {
      free_group(g);
      b->groups.erase(b->groups.begin() + gi);
      b->dirty = true;
    } else if (int rc = refresh_group(b, g)) {
      return rc;
    }
    break;
  }
  b->slots[slot] = nullptr;
  s->stream = s->home_stream;
  s->batch = nullptr;
  return 0;
}

int sem_lbm_batch_step(sem_lbm_batch_t* b, int64_t n_steps) {
  if (!b) return fail(SEMLBM_EINVAL, "NULL batch");
  DeviceGuard dg(b->device);
  if (n_steps < 0) return fail(SEMLBM_EINVAL, "n_steps must be >= 0");
  if (b->groups.empty() || n_steps == 0) return 0;
  if (b->dirty || !b->graph) {
    // programmatic edges between each group's kernels first, else plain edges
    int rc = capture(b, true);
    if (rc != 0) {
      cudaGetLastError();
      rc = capture(b, false);
    }
    if (rc != 0) {
      // a capture that failed leaves no graph: run these steps as direct
      // launches of the same kernels (same results) and capture next time
      cudaGetLastError();
      ++b->capture_failures;
      for (int64_t i = 0; i < n_steps; ++i)
        for (BatchGroup* g : b->groups)
          g->cands[g->choice].step(g->cands[g->choice], dev_of(g), b->stream, false);
      CUDA_TRY(cudaGetLastError());
      for (sem_lbm* s : b->slots)
        if (s) s->step += n_steps;
      return 0;
    }
  }
  for (int64_t i = 0; i < n_steps; ++i) CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
  for (sem_lbm* s : b->slots)
    if (s) s->step += n_steps;
  return 0;
}

int sem_lbm_batch_tune(sem_lbm_batch_t* b, int steps_per_candidate) {
  if (!b) return fail(SEMLBM_EINVAL, "NULL batch");
  DeviceGuard dg(b->device);
  if (steps_per_candidate < 2) return fail(SEMLBM_EINVAL, "steps_per_candidate must be >= 2");
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int rc = 0;
  for (BatchGroup* g : b->groups) {
    double best = 1e300;
    int best_c = g->choice;
    for (size_t c = 0; c < g->cands.size() && rc == 0; ++c) {
      g->choice = (int)c;
      if ((rc = refresh_group(b, g))) break;
      const GroupOps& o = g->cands[c];
      // a warm-up step, drained before timing (first launches can load modules
      // and stall), then the best of two timed runs of steps_per_candidate - 1
      o.step(o, dev_of(g), b->stream, false);
      if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        rc = fail(SEMLBM_ECUDA, "tuning step failed: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      double per = 1e300;
      for (int rep = 0; rep < 2 && rc == 0; ++rep) {
        cudaEventRecord(e0, b->stream);
        for (int k = 1; k < steps_per_candidate; ++k) o.step(o, dev_of(g), b->stream, false);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = fail(SEMLBM_ECUDA, "tuning step failed: %s", cudaGetErrorString(cudaGetLastError()));
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        per = std::min(per, (double)ms / (steps_per_candidate - 1));
      }
      if (rc) break;
      if (c < 4) g->tuned_ms[c] = per;
      if (per < best) {
        best = per;
        best_c = (int)c;
      }
      for (int m : g->members) b->slots[m]->step += 2 * steps_per_candidate - 1;
    }
    if (rc) break;
    g->choice = best_c;
    if ((rc = refresh_group(b, g))) break;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[{(int)g->lat, g->N, size_bucket(g->elems)}] = g->cands[best_c].epb;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->dirty = true;
  return rc;
}

int sem_lbm_batch_diagnostics(sem_lbm_batch_t* b, sem_lbm_diag* out, int n) {
  if (!b || (!out && n > 0)) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(b->device);
  std::vector<DiagPart> parts(n);
  std::vector<int> flags(2 * n, 0);
  for (int i = 0; i < n; ++i) {
    if (i >= (int)b->slots.size() || !b->slots[i]) continue;
    sem_lbm* s = b->slots[i];
    s->ops->diag(*s);
    CUDA_TRY(cudaMemcpyAsync(&parts[i], s->dout, sizeof(DiagPart), cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaMemcpyAsync(&flags[2 * i], s->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < n; ++i) {
    sem_lbm_diag& d = out[i];
    memset(&d, 0, sizeof d);
    if (i >= (int)b->slots.size() || !b->slots[i]) {
      d.step = -1;
      d.status = SEMLBM_EINVAL;
      continue;
    }
    const sem_lbm* s = b->slots[i];
    const DiagPart& p = parts[i];
    d.step = s->step;
    d.time = s->step * s->dt;
    d.mass = p.mass;
    d.ke_max = p.ke_max;
    d.ke_int = p.ke_int;
    d.umax = std::sqrt(p.u2max);
    d.rho_min = p.rho_min;
    d.rho_max = p.rho_max;
    d.n_nonfinite = (int64_t)p.nonfinite;
    d.status = (p.nonfinite > 0 || flags[2 * i + 1]) ? SEMLBM_ENONFINITE : SEMLBM_OK;
  }
  return 0;
}

int sem_lbm_batch_info(sem_lbm_batch_t* b, sem_lbm_batch_group_info* out, int max_groups,
                       int* n_groups) {
  if (!b) return fail(SEMLBM_EINVAL, "NULL batch");
  if (n_groups) *n_groups = (int)b->groups.size();
  for (int i = 0; i < max_groups && i < (int)b->groups.size(); ++i) {
    const BatchGroup* g = b->groups[i];
    sem_lbm_batch_group_info& o = out[i];
    memset(&o, 0, sizeof o);
    o.lattice = (int)g->lat;
    o.N = g->N;
    o.n_members = (int)g->members.size();
    o.epb = g->cands[g->choice].epb;
    o.elem_items = g->h_counts[0];
    o.node_items = g->h_counts[1];
    o.grid_elem = g->cands[g->choice].grid_rhs;
    o.grid_node = g->cands[g->choice].grid_node;
    o.capture_failures = b->capture_failures;
    o.n_candidates = (int)std::min<size_t>(g->cands.size(), 4);
    for (int c = 0; c < o.n_candidates; ++c) {
      o.candidate_epb[c] = g->cands[c].epb;
      o.candidate_ms[c] = g->tuned_ms[c];
    }
  }
  return 0;
}

void sem_lbm_batch_destroy(sem_lbm_batch_t* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (b->slots[i]) sem_lbm_batch_remove(b, (int)i);
  for (BatchGroup* g : b->groups) free_group(g);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

void* sem_lbm_batch_stream(const sem_lbm_batch_t* b) { return b ? (void*)b->stream : nullptr; }

int sem_lbm_batch_slot_of(const sem_lbm_t* s) {
  if (!s || !s->batch) return -1;
  for (size_t i = 0; i < s->batch->slots.size(); ++i)
    if (s->batch->slots[i] == s) return (int)i;
  return -1;
}

}  // extern "C"
