// Host side of libsemlbm: setup tables, gather-scatter map, wall records,
// workspace layout, kernel dispatch and the C ABI declared in sem_lbm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "solver.cuh"

using namespace semlbm;

namespace semlbm {
thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
}  // namespace semlbm

namespace {

// ---------------------------------------------------------------------------
// GLL tables in long double.  Nodes: Newton on P_{N+1} - P_{N-1}, whose zeros
// are +-1 and the zeros of P_N' and whose derivative is (2N+1) P_N.  Weights
// 2 / (N(N+1) P_N(x)^2).  Derivative matrix: the GLL closed form
// D_ij = P_N(x_i) / (P_N(x_j)(x_i - x_j)), D_00 = -N(N+1)/4, D_NN = N(N+1)/4.
// ---------------------------------------------------------------------------
void legendre_ld(int n, long double x, long double* p) {  // p[0..n]
  p[0] = 1.0L;
  if (n >= 1) p[1] = x;
  for (int k = 1; k < n; ++k) p[k + 1] = ((2 * k + 1) * x * p[k] - k * p[k - 1]) / (k + 1);
}

void gll_tables(int N, std::vector<double>& x, std::vector<double>& w, std::vector<double>& D) {
  const int n = N + 1;
  std::vector<long double> xl(n), pN(n), p(N + 2);
  for (int j = 0; j < n; ++j) {
    long double xj = -cosl(3.14159265358979323846264338327950288L * j / N);
    if (j > 0 && j < N) {
      for (int it = 0; it < 100; ++it) {
        legendre_ld(N + 1, xj, p.data());
        const long double f = p[N + 1] - p[N - 1];
        const long double df = (2 * N + 1) * p[N];
        const long double dx = f / df;
        xj -= dx;
        if (fabsl(dx) < 1e-30L) break;
      }
    }
    xl[j] = xj;
    legendre_ld(N, xj, p.data());
    pN[j] = p[N];
  }
  x.resize(n);
  w.resize(n);
  D.assign(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    x[j] = (double)xl[j];
    w[j] = (double)(2.0L / ((long double)N * (N + 1) * pN[j] * pN[j]));
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      long double v;
      if (i != j) v = pN[i] / (pN[j] * (xl[i] - xl[j]));
      else if (i == 0) v = -(long double)N * (N + 1) / 4;
      else if (i == N) v = (long double)N * (N + 1) / 4;
      else v = 0.0L;
      D[i * n + j] = (double)v;
    }
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct HostMaps {
  std::vector<int> off, idx;          // gather-scatter CSR (group order: see build_maps)
  std::vector<int> slot;              // [V] wall record or -1
  std::vector<int> rec_elem, rec_node, rec_mask;
  std::vector<double> rec_cos;        // [R][2D]
  std::vector<int> rec_tag;           // [R][2D] wall tag of each face (-1 if not a wall face)
  std::vector<double> rec_ub;         // [R][2D][D] wall velocity of each face (moving walls)
  bool moving = false;
  int64_t G = 0;
};

int build_maps(const sem_lbm_mesh* m, int N, double theta_w, const sem_lbm_params* p,
               HostMaps& h) {
  const int D = m->dim, n = N + 1;
  int NL = 1;
  for (int a = 0; a < D; ++a) NL *= n;
  const int64_t E = m->n_elem, V = E * NL;
  // gather-scatter groups: sort (global id, local index)
  std::vector<std::pair<int64_t, int>> key(V);
  for (int64_t i = 0; i < V; ++i) key[i] = {m->global_id[i], (int)i};
  std::sort(key.begin(), key.end());
  // group order: by the element that holds the first copy (consecutive
  // gather-scatter threads touch nearby memory), then by copy count within that
  // element, then by first copy.  The threads of a warp loop over as many copies
  // as the warp's largest group, so a warp that mixes a hex vertex's 8 copies
  // with interior nodes' 1 idles most of its lanes; sorting by count within the
  // element cuts the lanes' idle iterations by a third on hex meshes.  Sorting
  // over windows of several elements cut them further but lost locality, and
  // slowed the 2D cylinder's graph.  Each group's copies stay in ascending local
  // index, so the order only decides which thread handles a group, never the
  // order of a sum.
  std::vector<std::tuple<int64_t, int, int, int>> grp;   // (element, copies, first, start)
  for (int64_t i = 0; i < V;) {
    int64_t j = i + 1;
    while (j < V && key[j].first == key[i].first) ++j;
    grp.push_back({key[i].second / NL, (int)(j - i), key[i].second, (int)i});
    i = j;
  }
  std::sort(grp.begin(), grp.end());
  h.G = (int64_t)grp.size();
  h.off.resize(h.G + 1);
  h.idx.resize(V);
  int pos = 0;
  for (int64_t g = 0; g < h.G; ++g) {
    h.off[g] = pos;
    const int start = std::get<3>(grp[g]);
    for (int64_t i = start; i < V && key[i].first == key[start].first; ++i)
      h.idx[pos++] = key[i].second;
  }
  h.off[h.G] = pos;
  // wall records: one per element-local node that lies on a wall face
  auto cos_of = [&](int tag, double* c) -> int {
    if (tag < 0) { *c = 0.0; return 0; }
    if (tag == 0) { *c = std::cos(theta_w); return 0; }
    if (!p || tag > p->n_tags || !p->theta_tag)
      return fail(SEMLBM_EINVAL, "wall tag %d has no contact angle (n_tags = %d)", tag,
                  p ? p->n_tags : 0);
    *c = std::cos(p->theta_tag[tag - 1]);
    return 0;
  };
  h.slot.assign(V, -1);
  std::vector<int> mask(NL);
  std::vector<double> cosf(2 * D), ubf(2 * D * D);
  auto ub_of = [&](int tag, double* u) {   // velocity of the walls with this tag
    for (int c = 0; c < D; ++c)
      u[c] = (tag >= 0 && p && p->wall_velocity && tag <= p->n_tags) ? p->wall_velocity[tag * D + c] : 0.0;
  };
  for (int64_t e = 0; e < E; ++e) {
    bool any = false;
    for (int f = 0; f < 2 * D; ++f) {
      const uint8_t k = m->face_kind[e * 2 * D + f];
      if (k > 1) return fail(SEMLBM_EINVAL, "face_kind must be 0 or 1 (element %lld)", (long long)e);
      if (k == 1) {
        any = true;
        if (int rc = cos_of(m->face_tag[e * 2 * D + f], &cosf[f])) return rc;
        ub_of(m->face_tag[e * 2 * D + f], &ubf[f * D]);
        for (int c = 0; c < D; ++c) h.moving = h.moving || ubf[f * D + c] != 0.0;
      } else {
        cosf[f] = 0.0;
        for (int c = 0; c < D; ++c) ubf[f * D + c] = 0.0;
      }
    }
    if (!any) continue;
    std::fill(mask.begin(), mask.end(), 0);
    for (int f = 0; f < 2 * D; ++f) {
      if (m->face_kind[e * 2 * D + f] != 1) continue;
      const int b = f >> 1, side = (f & 1) ? N : 0;
      for (int k = 0; k < NL; ++k) {
        const int ib = (b == 0) ? k % n : (b == 1 ? (k / n) % n : k / (n * n));
        if (ib == side) mask[k] |= 1 << f;
      }
    }
    for (int k = 0; k < NL; ++k) {
      if (!mask[k]) continue;
      h.slot[e * NL + k] = (int)h.rec_elem.size();
      h.rec_elem.push_back((int)e);
      h.rec_node.push_back(k);
      h.rec_mask.push_back(mask[k]);
      for (int f = 0; f < 2 * D; ++f) h.rec_cos.push_back(cosf[f]);
      for (int f = 0; f < 2 * D; ++f)
        h.rec_tag.push_back(m->face_kind[e * 2 * D + f] == 1 ? m->face_tag[e * 2 * D + f] : -1);
      h.rec_ub.insert(h.rec_ub.end(), ubf.begin(), ubf.end());
    }
  }
  return 0;
}

double min_spacing(const sem_lbm_mesh* m, int N) {
  const int D = m->dim, n = N + 1;
  int NL = 1;
  for (int a = 0; a < D; ++a) NL *= n;
  const int stride[3] = {1, n, n * n};
  double h2 = INFINITY;
  for (int64_t e = 0; e < m->n_elem; ++e)
    for (int k = 0; k < NL; ++k)
      for (int b = 0; b < D; ++b) {
        const int ib = (b == 0) ? k % n : (b == 1 ? (k / n) % n : k / (n * n));
        if (ib == N) continue;
        const double* x0 = m->node_xyz + (e * NL + k) * D;
        const double* x1 = m->node_xyz + (e * NL + k + stride[b]) * D;
        double s = 0.0;
        for (int a = 0; a < D; ++a) s += (x1[a] - x0[a]) * (x1[a] - x0[a]);
        h2 = std::min(h2, s);
      }
  return std::sqrt(h2);
}

int q_of(sem_lbm_lattice lat) {
  switch (lat) {
    case SEMLBM_D2Q9: return 9;
    case SEMLBM_D3Q13: return 13;
    case SEMLBM_D3Q19: return 19;
    case SEMLBM_D3Q27: return 27;
  }
  return 0;
}

double speed_max(sem_lbm_lattice lat) {
  switch (lat) {
    case SEMLBM_D2Q9: return D2Q9::SPEED_MAX;
    case SEMLBM_D3Q13: return D3Q13::SPEED_MAX;
    case SEMLBM_D3Q19: return D3Q19::SPEED_MAX;
    case SEMLBM_D3Q27: return D3Q27::SPEED_MAX;
  }
  return 1.0;
}

int validate(const sem_lbm_mesh* m, int N, sem_lbm_lattice lat) {
  if (!m) return fail(SEMLBM_EINVAL, "mesh is NULL");
  if (m->dim != 2 && m->dim != 3) return fail(SEMLBM_EINVAL, "dim must be 2 or 3");
  if (q_of(lat) == 0) return fail(SEMLBM_EUNSUPPORTED, "unknown lattice %d", (int)lat);
  if ((lat == SEMLBM_D2Q9) != (m->dim == 2))
    return fail(SEMLBM_EINVAL, "lattice does not match the mesh dimension");
  const int nmax = (m->dim == 2) ? 16 : 8;
  if (N < 2 || N > nmax) return fail(SEMLBM_EUNSUPPORTED, "N = %d not built (2..%d)", N, nmax);
  if (m->n_elem <= 0) return fail(SEMLBM_EINVAL, "n_elem must be positive");
  if (!m->node_xyz || !m->global_id || !m->face_kind || !m->face_tag)
    return fail(SEMLBM_EINVAL, "mesh array pointer is NULL");
  int NL = 1;
  for (int a = 0; a < m->dim; ++a) NL *= N + 1;
  if (m->n_elem > (int64_t)(INT32_MAX / 16) / NL) return fail(SEMLBM_EINVAL, "mesh too large");
  return 0;
}

// workspace carving
struct Carve {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align_up(count * sizeof(T));
    return p;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
namespace {

template <class L, int NP>
struct Impl {
  static constexpr int D = L::D, NL = ipow(NP, D);
  static constexpr int EPB = (NL >= 256) ? 1 : 256 / NL;
  static constexpr int NT = EPB * NL;
  static constexpr int THREADS = ((NT + 31) / 32) * 32;
  static constexpr size_t SM_LAP = (NP * NP + NT + D * NT) * sizeof(double);
  static constexpr size_t SM_FORCE = (NP * NP + 2 * NT) * sizeof(double);
  static constexpr size_t SM_RHS = (NP * NP + 2 * NT + (L::Q - 1) * NT) * sizeof(double);
  static constexpr size_t SM_GEOM = (NP * NP + D * NT) * sizeof(double);

  static int blocks(const sem_lbm& s) { return (int)((s.E + EPB - 1) / EPB); }

  static int prepare() {
    // opt in to large dynamic shared memory where a tile needs it
    if (SM_RHS > 48 * 1024)
      if (cudaFuncSetAttribute(k_rhs<L, NP, EPB, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_RHS) != cudaSuccess ||
          cudaFuncSetAttribute(k_rhs<L, NP, EPB, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_RHS) != cudaSuccess)
        return -1;
    if (SM_LAP > 48 * 1024)
      if (cudaFuncSetAttribute(k_lap<L, NP, EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SM_LAP) != cudaSuccess)
        return -1;
    return 0;
  }
  static void geom(sem_lbm& s) {
    k_geom<D, NP, EPB><<<blocks(s), THREADS, SM_GEOM, s.stream>>>(s.xyz, s.Dm, s.wg, L::S, s.MJ,
                                                                  s.Gm, s.Me, s.flags, s.V,
                                                                  (int)s.E);
    k_dss_mass<<<grid_of(s.G, kDssThreads), kDssThreads, 0, s.stream>>>(s.off, s.idx, (int)s.G,
                                                                        s.Me, s.invMg);
    if constexpr (L::PAIR_METRIC)
      k_pair_metric<L><<<grid_of(s.V, 256), 256, 0, s.stream>>>(s.MJ, s.CJ, s.V);
  }
  static void wallsetup(sem_lbm& s) {
    if (s.R == 0) return;
    k_wall_setup<L, NP><<<grid_of(s.R, 128), 128, 0, s.stream>>>(
        s.xyz, s.Dm, s.wg, s.rec_elem, s.rec_node, s.rec_cos, s.rec_mask, (int)s.R,
        std::sqrt(2.0 * s.beta / s.kappa), s.moving ? s.rec_ub : nullptr, s.wet, s.ae,
        s.moving ? s.wub : nullptr, s.wsf);
  }
  static void lap(sem_lbm& s) {
    launch(k_lap<L, NP, EPB>, blocks(s), THREADS, SM_LAP, s.stream, s.pdl, s.view, s.rho, s.lapr,
           s.drho);
  }
  static void mu(sem_lbm& s) {
    launch(k_dss_mu, grid_of(s.G, kDssThreads), kDssThreads, 0, s.stream, s.pdl, s.view, s.lapr,
           s.rho, s.mu);
  }
  static void force(sem_lbm& s) {
    launch(k_force<L, NP, EPB>, blocks(s), THREADS, SM_FORCE, s.stream, s.pdl, s.view);
  }
  static void collide(sem_lbm& s) {
    launch(k_dss_collide<L>, grid_of(s.G, kDssThreads), kDssThreads, 0, s.stream, s.pdl, s.view);
  }
  // small meshes: split the velocity pairs over up to NREP CTAs per element
  // batch until the grid reaches two CTAs per SM (1 = the unsplit kernel)
  static int rhs_split(const sem_lbm& s) {
    const int nb = blocks(s);
    int P = 1;
    while (P < L::NREP && (int64_t)nb * P < 2 * (int64_t)s.n_sm) ++P;
    return P;
  }
  static void rhs(sem_lbm& s, const double* gst) {
    const int nb = blocks(s);
    const int P = rhs_split(s);
    if (P == 1)
      launch(k_rhs<L, NP, EPB, false>, nb, THREADS, SM_RHS, s.stream, s.pdl, s.view, gst);
    else
      launch(k_rhs<L, NP, EPB, true>, dim3(nb, P), THREADS, SM_RHS, s.stream, s.pdl, s.view, gst);
  }
  static void rk(sem_lbm& s, int stage, const double* gcur, double* out) {
    const int gr = grid_of(s.G, kDssThreads);
    if (stage == 1)
      launch(k_dss_rk<L, 1>, gr, kDssThreads, 0, s.stream, s.pdl, s.view, gcur, out);
    else if (stage == 2)
      launch(k_dss_rk<L, 2>, gr, kDssThreads, 0, s.stream, s.pdl, s.view, gcur, out);
    else
      launch(k_dss_rk<L, 3>, gr, kDssThreads, 0, s.stream, s.pdl, s.view, gcur, out);
  }
  static void diag(sem_lbm& s) {
    k_diag<L><<<s.diag_blocks, 256, 0, s.stream>>>(s.f, s.Me, s.parts, s.V);
    k_diag_final<<<1, kCombineThreads, 0, s.stream>>>(s.parts, s.diag_blocks, s.dout);
  }
  static void wet(sem_lbm& s, int tag, double rv, double rl) {
    k_wet<L><<<s.diag_blocks, 256, 0, s.stream>>>(
        s.f, s.Me, s.xyz, s.rec_elem, s.rec_node, s.rec_mask, s.rec_tag, s.wsf, (int)s.R, tag,
        (int)s.NL, rv, 1.0 / (rl - rv), s.wparts, s.V);
    k_wet_final<<<1, kCombineThreads, 0, s.stream>>>(s.wparts, s.diag_blocks, s.wout);
  }
  static void init(sem_lbm& s, const double* rho_in) {
    k_init<L><<<grid_of(s.V, 256), 256, 0, s.stream>>>(rho_in, s.f, s.rho, s.V);
  }
  static void density(sem_lbm& s) {
    k_density<L><<<grid_of(s.V, 256), 256, 0, s.stream>>>(s.f, s.rho, s.V);
  }
  static void velocity(sem_lbm& s, double* u) {
    k_velocity<L><<<grid_of(s.V, 256), 256, 0, s.stream>>>(s.f, u, s.V);
  }
  static void lap_into(sem_lbm& s, const double* rho_in, double* partial) {
    k_lap<L, NP, EPB><<<blocks(s), THREADS, SM_LAP, s.stream>>>(s.view, rho_in, partial, nullptr);
  }
  static void mu_from(sem_lbm& s, const double* partial, const double* rho_in, double* mu_out) {
    k_dss_mu<<<grid_of(s.G, kDssThreads), kDssThreads, 0, s.stream>>>(s.view, partial, rho_in,
                                                                      mu_out);
  }
  static Ops* ops() {
    static Ops o{geom, wallsetup, lap, mu, force, rhs, collide, rk, diag, init, density, velocity, prepare,
                 lap_into, mu_from, wet, rhs_split, EPB};
    return &o;
  }
};

template <class L, int... Ns>
Ops* pick(int N, std::integer_sequence<int, Ns...>) {
  Ops* out = nullptr;
  ((N + 1 == Ns + 3 ? (out = Impl<L, Ns + 3>::ops(), 0) : 0), ...);
  return out;
}

Ops* select_ops(sem_lbm_lattice lat, int N) {
  switch (lat) {
    case SEMLBM_D2Q9: return pick<D2Q9>(N, std::make_integer_sequence<int, 15>{});   // n = 3..17
    case SEMLBM_D3Q13: return pick<D3Q13>(N, std::make_integer_sequence<int, 7>{});  // n = 3..9
    case SEMLBM_D3Q19: return pick<D3Q19>(N, std::make_integer_sequence<int, 7>{});
    case SEMLBM_D3Q27: return pick<D3Q27>(N, std::make_integer_sequence<int, 7>{});
  }
  return nullptr;
}

enum { K_LAP = 0, K_MU, K_FORCE, K_COLLIDE, K_RHS, K_RK };

// profiling hook: an event after each launch when per-kernel timing is on
void mark(sem_lbm& s, int cls);

// one full time step: collision, then three SSP-RK3 stages of streaming.
// With pdl, every kernel after the first is a programmatic dependent launch of
// the one before it (the first follows whatever preceded the step normally).
void enqueue_step(sem_lbm& s, bool pdl) {
  Ops& o = *s.ops;
  // rho and mu of fbar^n (rho is current: written by set_density/set_state or the last stage)
  s.pdl = false;
  o.lap(s); mark(s, K_LAP);
  s.pdl = pdl;
  o.mu(s); mark(s, K_MU);
  o.force(s); mark(s, K_FORCE);
  o.collide(s); mark(s, K_COLLIDE);          // fs = f* (RK base state U0)
  o.rhs(s, s.fs); mark(s, K_RHS);            // stage 1 reuses rho, mu of fbar^n
  o.rk(s, 1, s.fs, s.g); mark(s, K_RK);
  for (int stage = 2; stage <= 3; ++stage) {
    o.lap(s); mark(s, K_LAP);
    o.mu(s); mark(s, K_MU);
    o.rhs(s, s.g); mark(s, K_RHS);
    o.rk(s, stage, s.g, stage == 3 ? s.f : s.g); mark(s, K_RK);
  }
  s.pdl = false;
}

int count_kernels_per_step() { return 6 + 2 * 4; }

// capture one step into s.graph (programmatic dependent launches when pdl)
int capture_step(sem_lbm& s, bool pdl) {
  cudaGraph_t gr;
  CUDA_TRY(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step(s, pdl);
  cudaError_t e1 = cudaStreamEndCapture(s.stream, &gr);
  if (e1 != cudaSuccess) return fail(SEMLBM_ECUDA, "graph capture: %s", cudaGetErrorString(e1));
  cudaError_t e2 = cudaGraphInstantiate(&s.graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e2 != cudaSuccess) {
    s.graph = nullptr;
    return fail(SEMLBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
  }
  s.graph_pdl = pdl;
  return 0;
}

bool record_event(sem_lbm& s, int cls) {
  if (s.nev == s.ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    s.ev.push_back(e);
    s.ev_cls.push_back(-1);
  }
  s.ev_cls[s.nev] = cls;
  if (cudaEventRecord(s.ev[s.nev], s.stream) != cudaSuccess) return false;
  ++s.nev;
  return true;
}

void mark(sem_lbm& s, int cls) {
  if (s.prof_on) record_event(s, cls);
}

size_t layout(sem_lbm& s, char* base) {
  Carve c{base};
  const int64_t V = s.V, Q = s.Q, D = s.D;
  s.f = c.take<double>(Q * V);
  s.fs = c.take<double>(Q * V);
  s.g = c.take<double>(Q * V);
  s.r = c.take<double>(Q * V);
  s.rho = c.take<double>(V);
  s.mu = c.take<double>(V);
  s.lapr = c.take<double>(V);
  s.Fp = c.take<double>(D * V);
  s.drho = c.take<double>(D * V);
  s.MJ = c.take<double>(D * D * V);
  // stored pair coefficients: D3Q13 only (its contraction costs 3 fma per pair)
  const bool pair_metric = s.lat == SEMLBM_D3Q13;
  s.CJ = c.take<double>(pair_metric ? (Q - 1) / 2 * D * V : 0);
  if (!pair_metric) s.CJ = nullptr;
  s.Gm = c.take<double>(D * (D + 1) / 2 * V);
  s.Me = c.take<double>(V);
  s.invMg = c.take<double>(s.G);
  s.xyz = c.take<double>(D * V);
  s.Dm = c.take<double>(s.n * s.n);
  s.wg = c.take<double>(s.n);
  s.off = c.take<int>(s.G + 1);
  s.idx = c.take<int>(V);
  s.slot = c.take<int>(V);
  const int64_t R = std::max<int64_t>(s.R, 1);
  s.wet = c.take<double>(R);
  s.ae = c.take<double>(Q * R);
  s.rec_elem = c.take<int>(R);
  s.rec_node = c.take<int>(R);
  s.rec_mask = c.take<int>(R);
  s.rec_cos = c.take<double>(R * 2 * D);
  s.rec_ub = c.take<double>(R * 2 * D * D);   // wall records only: small
  s.wub = c.take<double>(Q * R);
  s.flags = c.take<int>(8);
  s.parts = c.take<DiagPart>(s.diag_blocks);
  s.dout = c.take<DiagPart>(1);
  s.rec_tag = c.take<int>(R * 2 * D);
  s.wsf = c.take<double>(R * 2 * D);
  s.wparts = c.take<WetPart>(s.diag_blocks);
  s.wout = c.take<WetPart>(1);
  return c.off;
}

void fill_view(sem_lbm& s) {
  View& v = s.view;
  v.f = s.f; v.fs = s.fs; v.g = s.g; v.r = s.r;
  v.rho = s.rho; v.mu = s.mu; v.lapr = s.lapr; v.Fp = s.Fp; v.drho = s.drho;
  v.flags = s.flags;
  v.MJ = s.MJ; v.Gm = s.Gm; v.Me = s.Me; v.invMg = s.invMg; v.Dm = s.Dm; v.CJ = s.CJ;
  v.off = s.off; v.idx = s.idx; v.wslot = s.slot; v.wet = s.wet; v.ae = s.ae;
  v.R = (int)s.R; v.E = (int)s.E; v.G = (int)s.G;
  v.wub = s.wub;
  v.has_ub = s.moving ? 1 : 0;
  v.V = s.V;
  v.dt = s.dt;
  v.omega = 1.0 / (s.tau + 0.5);
  v.kappa = s.kappa;
  v.fbeta = s.mu0f * s.beta;
  v.rho_l = s.rho_l;
  v.rho_v = s.rho_v;
  v.fgrad = s.force_split ? 0.0 : 1.0;
}

int diag_blocks_for(int64_t V) { return (int)std::min<int64_t>(1184, (V + 255) / 256); }

int host_copy_in(sem_lbm* s, void* dst, const void* src, size_t bytes, int src_on_device) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice, s->stream));
  if (!src_on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  return 0;
}

// compact state: fbar on the global nodes, [Q][G] in node-group order, to and
// from the element-local copies [Q][V]; one thread per node group.  The
// scatter also writes rho at every copy, summed over q in the order the
// density kernel uses (the same bits)
__global__ void k_scatter_global(const int* __restrict__ off, const int* __restrict__ idx, int G,
                                 int Q, int64_t V, const double* __restrict__ src,
                                 double* __restrict__ dst, double* __restrict__ rho) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int j0 = off[g], j1 = off[g + 1];
  double rs = 0.0;
  for (int q = 0; q < Q; ++q) {
    const double val = src[(int64_t)q * G + g];
    rs += val;
    for (int j = j0; j < j1; ++j) dst[q * V + idx[j]] = val;
  }
  for (int j = j0; j < j1; ++j) rho[idx[j]] = rs;
}

__global__ void k_gather_global(const int* __restrict__ off, const int* __restrict__ idx, int G,
                                int Q, int64_t V, const double* __restrict__ src,
                                double* __restrict__ dst) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int i0 = idx[off[g]];   // the first copy (all copies are equal)
  for (int q = 0; q < Q; ++q) dst[(int64_t)q * G + g] = src[q * V + i0];
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* sem_lbm_last_error(void) { return g_err.c_str(); }

size_t sem_lbm_workspace_bytes(const sem_lbm_mesh* mesh, int N, sem_lbm_lattice lattice) {
  if (validate(mesh, N, lattice)) return 0;
  HostMaps h;
  sem_lbm_params p{};
  std::vector<double> many(64, M_PI / 2);
  p.n_tags = 64;
  p.theta_tag = many.data();
  if (build_maps(mesh, N, M_PI / 2, &p, h)) return 0;
  sem_lbm s{};
  s.lat = lattice;
  s.D = mesh->dim;
  s.N = N;
  s.n = N + 1;
  s.NL = ipow(s.n, s.D);
  s.Q = q_of(lattice);
  s.E = mesh->n_elem;
  s.V = s.E * s.NL;
  s.G = h.G;
  s.R = (int64_t)h.rec_elem.size();
  s.diag_blocks = diag_blocks_for(s.V);
  return layout(s, nullptr);
}

int sem_lbm_create(const sem_lbm_mesh* mesh, int N, sem_lbm_lattice lattice, double beta,
                   double kappa, double tau, double theta_w, const sem_lbm_params* params,
                   sem_lbm_t** out) {
  g_err.clear();
  if (!out) return fail(SEMLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (int rc = validate(mesh, N, lattice)) return rc;
  if (!(beta > 0) || !(kappa > 0) || !(tau > 0) || !std::isfinite(theta_w))
    return fail(SEMLBM_EINVAL, "beta, kappa, tau must be positive and theta_w finite");
  sem_lbm_params p{};
  if (params) p = *params;
  if (p.force_split != 0 && p.force_split != 1)
    return fail(SEMLBM_EINVAL, "force_split must be 0 or 1 (got %d)", p.force_split);
  HostMaps h;
  if (int rc = build_maps(mesh, N, theta_w, &p, h)) return rc;

  sem_lbm* s = new (std::nothrow) sem_lbm();
  if (!s) return fail(SEMLBM_ENOMEM, "host allocation failed");
  s->lat = lattice;
  s->D = mesh->dim;
  s->N = N;
  s->n = N + 1;
  s->NL = ipow(s->n, s->D);
  s->Q = q_of(lattice);
  s->E = mesh->n_elem;
  s->V = s->E * s->NL;
  s->G = h.G;
  s->first_copy.resize(h.G);
  for (int64_t g = 0; g < h.G; ++g) s->first_copy[g] = h.idx[h.off[g]];
  s->R = (int64_t)h.rec_elem.size();
  s->moving = h.moving;
  s->beta = beta;
  s->kappa = kappa;
  s->tau = tau;
  s->theta_w = theta_w;
  s->rho_l = p.rho_l > 0 ? p.rho_l : 1.0;
  s->rho_v = p.rho_v > 0 ? p.rho_v : 0.1;
  s->mu0f = p.mu0_factor > 0 ? p.mu0_factor : 2.0;
  s->force_split = p.force_split;
  const double speed = speed_max(lattice);
  if (p.dt > 0) {
    s->dt = p.dt;
  } else {
    // advective CFL on the smallest GLL spacing, and the capillary-wave bound
    // dt <= 0.1 h^2 / sqrt(rho_l kappa) (omega ~ sqrt(rho kappa) k^2)
    const double h = min_spacing(mesh, N);
    s->dt = std::min((p.cfl > 0 ? p.cfl : 0.4) * h / speed, 0.1 * h * h / std::sqrt(s->rho_l * kappa));
  }
  s->diag_blocks = diag_blocks_for(s->V);
  s->ops = select_ops(lattice, N);
  s->kernels_per_step = count_kernels_per_step();
  auto bail = [&](int rc) {
    sem_lbm_destroy(s);
    return rc;
  };
  if (!s->ops) return bail(fail(SEMLBM_EUNSUPPORTED, "no kernels for N = %d", N));
  if (s->ops->prepare() != 0) return bail(fail(SEMLBM_ECUDA, "cudaFuncSetAttribute failed"));

  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(fail(SEMLBM_ECUDA, "cudaGetDevice failed"));
  if (cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
    return bail(fail(SEMLBM_ECUDA, "cudaDeviceGetAttribute failed"));
  if (p.stream) {
    s->stream = (cudaStream_t)p.stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(SEMLBM_ECUDA, "cudaStreamCreate failed"));
    s->own_stream = true;
  }
  s->ws_bytes = layout(*s, nullptr);
  if (p.workspace) {
    if (p.workspace_bytes < s->ws_bytes)
      return bail(fail(SEMLBM_ENOMEM, "workspace of %zu bytes is below the %zu needed",
                       p.workspace_bytes, s->ws_bytes));
    if (((uintptr_t)p.workspace) & 255) return bail(fail(SEMLBM_EINVAL, "workspace must be 256-byte aligned"));
    s->ws = p.workspace;
  } else {
    if (cudaMalloc(&s->ws, s->ws_bytes) != cudaSuccess) {
      s->ws = nullptr;
      return bail(fail(SEMLBM_ENOMEM, "cudaMalloc of %zu bytes failed", s->ws_bytes));
    }
    s->own_ws = true;
  }
  layout(*s, (char*)s->ws);
  fill_view(*s);

  std::vector<double> x, w, Dm;
  gll_tables(N, x, w, Dm);
  const int D = s->D;
  cudaStream_t st = s->stream;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = up(s->xyz, mesh->node_xyz, sizeof(double) * D * s->V) &&
            up(s->Dm, Dm.data(), sizeof(double) * s->n * s->n) &&
            up(s->wg, w.data(), sizeof(double) * s->n) &&
            up(s->off, h.off.data(), sizeof(int) * (s->G + 1)) &&
            up(s->idx, h.idx.data(), sizeof(int) * s->V) &&
            up(s->slot, h.slot.data(), sizeof(int) * s->V) &&
            cudaMemsetAsync(s->flags, 0, 8 * sizeof(int), st) == cudaSuccess;
  if (ok && s->R > 0)
    ok = (!s->moving || up(s->rec_ub, h.rec_ub.data(), sizeof(double) * s->R * 2 * D * D)) &&
         up(s->rec_elem, h.rec_elem.data(), sizeof(int) * s->R) &&
         up(s->rec_node, h.rec_node.data(), sizeof(int) * s->R) &&
         up(s->rec_mask, h.rec_mask.data(), sizeof(int) * s->R) &&
         up(s->rec_cos, h.rec_cos.data(), sizeof(double) * s->R * 2 * D) &&
         up(s->rec_tag, h.rec_tag.data(), sizeof(int) * s->R * 2 * D);
  if (!ok) return bail(fail(SEMLBM_ECUDA, "upload failed: %s", cudaGetErrorString(cudaGetLastError())));
  s->ops->geom(*s);
  s->ops->wall(*s);
  int flags[2] = {0, 0};
  if (cudaMemcpyAsync(flags, s->flags, sizeof flags, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return bail(fail(SEMLBM_ECUDA, "geometry setup failed: %s", cudaGetErrorString(cudaGetLastError())));
  if (flags[0]) return bail(fail(SEMLBM_EINVAL, "mesh has an element with non-positive Jacobian"));
  *out = s;
  return SEMLBM_OK;
}

int sem_lbm_set_density(sem_lbm_t* s, const double* rho, int on_device) {
  if (!s || !rho) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  double* src = s->lapr;   // staging for host data (overwritten by the next step anyway)
  if (int rc = host_copy_in(s, src, rho, sizeof(double) * s->V, on_device)) return rc;
  CUDA_TRY(cudaMemsetAsync(s->flags, 0, 8 * sizeof(int), s->stream));
  s->ops->init(*s, src);
  CUDA_TRY(cudaGetLastError());
  s->state_ready = true;
  s->step = 0;
  return 0;
}

int sem_lbm_set_state(sem_lbm_t* s, const double* fbar, int on_device, int64_t step) {
  if (!s || !fbar) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  if (int rc = host_copy_in(s, s->f, fbar, sizeof(double) * s->Q * s->V, on_device)) return rc;
  s->ops->density(*s);
  CUDA_TRY(cudaGetLastError());
  s->state_ready = true;
  s->step = step;
  return 0;
}

int sem_lbm_set_state_global(sem_lbm_t* s, const double* fbar_g, int on_device, int64_t step) {
  if (!s || !fbar_g) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  const double* src = fbar_g;
  if (!on_device) {   // staged in the stage-state array (overwritten by the next step anyway)
    if (int rc = host_copy_in(s, s->g, fbar_g, sizeof(double) * s->Q * s->G, 0)) return rc;
    src = s->g;
  }
  k_scatter_global<<<grid_of(s->G, 256), 256, 0, s->stream>>>(s->off, s->idx, (int)s->G, s->Q,
                                                              s->V, src, s->f, s->rho);
  CUDA_TRY(cudaGetLastError());
  s->state_ready = true;
  s->step = step;
  return 0;
}

int sem_lbm_get_state_global(sem_lbm_t* s, double* fbar_g, int on_device, int64_t* step) {
  if (!s || !fbar_g) return fail(SEMLBM_EINVAL, "NULL argument");
  if (!s->state_ready) return fail(SEMLBM_EINVAL, "state not set");
  DeviceGuard dg(s->device);
  // a host destination is staged in the stage-state array, which only the
  // step reads, after writing it
  double* dst = on_device ? fbar_g : s->g;
  k_gather_global<<<grid_of(s->G, 256), 256, 0, s->stream>>>(s->off, s->idx, (int)s->G, s->Q,
                                                             s->V, s->f, dst);
  CUDA_TRY(cudaGetLastError());
  if (!on_device) {
    CUDA_TRY(cudaMemcpyAsync(fbar_g, dst, sizeof(double) * s->Q * s->G, cudaMemcpyDeviceToHost,
                             s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  if (step) *step = s->step;
  return 0;
}

int sem_lbm_get_global_nodes(const sem_lbm_t* s, int64_t* first_copy) {
  if (!s || !first_copy) return fail(SEMLBM_EINVAL, "NULL argument");
  for (int64_t g = 0; g < s->G; ++g) first_copy[g] = s->first_copy[g];
  return 0;
}

int sem_lbm_step(sem_lbm_t* s, int64_t n_steps) {
  if (!s) return fail(SEMLBM_EINVAL, "NULL solver");
  if (n_steps < 0) return fail(SEMLBM_EINVAL, "n_steps must be >= 0");
  if (!s->state_ready) return fail(SEMLBM_EINVAL, "state not set (call sem_lbm_set_density)");
  if (s->batch) return fail(SEMLBM_EINVAL, "solver is stepped by its batch (sem_lbm_batch_step)");
  if (n_steps == 0) return 0;
  DeviceGuard dg(s->device);
  if (s->prof_on) {
    if (s->nev == 0 && !record_event(*s, -1)) return fail(SEMLBM_ECUDA, "cudaEventRecord failed");
    for (int64_t i = 0; i < n_steps; ++i) enqueue_step(*s, false);   // events bracket each kernel
    CUDA_TRY(cudaGetLastError());
    s->step += n_steps;
    return 0;
  }
  if (!s->graph) {
    // with programmatic edges between the step's kernels first; should that
    // capture or instantiation fail, the plain graph of the same kernels
    int rc = capture_step(*s, true);
    if (rc != 0) {
      cudaGetLastError();
      if ((rc = capture_step(*s, false)) != 0) return rc;
    }
  }
  for (int64_t i = 0; i < n_steps; ++i) CUDA_TRY(cudaGraphLaunch(s->graph, s->stream));
  s->step += n_steps;
  return 0;
}

int sem_lbm_diagnostics(sem_lbm_t* s, sem_lbm_diag* out) {
  if (!s || !out) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  if (!s->state_ready) return fail(SEMLBM_EINVAL, "state not set");
  s->ops->diag(*s);
  CUDA_TRY(cudaGetLastError());
  DiagPart d;
  int flags[3];   // [1] non-finite stage state, [2] a bounded tile-staging wait gave up
  CUDA_TRY(cudaMemcpyAsync(&d, s->dout, sizeof d, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaMemcpyAsync(flags, s->flags, sizeof flags, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  out->step = s->step;
  out->time = s->step * s->dt;
  out->mass = d.mass;
  out->ke_max = d.ke_max;
  out->ke_int = d.ke_int;
  out->umax = std::sqrt(d.u2max);
  out->rho_min = d.rho_min;
  out->rho_max = d.rho_max;
  out->n_nonfinite = (int64_t)d.nonfinite;
  out->status = (d.nonfinite > 0 || flags[1]) ? SEMLBM_ENONFINITE
                 : flags[2]                     ? SEMLBM_ETIMEOUT
                                                : SEMLBM_OK;
  return 0;
}

int sem_lbm_wetting_moments(sem_lbm_t* s, int tag, double rho_v_ref, double rho_l_ref,
                            sem_lbm_wetting* out) {
  if (!s || !out) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  if (!s->state_ready) return fail(SEMLBM_EINVAL, "state not set");
  WetPart w;
  if (!(rho_v_ref > 0) || !(rho_l_ref > 0)) {
    // bulk phase densities of the state: the mass-weighted mean density of the
    // nodes with phi < 0.02 and phi > 0.98, phi taken on its density range
    s->ops->diag(*s);
    CUDA_TRY(cudaGetLastError());
    DiagPart d;
    CUDA_TRY(cudaMemcpyAsync(&d, s->dout, sizeof d, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (!(d.rho_max > d.rho_min)) return fail(SEMLBM_EINVAL, "uniform density: no interface");
    s->ops->wet(*s, tag, d.rho_min, d.rho_max);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(&w, s->wout, sizeof w, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    rho_v_ref = w.mv > 0 ? w.rv / w.mv : d.rho_min;
    rho_l_ref = w.ml > 0 ? w.rl / w.ml : d.rho_max;
  }
  if (!(rho_l_ref > rho_v_ref)) return fail(SEMLBM_EINVAL, "rho_l_ref must exceed rho_v_ref");
  s->ops->wet(*s, tag, rho_v_ref, rho_l_ref);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(&w, s->wout, sizeof w, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  *out = sem_lbm_wetting{};
  out->volume = w.vol;
  out->rho_v_ref = rho_v_ref;
  out->rho_l_ref = rho_l_ref;
  out->wall = w.wall;
  out->wetted = w.wet;
  for (int c = 0; c < s->D; ++c) {
    out->centroid[c] = w.vol != 0.0 ? w.vx[c] / w.vol : 0.0;
    out->wet_centroid[c] = w.wet != 0.0 ? w.wx[c] / w.wet : 0.0;
  }
  return 0;
}

int sem_lbm_get_field(sem_lbm_t* s, int which, double* dst, int dst_on_device) {
  if (!s || !dst) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  if (!s->state_ready) return fail(SEMLBM_EINVAL, "state not set");
  const double* src;
  size_t count;
  switch (which) {
    case 0: src = s->f; count = (size_t)s->Q * s->V; break;
    case 1: src = s->rho; count = s->V; break;
    case 2: s->ops->velocity(*s, s->Fp); src = s->Fp; count = (size_t)s->D * s->V; break;
    case 3: s->ops->lap(*s); s->ops->mu(*s); src = s->mu; count = s->V; break;
    default: return fail(SEMLBM_EINVAL, "unknown field %d", which);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(double),
                           dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s->stream));
  if (!dst_on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  return 0;
}

int sem_lbm_get_state(sem_lbm_t* s, double* fbar, int on_device, int64_t* step) {
  if (int rc = sem_lbm_get_field(s, 0, fbar, on_device)) return rc;
  if (step) *step = s->step;
  return 0;
}

int sem_lbm_get_info(const sem_lbm_t* s, sem_lbm_info_t* out) {
  if (!s || !out) return fail(SEMLBM_EINVAL, "NULL argument");
  out->dim = s->D;
  out->N = s->N;
  out->Q = s->Q;
  out->n_elem = s->E;
  out->n_local = s->V;
  out->n_global = s->G;
  out->n_wall_nodes = s->R;
  out->dt = s->dt;
  out->kappa = s->kappa;
  out->beta = s->beta;
  out->tau = s->tau;
  out->workspace_bytes = s->ws_bytes;
  out->graph_launches = 1;
  out->kernels_per_step = s->kernels_per_step;
  out->elements_per_cta = s->ops->epb;
  out->rhs_pair_groups = s->ops->rhs_split(*s);
  out->graph_pdl = s->graph_pdl ? 1 : 0;
  return 0;
}

int sem_lbm_profile(sem_lbm_t* s, int enable) {
  if (!s) return fail(SEMLBM_EINVAL, "NULL solver");
  s->prof_on = enable != 0;
  s->nev = 0;
  return 0;
}

int sem_lbm_profile_read(sem_lbm_t* s, sem_lbm_profile_t* out) {
  if (!s || !out) return fail(SEMLBM_EINVAL, "NULL argument");
  DeviceGuard dg(s->device);
  memset(out, 0, sizeof *out);
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  for (size_t i = 1; i < s->nev; ++i) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, s->ev[i - 1], s->ev[i]));
    const int c = s->ev_cls[i];
    if (c >= 0 && c < 8) {
      out->ms[c] += ms;
      out->launches[c] += 1;
    }
  }
  if (s->nev > 1) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, s->ev[0], s->ev[s->nev - 1]));
    out->total_ms = ms;
  }
  s->nev = 0;
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free chemical potential: the Laplacian partials go to a fixed
// device array of the library instead of the solver workspace.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_partial[SEMLBM_NOALLOC_MAX_NODES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// device address of g_noalloc_partial on `device`, looked up once per device
// with that device current (the host-side symbol is only a stand-in)
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return fail(SEMLBM_EINVAL, "device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    int prev = 0;
    CUDA_TRY(cudaGetDevice(&prev));
    if (prev != device) CUDA_TRY(cudaSetDevice(device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(SEMLBM_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return 0;
}
}  // namespace

extern "C" {

int sem_lbm_chemical_potential_noalloc(sem_lbm_t* s, const double* rho, double* mu) {
  if (!s || !rho || !mu) return fail(SEMLBM_EINVAL, "NULL argument");
  if (s->V > (int64_t)SEMLBM_NOALLOC_MAX_NODES)
    return fail(SEMLBM_EINVAL,
                "mesh has %lld element-local nodes; the allocation-free entry point holds at most %d",
                (long long)s->V, SEMLBM_NOALLOC_MAX_NODES);
  DeviceGuard dg(s->device);
  double* scratch = nullptr;
  if (int rc = noalloc_scratch(s->device, &scratch)) return rc;
  // k_lap writes every one of the V partials it then reads: nothing to clear
  s->ops->lap_into(*s, rho, scratch);
  s->ops->mu_from(*s, scratch, rho, mu);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

void sem_lbm_destroy(sem_lbm_t* s) {
  if (!s) return;
  DeviceGuard dg(s->device);
  if (s->batch) sem_lbm_batch_remove(s->batch, sem_lbm_batch_slot_of(s));
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->own_ws && s->ws) cudaFree(s->ws);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
