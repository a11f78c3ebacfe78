// FP64 kernels of the SEM-LBM time step (sm_103a).
//
// Element kernels (k_lap, k_force, k_rhs, k_geom): one CTA per batch of EPB
// consecutive elements, one thread per element-local GLL node; the element
// tiles of every field a kernel reads (rho, mu, the Q-1 moving f_alpha) and
// the GLL derivative matrix are staged in shared memory, and each thread
// applies the tensor-product (sum-factorised) derivative along each reference
// axis, with its rows of D held in registers (k_lap, k_force) or read from
// shared memory at each use (k_rhs, whose velocity loop would otherwise spill).
//
// Gather-scatter kernels (k_dss_*): one thread per global node group; the
// copies of a shared node are summed in a fixed order (ascending local index),
// so results do not depend on scheduling.  The streaming partials that k_rhs
// hands to k_dss_rk are node-major (the Q-1 values of a node contiguous, in
// opposite-velocity pairs), so each copy of a node is gathered with 16-byte
// loads from consecutive addresses.
//
// B300's FP64 pipe (about 1.1 TFLOP/s, measured) is the bound of this step, so
// the formulation minimises FP64 instructions: velocity contractions use only
// the non-zero components of e_alpha, opposite directions share their
// coefficients, the rest population (e = 0) does not stream, and all index
// arithmetic is integer.
#pragma once
#include <cstdint>

#include "lattice.cuh"

namespace semlbm {

// threads of an element-kernel CTA: EPB elements of NP^D nodes, rounded to warps
template <int D, int NP, int EPB>
constexpr int cta_threads() { return ((EPB * ipow(NP, D) + 31) / 32) * 32; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <int D, int NP>
struct NodeIdx {
  int i[3];
  __device__ __forceinline__ explicit NodeIdx(int k) {
    i[0] = k % NP;
    i[1] = (k / NP) % NP;
    i[2] = (D == 3) ? k / (NP * NP) : 0;
  }
};

// d/dxi_b of the element tile s (node k) with D row held in registers
template <int NP, int STRIDE>
__device__ __forceinline__ double dline(const double (&row)[NP], const double* __restrict__ line) {
  double acc = row[0] * line[0];
#pragma unroll
  for (int m = 1; m < NP; ++m) acc = fma(row[m], line[m * STRIDE], acc);
  return acc;
}

template <int D, int NP>
__device__ __forceinline__ void grad_ref(const double (&Dr)[D][NP], const NodeIdx<D, NP>& ix,
                                         const double* __restrict__ tile, int k, double (&out)[D]) {
  out[0] = dline<NP, 1>(Dr[0], tile + k - ix.i[0]);
  out[1] = dline<NP, NP>(Dr[1], tile + k - ix.i[1] * NP);
  if constexpr (D == 3) out[2] = dline<NP, NP * NP>(Dr[2], tile + k - ix.i[2] * NP * NP);
}

// reference gradients of two tiles at node k, as 2D independent chains, each
// subtracted from a start value: oa[b] = init[b] - sum_m D[i_b][m] ta[...] and
// ob[b] = init[b] - sum_m D[i_b][m] tb[...], every term an fma (the streaming
// kernel starts both from t v_b).  The rows of D are read from shared memory at
// every use (sD + i_b NP for axis b): holding them in registers across the
// streaming kernel's velocity loop made it spill
__device__ __forceinline__ double lds(const double* p) { return *(volatile const double*)p; }

template <int D, int NP>
__device__ __forceinline__ void grad_ref2_from(const double* sD, const NodeIdx<D, NP>& ix,
                                               const double* __restrict__ ta,
                                               const double* __restrict__ tb, int k,
                                               const double (&init)[D], double (&oa)[D],
                                               double (&ob)[D]) {
  constexpr int st[3] = {1, NP, NP * NP};
  int k0[D];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    k0[b] = k - ix.i[b] * st[b];
    const double d0 = lds(sD + ix.i[b] * NP);
    oa[b] = fma(-d0, ta[k0[b]], init[b]);
    ob[b] = fma(-d0, tb[k0[b]], init[b]);
  }
#pragma unroll
  for (int m = 1; m < NP; ++m)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const double dm = lds(sD + ix.i[b] * NP + m);
      oa[b] = fma(-dm, ta[k0[b] + m * st[b]], oa[b]);
      ob[b] = fma(-dm, tb[k0[b] + m * st[b]], ob[b]);
    }
}

template <int D, int NP>
__device__ __forceinline__ void load_rows(const double* __restrict__ sD, const NodeIdx<D, NP>& ix,
                                          bool transpose, double (&Dr)[D][NP]) {
#pragma unroll
  for (int b = 0; b < D; ++b)
#pragma unroll
    for (int m = 0; m < NP; ++m)
      Dr[b][m] = transpose ? sD[m * NP + ix.i[b]] : sD[ix.i[b] * NP + m];
}

__device__ __forceinline__ void stage_in(double* __restrict__ s, const double* __restrict__ g,
                                         int64_t base, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) s[i] = __ldg(g + base + i);
}

// Tile staging by the bulk-copy engine (cp.async.bulk, the one-dimensional form
// of TMA, sm_90 and later): thread 0 starts `ntiles` copies of `count` doubles,
// tile t from src(t) (global) to dst(t) (shared), all completing on one
// mbarrier, and every thread of the CTA waits for their bytes.  The caller
// guarantees 16-byte aligned sources, destinations and sizes (count even).  The
// wait is bounded: after kBulkWaitPolls polls it sets flags[2] (reported as
// SEMLBM_ETIMEOUT), waits once more with the same bound for the copies still in
// flight into this CTA's shared memory, and returns, so a copy that never lands
// cannot hang the GPU.  One use per CTA lifetime (the barrier is initialised
// here, phase 0).
constexpr int kBulkWaitPolls = 1 << 22;

template <class Tile>
__device__ __forceinline__ void stage_bulk(int ntiles, int count, Tile tile, int* flags) {
  __shared__ alignas(8) unsigned long long bar;
  const unsigned mb = (unsigned)__cvta_generic_to_shared(&bar);
  const unsigned bytes = (unsigned)count * 8u;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                 "r"(bytes * (unsigned)ntiles) : "memory");
    for (int t = 0; t < ntiles; ++t) {
      double* dst;
      const double* src;
      tile(t, dst, src);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src), "r"(bytes), "r"(mb)
          : "memory");
    }
  }
  __syncthreads();   // the barrier is initialised before anyone polls it
  auto wait = [&]() {
    unsigned done = 0;
    for (int it = 0; it < kBulkWaitPolls && !done; ++it)
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(done)
          : "r"(mb), "r"(0u)
          : "memory");
    return done != 0;
  };
  if (!wait()) {
    atomicOr(flags + 2, 1);
    wait();   // the copies in flight, before the CTA reuses or releases its tiles
  }
}

// Stages ntiles element tiles of `count` doubles each (tile(t, dst, src) names
// tile t): by bulk copies when `bulk` is set and every source, destination and
// size is 16-byte aligned (the same decision on every thread of the CTA), else
// by the load loop.  The caller synchronises the CTA before reading the tiles.
template <class Tile>
__device__ __forceinline__ void stage_tiles(bool bulk, int ntiles, int count, Tile tile,
                                            int* flags) {
  bool ok = bulk && (count & 1) == 0;
  for (int t = 0; t < ntiles && ok; ++t) {
    double* dst;
    const double* src;
    tile(t, dst, src);
    ok = ((reinterpret_cast<uintptr_t>(src) | (unsigned)__cvta_generic_to_shared(dst)) & 15) == 0;
  }
  if (ok) {
    stage_bulk(ntiles, count, tile, flags);
    return;
  }
  for (int t = 0; t < ntiles; ++t) {
    double* dst;
    const double* src;
    tile(t, dst, src);
    for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
  }
}

// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic-serialization attribute may start while its predecessor on the
// stream is still running; pdl_wait() blocks until the predecessor has
// completed and its memory is visible, and is a no-op for an ordinary launch.
// pdl_trigger() lets the successor be scheduled once every CTA of this kernel
// has issued it (or exited).  The step kernels wait before touching global
// memory, so every data dependency is that of a serialised stream, and trigger
// after their work: a successor triggered at the start would occupy SM slots
// with waiting CTAs for the whole of its predecessor (and, transitively, pull
// the rest of the step in behind it), which slowed concurrent branches of a
// batch and split-pair meshes by up to 45 %.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ bool nonfinite(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff;
}

// ---------------------------------------------------------------------------
// setup: geometry per node (Jacobian by D on the coordinates), Eq. (spetrum) M;
// MJ = M_e S J^-1 (S = the velocity set's speed scale) is the metric of the
// force and the streaming right-hand side, with the mass and the speed folded in
// ---------------------------------------------------------------------------
template <int D, int NP, int EPB>
__global__ void __launch_bounds__(cta_threads<D, NP, EPB>()) k_geom(const double* __restrict__ xyz, const double* __restrict__ Dmat,
                       const double* __restrict__ wgll, double scale, double* __restrict__ MJ,
                       double* __restrict__ Gm, double* __restrict__ Me, int* __restrict__ bad,
                       int64_t V, int E) {
  constexpr int NL = ipow(NP, D), NT = EPB * NL;
  extern __shared__ double sm[];
  double* sD = sm;
  double* sx = sD + NP * NP;   // [D][NT]
  const int e0 = blockIdx.x * EPB;
  const int count = min(EPB, E - e0) * NL;
  const int64_t base = (int64_t)e0 * NL;
  for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sD[i] = Dmat[i];
  for (int i = threadIdx.x; i < count * D; i += blockDim.x) {
    const int node = i / D, a = i - node * D;
    sx[a * NT + node] = xyz[(base + node) * D + a];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  if (tid >= count) return;
  const int le = tid / NL, k = tid - le * NL;
  const NodeIdx<D, NP> ix(k);
  double Dr[D][NP];
  load_rows<D, NP>(sD, ix, false, Dr);
  double J[3][3] = {};
  for (int a = 0; a < D; ++a) {
    double g[D];
    grad_ref<D, NP>(Dr, ix, sx + a * NT + le * NL, k, g);
    for (int b = 0; b < D; ++b) J[a][b] = g[b];        // J[a][b] = dx_a / dxi_b
  }
  double adj[3][3], det;
  if constexpr (D == 2) {
    adj[0][0] = J[1][1]; adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0]; adj[1][1] = J[0][0];
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    // row b of adj(J) = (column c) x (column d), (b, c, d) cyclic
    for (int b = 0; b < 3; ++b) {
      const int c = (b + 1) % 3, d = (b + 2) % 3;
      adj[b][0] = J[1][c] * J[2][d] - J[2][c] * J[1][d];
      adj[b][1] = J[2][c] * J[0][d] - J[0][c] * J[2][d];
      adj[b][2] = J[0][c] * J[1][d] - J[1][c] * J[0][d];
    }
    det = J[0][0] * adj[0][0] + J[1][0] * adj[0][1] + J[2][0] * adj[0][2];
  }
  if (!(det > 0.0)) atomicOr(bad, 1);
  const double inv = 1.0 / det;
  const int64_t idx = base + tid;
  double W = wgll[ix.i[0]] * wgll[ix.i[1]];
  if constexpr (D == 3) W *= wgll[ix.i[2]];
  const double me = W * det;
  Me[idx] = me;
  const double ms = me * scale;
  double Ji[3][3];
  for (int b = 0; b < D; ++b)
    for (int a = 0; a < D; ++a) {
      Ji[b][a] = adj[b][a] * inv;                        // dxi_b / dx_a
      MJ[(b * D + a) * V + idx] = ms * Ji[b][a];
    }
  int p = 0;
  for (int b = 0; b < D; ++b)
    for (int c = b; c < D; ++c) {
      double s = 0.0;
      for (int a = 0; a < D; ++a) s += Ji[b][a] * Ji[c][a];
      Gm[(p++) * V + idx] = me * s;
    }
}

// pair coefficients of the streaming right-hand side, stored once per node for
// sets whose contraction costs multiplies: CJ[p][b] = (M_e S J^-1 C_rep(p))_b,
// the same expression k_rhs would evaluate (same bits)
template <class L>
__global__ void k_pair_metric(const double* __restrict__ MJ, double* __restrict__ CJ, int64_t V) {
  constexpr int D = L::D;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V) return;
  double J[D][D];
  for (int b = 0; b < D; ++b)
    for (int a = 0; a < D; ++a) J[b][a] = MJ[(b * D + a) * V + i];
  static_for<0, L::NREP>([&](auto RR) {
    constexpr int A = L::rep(decltype(RR)::value);
#pragma unroll
    for (int b = 0; b < D; ++b)
      CJ[(int64_t)(decltype(RR)::value * D + b) * V + i] = L::template cdot<A>(J[b]);
  });
}

// assembled mass: invMg[g] = 1 / sum over copies of M_e
static __global__ void k_dss_mass(const int* __restrict__ off, const int* __restrict__ idx, int G,
                           const double* __restrict__ Me, double* __restrict__ invMg) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  double s = 0.0;
  for (int j = off[g]; j < off[g + 1]; ++j) s += Me[idx[j]];
  invMg[g] = 1.0 / s;
}

// wall records: area vector of each wall face at the node (cofactor row of J
// times the face's GLL weights, outward), summed over the node's wall faces
template <class L, int NP>
__global__ void k_wall_setup(const double* __restrict__ xyz, const double* __restrict__ Dmat,
                             const double* __restrict__ wgll, const int* __restrict__ rec_elem,
                             const int* __restrict__ rec_node, const double* __restrict__ rec_cos,
                             const int* __restrict__ rec_mask, int R, double sq2bk,
                             const double* __restrict__ rec_ub, double* __restrict__ wet,
                             double* __restrict__ ae, double* __restrict__ wub,
                             double* __restrict__ wsf) {
  constexpr int D = L::D, NL = ipow(NP, D);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int e = rec_elem[r], k = rec_node[r], mask = rec_mask[r];
  const NodeIdx<D, NP> ix(k);
  const double* X = xyz + (int64_t)e * NL * D;
  const int stride[3] = {1, NP, NP * NP};
  double J[3][3] = {};
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double s = 0.0;
      const int k0 = k - ix.i[b] * stride[b];
      for (int m = 0; m < NP; ++m) s += Dmat[ix.i[b] * NP + m] * X[(k0 + m * stride[b]) * D + a];
      J[a][b] = s;
    }
  double adj[3][3];
  if constexpr (D == 2) {
    adj[0][0] = J[1][1]; adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0]; adj[1][1] = J[0][0];
  } else {
    for (int b = 0; b < 3; ++b) {
      const int c = (b + 1) % 3, d = (b + 2) % 3;
      adj[b][0] = J[1][c] * J[2][d] - J[2][c] * J[1][d];
      adj[b][1] = J[2][c] * J[0][d] - J[0][c] * J[2][d];
      adj[b][2] = J[0][c] * J[1][d] - J[1][c] * J[0][d];
    }
  }
  double wsum = 0.0;
  double acc[L::Q], accu[L::Q];
  for (int q = 0; q < L::Q; ++q) acc[q] = accu[q] = 0.0;
  for (int f = 0; f < 2 * D; ++f) {
    if (!((mask >> f) & 1)) {
      wsf[r * 2 * D + f] = 0.0;
      continue;
    }
    const int b = f >> 1;
    const double sgn = (f & 1) ? 1.0 : -1.0;
    double wf = 1.0;
    for (int c = 0; c < D; ++c)
      if (c != b) wf *= wgll[ix.i[c]];
    double a[3], an = 0.0;
    for (int c = 0; c < D; ++c) {
      a[c] = sgn * adj[b][c] * wf;
      an += a[c] * a[c];
    }
    an = sqrt(an);
    wsf[r * 2 * D + f] = an;   // face quadrature weight w |a| of this face-node
    wsum += an * rec_cos[r * 2 * D + f] * sq2bk;
    for (int q = 1; q < L::Q; ++q) {
      double dot = 0.0;
      for (int c = 0; c < D; ++c) dot += L::C(q, c) * a[c];
      dot *= L::S;
      // tangential directions (a . e = 0 up to rounding) are not incoming
      if (dot < -1e-13 * an * L::SPEED_MAX) {
        acc[q] += dot;
        if (rec_ub) {   // this face's wall velocity: -2 t e.u_b / c_s^2 times w (a.e)
          double eu = 0.0;
          for (int c = 0; c < D; ++c) eu += L::C(q, c) * rec_ub[((int64_t)r * 2 * D + f) * D + c];
          accu[q] += dot * (-2.0 * kInvCs2 * L::t(q) * L::S * eu);
        }
      }
    }
  }
  wet[r] = wsum;
  for (int q = 0; q < L::Q; ++q) ae[(int64_t)q * R + r] = acc[q];
  if (wub)
    for (int q = 0; q < L::Q; ++q) wub[(int64_t)q * R + r] = accu[q];
}

// ---------------------------------------------------------------------------
// Everything a time-step kernel needs of one solve.  The single-solve kernels
// receive it as a kernel parameter; the batched persistent kernels read it
// from a device-resident slot table.  Both run the same body functions, so a
// solve computes bit-identical results alone and inside a batch.
// ---------------------------------------------------------------------------
struct View {
  double *f, *fs, *g, *r, *rho, *mu, *lapr, *Fp;   // state and scratch; r is node-major:
                                                   // [V][Q-1], pair p of node i at r + i(Q-1) + 2p
  double* drho;                                    // [D][V] reference gradient of rho (k_lap)
  int* flags;                                      // [0] setup, [1] non-finite
  const double *MJ, *Gm, *Me, *invMg, *Dm;        // geometry (MJ = M_e S J^-1), GLL D
  const double* CJ;   // [NREP][D][V] (M_e S J^-1 C_rep(p))_b, sets with PAIR_METRIC
  const int *off, *idx, *wslot;                    // gather-scatter CSR, wall slots
  const double *wet, *ae;                          // wall records
  const double* wub;   // [Q][R] flux bounce-back wall-velocity coefficients (or unused)
  int R, E, G, has_ub;
  int64_t V;
  double dt, omega, kappa, fbeta, rho_l, rho_v;    // omega = 1/(tau + 1/2), fbeta = mu0 factor * beta
  double fgrad;   // 1: F** uses c_s^2 grad rho - rho grad mu; 0: -rho grad mu alone
};

// ---------------------------------------------------------------------------
// a2: element-local weak Laplacian with the wetting wall term, Eq. (weak)
//     r_i = -sum_b D^T_b [ sum_c G_bc d_c rho ] + wall_i ws cos(theta) sqrt(2b/k)(rl-rho)(rho-rv)
// ---------------------------------------------------------------------------
template <class L, int NP, int EPB>
__device__ __forceinline__ void body_lap(const View& v, const double* __restrict__ rho,
                                         double* __restrict__ out, double* __restrict__ drho,
                                         int eb, double* sm, bool bulk = false) {
  constexpr int D = L::D, NL = ipow(NP, D), NT = EPB * NL;
  const int64_t V = v.V;
  const int E = v.E;
  const double* __restrict__ Gm = v.Gm;
  const double* __restrict__ Dmat = v.Dm;
  const int* __restrict__ wslot = v.wslot;
  const double* __restrict__ wet = v.wet;
  const double rho_l = v.rho_l, rho_v = v.rho_v;
  double* sD = sm;
  double* sr = sD + NP * NP;
  double* st = sr + NT;     // [D][NT]
  const int e0 = eb * EPB;
  const int count = min(EPB, E - e0) * NL;
  const int64_t base = (int64_t)e0 * NL;
  for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sD[i] = __ldg(Dmat + i);
  stage_tiles(bulk, 1, count, [&](int, double*& dst, const double*& src) {
    dst = sr;
    src = rho + base;
  }, v.flags);
  __syncthreads();
  const int tid = threadIdx.x;
  const bool act = tid < count;
  const int le = tid / NL, k = tid - le * NL;
  const NodeIdx<D, NP> ix(act ? k : 0);
  const int64_t idx = base + tid;
  if (act) {
    double Dr[D][NP];
    load_rows<D, NP>(sD, ix, false, Dr);
    double g[D];
    grad_ref<D, NP>(Dr, ix, sr + le * NL, k, g);
    if (drho) {   // reused by k_force and k_rhs of the same stage
#pragma unroll
      for (int b = 0; b < D; ++b) drho[b * V + idx] = g[b];
    }
    if constexpr (D == 2) {
      const double g00 = __ldg(Gm + idx), g01 = __ldg(Gm + V + idx), g11 = __ldg(Gm + 2 * V + idx);
      st[tid] = fma(g01, g[1], g00 * g[0]);
      st[NT + tid] = fma(g11, g[1], g01 * g[0]);
    } else {
      const double g00 = __ldg(Gm + idx), g01 = __ldg(Gm + V + idx), g02 = __ldg(Gm + 2 * V + idx);
      const double g11 = __ldg(Gm + 3 * V + idx), g12 = __ldg(Gm + 4 * V + idx);
      const double g22 = __ldg(Gm + 5 * V + idx);
      st[tid] = fma(g02, g[2], fma(g01, g[1], g00 * g[0]));
      st[NT + tid] = fma(g12, g[2], fma(g11, g[1], g01 * g[0]));
      st[2 * NT + tid] = fma(g22, g[2], fma(g12, g[1], g02 * g[0]));
    }
  }
  __syncthreads();
  if (act) {
    double Dt[D][NP];
    load_rows<D, NP>(sD, ix, true, Dt);
    const int lb = le * NL;
    double acc = dline<NP, 1>(Dt[0], st + lb + k - ix.i[0]);
    acc += dline<NP, NP>(Dt[1], st + NT + lb + k - ix.i[1] * NP);
    if constexpr (D == 3) acc += dline<NP, NP * NP>(Dt[2], st + 2 * NT + lb + k - ix.i[2] * NP * NP);
    double r = -acc;
    const int slot = __ldg(wslot + idx);
    if (slot >= 0) {
      const double rh = sr[lb + k];
      r = fma(__ldg(wet + slot), (rho_l - rh) * (rh - rho_v), r);
    }
    out[idx] = r;
  }
}

// a3: DSS of the Laplacian partials and the chemical potential, Eq. (chemi)
__device__ __forceinline__ void body_dss_mu(const View& v, const double* __restrict__ lapr,
                                            const double* __restrict__ rho,
                                            double* __restrict__ mu, int g) {
  if (g >= v.G) return;
  const int* __restrict__ off = v.off;
  const int* __restrict__ idx = v.idx;
  const double rho_l = v.rho_l, rho_v = v.rho_v;
  const int j0 = off[g], j1 = off[g + 1];
  const int i0 = idx[j0];
  double s = lapr[i0];
  for (int j = j0 + 1; j < j1; ++j) s += lapr[idx[j]];
  const double lap = s * __ldg(v.invMg + g);
  const double r = rho[i0];
  const double m0 = v.fbeta * (r - rho_l) * (r - rho_v) * (2.0 * r - rho_l - rho_v);
  const double val = fma(-v.kappa, lap, m0);
  for (int j = j0; j < j1; ++j) mu[idx[j]] = val;
}

// a4 (part 1): element-local force M_e (c_s^2 grad rho - rho grad mu) (Sec. 2.1)
template <class L, int NP, int EPB>
__device__ __forceinline__ void body_force(const View& v, int eb, double* sm, bool bulk = false) {
  constexpr int D = L::D, NL = ipow(NP, D), NT = EPB * NL;
  const int64_t V = v.V;
  const int E = v.E;
  const double* __restrict__ MJ = v.MJ;
  const double* __restrict__ Dmat = v.Dm;
  double* __restrict__ Fp = v.Fp;
  double* sD = sm;
  double* sr = sD + NP * NP;
  double* smu = sr + NT;
  const int e0 = eb * EPB;
  const int count = min(EPB, E - e0) * NL;
  const int64_t base = (int64_t)e0 * NL;
  for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sD[i] = __ldg(Dmat + i);
  stage_tiles(bulk, 2, count, [&](int t, double*& dst, const double*& src) {
    dst = t == 0 ? sr : smu;
    src = (t == 0 ? v.rho : v.mu) + base;
  }, v.flags);
  __syncthreads();
  const int tid = threadIdx.x;
  if (tid < count) {
    const int le = tid / NL, k = tid - le * NL;
    const NodeIdx<D, NP> ix(k);
    const int64_t idx = base + tid;
    double Dr[D][NP];
    load_rows<D, NP>(sD, ix, false, Dr);
    double dr[D], dm[D];
#pragma unroll
    for (int b = 0; b < D; ++b) dr[b] = v.drho[b * V + idx];
    grad_ref<D, NP>(Dr, ix, smu + le * NL, k, dm);
    // reference components of (c_s^2 d rho - rho d mu) / S (the first term
    // times fgrad); MJ carries M_e S
    constexpr double kInvS = 1.0 / L::S;
    const double kF = (kCs2 / L::S) * v.fgrad;
    const double rs = sr[le * NL + k] * kInvS;
    double w[D];
#pragma unroll
    for (int b = 0; b < D; ++b) w[b] = fma(kF, dr[b], -rs * dm[b]);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double F = __ldg(MJ + a * V + idx) * w[0];
#pragma unroll
      for (int b = 1; b < D; ++b) F = fma(__ldg(MJ + (b * D + a) * V + idx), w[b], F);
      Fp[a * V + idx] = F;
    }
  }
}

// a4 (part 2): DSS average of the force and BGK collision with F**
//   f* = fbar - (fbar - fbar_eq)/(tau + 1/2) + dt F**, fbar_eq = f^eq - dt F**/2
template <class L>
__device__ __forceinline__ void body_dss_collide(const View& v, int g) {
  constexpr int D = L::D, Q = L::Q;
  if (g >= v.G) return;
  const int64_t V = v.V;
  const int* __restrict__ off = v.off;
  const int* __restrict__ idx = v.idx;
  const double* __restrict__ Fp = v.Fp;
  const double* __restrict__ f = v.f;
  double* __restrict__ fs = v.fs;
  const double omega = v.omega, dt = v.dt;
  const int j0 = off[g], j1 = off[g + 1];
  const int i0 = idx[j0];
  const double im = __ldg(v.invMg + g);
  double F[D];   // gather-scatter average of M_e F_e (copy loop outermost)
#pragma unroll
  for (int a = 0; a < D; ++a) F[a] = Fp[a * V + i0];
  for (int j = j0 + 1; j < j1; ++j) {
    const int ii = idx[j];
#pragma unroll
    for (int a = 0; a < D; ++a) F[a] += Fp[a * V + ii];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) F[a] *= im;
  double fa[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) fa[q] = f[q * V + i0];
  const double rh = v.rho[i0];
  // rho u = sum_a fbar_a e_a (Eq. momentum), via opposite-direction differences
  double m[D];
#pragma unroll
  for (int a = 0; a < D; ++a) m[a] = 0.0;
  static_for<0, L::NREP>([&](auto R) {
    constexpr int A = L::rep(decltype(R)::value), B = L::opp(A);
    const double dfa = fa[A] - fa[B];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double c = L::C(A, a);
      if (c == 1.0) m[a] += dfa;
      else if (c == -1.0) m[a] -= dfa;
      else if (c != 0.0) m[a] = fma(c, dfa, m[a]);
    }
  });
  const double su = L::S / rh;
  double u[D];
#pragma unroll
  for (int a = 0; a < D; ++a) u[a] = m[a] * su;
  double uu = u[0] * u[0], uF = u[0] * F[0];
#pragma unroll
  for (int a = 1; a < D; ++a) {
    uu = fma(u[a], u[a], uu);
    uF = fma(u[a], F[a], uF);
  }
  const double base_eq = fma(-1.5, uu, 1.0);   // 1 - u^2/(2 c_s^2)
  // f* = fbar - omega (fbar - f^eq + dt F**/2) + dt F**
  //    = (1 - omega) fbar + omega f^eq + dt (1 - omega/2) F**,
  // f^eq = rho t (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u^2)   (Eq. geq_s, c_s^2 = 1/3)
  // F**  = 3 t (3 (e.u)(e.F) - u.F)                      (Sec. 2.1)
  const double a = 1.0 - omega;
  const double wr = omega * rh;
  const double bdt = dt * (1.0 - 0.5 * omega);
  double out[Q];
  {
    constexpr double T0 = L::t(0);
    out[0] = fma(a, fa[0], fma(wr * T0, base_eq, (3.0 * T0 * bdt) * -uF));
  }
  static_for<0, L::NREP>([&](auto R) {
    constexpr int A = L::rep(decltype(R)::value), B = L::opp(A);
    constexpr double T = L::t(A);
    const double cu = L::template cdot<A>(u);
    const double cF = L::template cdot<A>(F);
    const double eu = L::S * cu;
    const double fss = (3.0 * T * bdt) * fma(3.0 * L::S * L::S, cu * cF, -uF);  // same for A and B
    const double wrt = wr * T;
    out[A] = fma(a, fa[A], fma(wrt, fma(eu, fma(4.5, eu, 3.0), base_eq), fss));
    out[B] = fma(a, fa[B], fma(wrt, fma(-eu, fma(-4.5, eu, 3.0), base_eq), fss));
  });
  for (int j = j0; j < j1; ++j) {
    const int ii = idx[j];
#pragma unroll
    for (int q = 0; q < Q; ++q) fs[q * V + ii] = out[q];
  }
}

// a5: the element-local right-hand side of one element batch from its staged
// tiles (sD: D; sr, smu: rho and mu; sg: the moving velocities, [Q-1][NT]) for
// the opposite-velocity pairs [pr0, pr1) when SPLIT (all pairs otherwise)
//   r_a = M_e [ -e_a . grad(g_a - t_a rho) - (t_a/c_s^2) rho e_a . grad(mu) ]
//         + flux bounce-back on incoming wall directions (Sec. 2.2)
template <class L, int NP, int EPB, bool SPLIT>
__device__ __forceinline__ void rhs_compute(const View& v, const double* sD, const double* sr,
                                            const double* smu, const double* sg, int count,
                                            int64_t base, int pr0, int pr1) {
  constexpr int D = L::D, Q = L::Q, NL = ipow(NP, D), NT = EPB * NL;
  const int64_t V = v.V;
  const double* __restrict__ MJ = v.MJ;
  const int* __restrict__ wslot = v.wslot;
  const double* __restrict__ wae = v.ae;
  const int R = v.R;
  double* __restrict__ r = v.r;
  const int tid = threadIdx.x;
  if (tid >= count) return;
  const int le = tid / NL, k = tid - le * NL, lb = le * NL;
  const NodeIdx<D, NP> ix(k);
  const int64_t idx = base + tid;
  double dr[D], dm[D];
#pragma unroll
  for (int b = 0; b < D; ++b) dr[b] = v.drho[b * V + idx];
  {
    double Dr[D][NP];
    load_rows<D, NP>(sD, ix, false, Dr);
    grad_ref<D, NP>(Dr, ix, smu + lb, k, dm);
  }
  const double rh_node = sr[lb + k];
  const double rh3 = kInvCs2 * rh_node;
  double vv[D];   // d_b rho - (rho / c_s^2) d_b mu, reference components
#pragma unroll
  for (int b = 0; b < D; ++b) vv[b] = fma(-rh3, dm[b], dr[b]);
  double J[D][D];   // M_e S J^-1 (unless the pair coefficients are stored)
  if constexpr (!L::PAIR_METRIC) {
#pragma unroll
    for (int b = 0; b < D; ++b)
#pragma unroll
      for (int a = 0; a < D; ++a) J[b][a] = __ldg(MJ + (b * D + a) * V + idx);
  }
  const int slot = __ldg(wslot + idx);
  static_for<0, L::NREP>([&](auto RR) {
    constexpr int A = L::rep(decltype(RR)::value), B = L::opp(A);
    constexpr double T = L::t(A);
    if constexpr (SPLIT) {
      constexpr int RI = decltype(RR)::value;
      if (RI < pr0 || RI >= pr1) return;
    }
    double c[D];   // (M_e S J^-1 C_A)_b: M_e e_A . grad = sum_b c_b d_b
    if constexpr (L::PAIR_METRIC) {
#pragma unroll
      for (int b = 0; b < D; ++b)
        c[b] = __ldg(v.CJ + (int64_t)(decltype(RR)::value * D + b) * V + idx);
    } else {
#pragma unroll
      for (int b = 0; b < D; ++b) c[b] = L::template cdot<A>(J[b]);
    }
    // r_A = M_e (t e_A.v - e_A.grad g_A), r_B = -M_e (t e_A.v - e_A.grad g_B), e_B = -e_A
    double rA, rB;
    if constexpr (L::TV_START) {
      // = sum_b c_b (t v_b - d_b g_A) and -sum_b c_b (t v_b - d_b g_B): each
      // derivative chain starts from t v_b, so every term of it is an fma
      double tv[D];
#pragma unroll
      for (int b = 0; b < D; ++b) tv[b] = T * vv[b];
      double xA[D], xB[D];
      grad_ref2_from<D, NP>(sD, ix, sg + (A - 1) * NT + lb, sg + (B - 1) * NT + lb, k, tv, xA,
                            xB);
      rA = c[0] * xA[0];
      rB = -c[0] * xB[0];
#pragma unroll
      for (int b = 1; b < D; ++b) {
        rA = fma(c[b], xA[b], rA);
        rB = fma(-c[b], xB[b], rB);
      }
    } else {
      // t (c.v) once per pair, minus the derivatives nA = -grad g_A, nB = -grad g_B
      const double zero[D] = {};
      double nA[D], nB[D];
      grad_ref2_from<D, NP>(sD, ix, sg + (A - 1) * NT + lb, sg + (B - 1) * NT + lb, k, zero, nA,
                            nB);
      double cv = c[0] * vv[0];
#pragma unroll
      for (int b = 1; b < D; ++b) cv = fma(c[b], vv[b], cv);
      const double tcv = T * cv;
      rA = fma(c[0], nA[0], tcv);
      rB = fma(-c[0], nB[0], -tcv);
#pragma unroll
      for (int b = 1; b < D; ++b) {
        rA = fma(c[b], nA[b], rA);
        rB = fma(-c[b], nB[b], rB);
      }
    }
    if (slot >= 0) {
      const double gA = sg[(A - 1) * NT + lb + k], gB = sg[(B - 1) * NT + lb + k];
      rA = fma(__ldg(wae + (int64_t)A * R + slot), gA - gB, rA);
      rB = fma(__ldg(wae + (int64_t)B * R + slot), gB - gA, rB);
      if (v.has_ub) {   // moving walls: -2 t rho e.u_b / c_s^2 on incoming directions
        rA = fma(__ldg(v.wub + (int64_t)A * R + slot), rh_node, rA);
        rB = fma(__ldg(v.wub + (int64_t)B * R + slot), rh_node, rB);
      }
    }
    // node-major partials: the pair's two values side by side (one 16-byte store)
    reinterpret_cast<double2*>(r + idx * (Q - 1))[decltype(RR)::value] = make_double2(rA, rB);
  });
}

// a5: element-local right-hand side of the force-split streaming (Sec. 3.3) for
// element batch eb: stage its tiles, then rhs_compute.  For the
// opposite-velocity pairs [pr0, pr1) of the velocity set when SPLIT (all pairs
// otherwise); a pair's two values do not depend on which other pairs a CTA
// computes, so splitting the pairs over CTAs gives the same bits
template <class L, int NP, int EPB, bool SPLIT = false>
__device__ __forceinline__ void body_rhs(const View& v, const double* __restrict__ gst, int eb,
                                         double* sm, int pr0 = 0, int pr1 = L::NREP,
                                         bool bulk = false) {
  constexpr int D = L::D, Q = L::Q, NL = ipow(NP, D), NT = EPB * NL;
  const int64_t V = v.V;
  const int E = v.E;
  const double* __restrict__ Dmat = v.Dm;
  double* sD = sm;
  double* sr = sD + NP * NP;
  double* smu = sr + NT;
  double* sg = smu + NT;   // [Q-1][NT], moving directions only
  const int e0 = eb * EPB;
  const int count = min(EPB, E - e0) * NL;
  const int64_t base = (int64_t)e0 * NL;
  for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sD[i] = __ldg(Dmat + i);
  if constexpr (!SPLIT) {   // rho, mu and the Q-1 moving velocities
    stage_tiles(bulk, Q + 1, count, [&](int t, double*& dst, const double*& src) {
      if (t == 0) { dst = sr; src = v.rho + base; }
      else if (t == 1) { dst = smu; src = v.mu + base; }
      else { dst = sg + (t - 2) * NT; src = gst + (t - 1) * V + base; }
    }, v.flags);
  } else {
    stage_in(sr, v.rho, base, count);
    stage_in(smu, v.mu, base, count);
#pragma unroll 1
    for (int p = pr0; p < pr1; ++p) {
      const int A = L::rep(p), B = L::opp(A);
      stage_in(sg + (A - 1) * NT, gst + A * V, base, count);
      stage_in(sg + (B - 1) * NT, gst + B * V, base, count);
    }
  }
  __syncthreads();
  rhs_compute<L, NP, EPB, SPLIT>(v, sD, sr, smu, sg, count, base, pr0, pr1);
}

// SSP-RK3 stage value from the base state u0, the current stage state gc and
// sq = DSS(r_q) (imdt = dt / M_g); the rest population (q = 0) has L = 0
template <int STAGE>
__device__ __forceinline__ double rk_update(int q, double sq, double imdt, double u0, double gc) {
  if constexpr (STAGE == 1) {
    return (q > 0) ? fma(sq, imdt, u0) : u0;
  } else if constexpr (STAGE == 2) {
    const double base = fma(0.25, gc, 0.75 * u0);
    return (q > 0) ? fma(sq, 0.25 * imdt, base) : base;
  } else {
    const double base = fma(2.0 / 3.0, gc, u0 * (1.0 / 3.0));
    return (q > 0) ? fma(sq, (2.0 / 3.0) * imdt, base) : base;
  }
}

// copies of a global node whose local indices a gather-scatter thread loads up
// front, so that the loads of all its copies are in flight together (a vertex
// of a hex mesh has 8 copies); further copies are read in a loop
constexpr int kCopiesAhead = 8;

__device__ __forceinline__ void load_copies(const int* __restrict__ idx, int j0, int nc,
                                            int (&ic)[kCopiesAhead]) {
#pragma unroll
  for (int c = 0; c < kCopiesAhead; ++c) ic[c] = (c < nc) ? idx[j0 + c] : 0;
}

// a5 (part 2): DSS of the right-hand side, M^-1, and the SSP-RK3 stage update
//   stage 1: U1 = U0 + dt L;  stage 2: U2 = 3/4 U0 + 1/4 (U1 + dt L);
//   stage 3: f^{n+1} = 1/3 U0 + 2/3 (U2 + dt L); rho of the new state
// gcur and out may be the same array (stage 2 updates the stage state in
// place): each group reads all its values before writing any, so the pointers
// are deliberately not restrict-qualified
template <class L, int STAGE>
__device__ __forceinline__ void body_dss_rk(const View& v, const double* gcur, double* out,
                                            int g) {
  constexpr int Q = L::Q, NR = L::NREP;
  if (g >= v.G) return;
  const int64_t V = v.V;
  const int* __restrict__ off = v.off;
  const int* __restrict__ idx = v.idx;
  const double2* __restrict__ r2 = reinterpret_cast<const double2*>(v.r);
  const double* __restrict__ U0 = v.fs;
  double* __restrict__ rho = v.rho;
  const int j0 = off[g], j1 = off[g + 1];
  const int nc = j1 - j0;
  // the local indices of the first kCopiesAhead copies, in one round trip
  int ic[kCopiesAhead];
  load_copies(idx, j0, nc, ic);
  const int i0 = ic[0];
  const double imdt = __ldg(v.invMg + g) * v.dt;   // dt L = dt DSS(r) / M_g
  // DSS(r): the partials are node-major, pair p of a node at r2[node NR + p]
  // (values of rep(p) and its opposite), summed copy by copy in the group's
  // fixed order
  double sa[NR], sb[NR];
#pragma unroll
  for (int p = 0; p < NR; ++p) {
    const double2 t = r2[(int64_t)i0 * NR + p];
    sa[p] = t.x;
    sb[p] = t.y;
  }
#pragma unroll
  for (int c = 1; c < kCopiesAhead; ++c) {
    if (c < nc) {
#pragma unroll
      for (int p = 0; p < NR; ++p) {
        const double2 t = r2[(int64_t)ic[c] * NR + p];
        sa[p] += t.x;
        sb[p] += t.y;
      }
    }
  }
  for (int j = j0 + kCopiesAhead; j < j1; ++j) {
    const int ii = idx[j];
#pragma unroll
    for (int p = 0; p < NR; ++p) {
      const double2 t = r2[(int64_t)ii * NR + p];
      sa[p] += t.x;
      sb[p] += t.y;
    }
  }
  double val[Q];
  val[0] = 0.0;   // the rest population does not stream
  static_for<0, NR>([&](auto P) {
    constexpr int A = L::rep(decltype(P)::value), B = L::opp(A);
    val[A] = sa[decltype(P)::value];
    val[B] = sb[decltype(P)::value];
  });
  double rs = 0.0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    val[q] = rk_update<STAGE>(q, val[q], imdt, U0[q * V + i0], gcur[q * V + i0]);
    rs += val[q];
  }
  if (nonfinite(rs)) atomicOr(v.flags + 1, 1);
#pragma unroll
  for (int c = 0; c < kCopiesAhead; ++c) {
    if (c < nc) {
      const int ii = ic[c];
#pragma unroll
      for (int q = 0; q < Q; ++q) out[q * V + ii] = val[q];
      rho[ii] = rs;
    }
  }
  for (int j = j0 + kCopiesAhead; j < j1; ++j) {
    const int ii = idx[j];
#pragma unroll
    for (int q = 0; q < Q; ++q) out[q * V + ii] = val[q];
    rho[ii] = rs;
  }
}

// resident CTAs per SM the streaming kernel is compiled for (register cap)
// (four CTAs of up to 256 threads, 72 registers; larger tiles keep the
// compiler's choice)
template <int D, int NP, int EPB>
constexpr int rhs_min_blocks() {
  return cta_threads<D, NP, EPB>() <= 256 ? 4 : 1;
}

// ---------------------------------------------------------------------------
// single-solve kernels: one CTA per element batch / one thread per node group
// ---------------------------------------------------------------------------
template <class L, int NP, int EPB>
__global__ void __launch_bounds__(cta_threads<L::D, NP, EPB>())
    k_lap(View v, const double* __restrict__ rho, double* __restrict__ out,
          double* __restrict__ drho) {
  extern __shared__ double sm[];
  pdl_wait();
  body_lap<L, NP, EPB>(v, rho, out, drho, blockIdx.x, sm);   // one tile: the load loop
  pdl_trigger();
}

static __global__ void k_dss_mu(View v, const double* __restrict__ lapr, const double* __restrict__ rho,
                         double* __restrict__ mu) {
  pdl_wait();
  body_dss_mu(v, lapr, rho, mu, blockIdx.x * blockDim.x + threadIdx.x);
  pdl_trigger();
}

template <class L, int NP, int EPB>
__global__ void __launch_bounds__(cta_threads<L::D, NP, EPB>()) k_force(View v) {
  extern __shared__ double sm[];
  pdl_wait();
  body_force<L, NP, EPB>(v, blockIdx.x, sm);   // two tiles: the load loop
  pdl_trigger();
}

template <class L>
__global__ void k_dss_collide(View v) {
  pdl_wait();
  body_dss_collide<L>(v, blockIdx.x * blockDim.x + threadIdx.x);
  pdl_trigger();
}

template <class L, int NP, int EPB, bool SPLIT>
__global__ void __launch_bounds__(cta_threads<L::D, NP, EPB>(), rhs_min_blocks<L::D, NP, EPB>())
    k_rhs(View v, const double* __restrict__ gst) {
  // SPLIT: the velocity pairs of each element batch are spread over gridDim.y
  // CTAs (meshes too small to fill the GPU with one CTA per element batch)
  extern __shared__ __align__(128) double sm[];
  pdl_wait();
  if constexpr (SPLIT) {
    const int P = gridDim.y, y = blockIdx.y;
    body_rhs<L, NP, EPB, true>(v, gst, blockIdx.x, sm, y * L::NREP / P, (y + 1) * L::NREP / P);
  } else {
    body_rhs<L, NP, EPB>(v, gst, blockIdx.x, sm, 0, L::NREP, true);   // one element batch: bulk staging
  }
  pdl_trigger();
}

template <class L, int STAGE>
__global__ void k_dss_rk(View v, const double* gcur, double* out) {
  pdl_wait();
  body_dss_rk<L, STAGE>(v, gcur, out, blockIdx.x * blockDim.x + threadIdx.x);
  pdl_trigger();
}

// ---------------------------------------------------------------------------
// batched persistent kernels: a fixed grid loops over a device-resident work
// list of (slot, element batch) or (slot, node-group chunk) items; the slot
// table and the list live in device memory, so solves can join or leave a
// batch between launches without re-capturing the CUDA graph
// ---------------------------------------------------------------------------
struct WorkItem {
  int slot, unit;
};

template <class L, int NP, int EPB>
__global__ void __launch_bounds__(cta_threads<L::D, NP, EPB>())
    kb_lap(const View* __restrict__ slots, const WorkItem* __restrict__ items,
           const int* __restrict__ count) {
  extern __shared__ double sm[];
  pdl_wait();
  const int n = *count;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const WorkItem it = items[w];
    const View& v = slots[it.slot];
    body_lap<L, NP, EPB>(v, v.rho, v.lapr, v.drho, it.unit, sm);
    __syncthreads();
  }
  pdl_trigger();
}

template <class L>
__global__ void kb_dss_mu(const View* __restrict__ slots, const WorkItem* __restrict__ items,
                          const int* __restrict__ count) {
  pdl_wait();
  const int n = *count;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const WorkItem it = items[w];
    const View& v = slots[it.slot];
    body_dss_mu(v, v.lapr, v.rho, v.mu, it.unit * blockDim.x + threadIdx.x);
  }
  pdl_trigger();
}

template <class L, int NP, int EPB>
__global__ void __launch_bounds__(cta_threads<L::D, NP, EPB>())
    kb_force(const View* __restrict__ slots, const WorkItem* __restrict__ items,
             const int* __restrict__ count) {
  extern __shared__ double sm[];
  pdl_wait();
  const int n = *count;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const WorkItem it = items[w];
    body_force<L, NP, EPB>(slots[it.slot], it.unit, sm);
    __syncthreads();
  }
  pdl_trigger();
}

template <class L>
__global__ void kb_dss_collide(const View* __restrict__ slots, const WorkItem* __restrict__ items,
                               const int* __restrict__ count) {
  pdl_wait();
  const int n = *count;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const WorkItem it = items[w];
    body_dss_collide<L>(slots[it.slot], it.unit * blockDim.x + threadIdx.x);
  }
  pdl_trigger();
}

template <class L, int NP, int EPB>
__global__ void __launch_bounds__(cta_threads<L::D, NP, EPB>(), rhs_min_blocks<L::D, NP, EPB>())
    kb_rhs(const View* __restrict__ slots, const WorkItem* __restrict__ items,
           const int* __restrict__ count, int from_fs) {
  extern __shared__ double sm[];
  pdl_wait();
  const int n = *count;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const WorkItem it = items[w];
    const View& v = slots[it.slot];
    body_rhs<L, NP, EPB>(v, from_fs ? v.fs : v.g, it.unit, sm);
    __syncthreads();
  }
  pdl_trigger();
}

template <class L, int STAGE>
__global__ void kb_dss_rk(const View* __restrict__ slots, const WorkItem* __restrict__ items,
                          const int* __restrict__ count) {
  pdl_wait();
  const int n = *count;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const WorkItem it = items[w];
    const View& v = slots[it.slot];
    const double* gcur = (STAGE == 1) ? v.fs : v.g;
    double* out = (STAGE == 3) ? v.f : v.g;
    body_dss_rk<L, STAGE>(v, gcur, out, it.unit * blockDim.x + threadIdx.x);
  }
  pdl_trigger();
}

// a6: diagnostics (Sec. 3.3 KE_max), deterministic two-pass reduction
struct DiagPart {
  double mass, ke_int, ke_max, u2max, rho_min, rho_max, nonfinite;
};

__device__ __forceinline__ void diag_combine(DiagPart& a, const DiagPart& b) {
  a.mass += b.mass;
  a.ke_int += b.ke_int;
  a.ke_max = fmax(a.ke_max, b.ke_max);
  a.u2max = fmax(a.u2max, b.u2max);
  a.rho_min = fmin(a.rho_min, b.rho_min);
  a.rho_max = fmax(a.rho_max, b.rho_max);
  a.nonfinite += b.nonfinite;
}

// momentum sum_a C_a f_a (lattice units) from the opposite pairs: the
// difference f_A - f_B once per pair, then only the non-zero components of C_A
// (an add or subtract for unit ones, an fma for phi): B300 retires two FP64
// operations per SM per cycle, so multiplying by zeros is not free
template <class L>
__device__ __forceinline__ void pair_momentum(const double* fa, double* m) {
#pragma unroll
  for (int c = 0; c < L::D; ++c) m[c] = 0.0;
  static_for<0, L::NREP>([&](auto RR) {
    constexpr int A = L::rep(decltype(RR)::value), B = L::opp(A);
    const double d = fa[A] - fa[B];
    static_for<0, L::D>([&](auto CC) {
      constexpr int c = decltype(CC)::value;
      constexpr double w = L::C(A, c);
      if constexpr (w == 1.0) m[c] += d;
      else if constexpr (w == -1.0) m[c] -= d;
      else if constexpr (w != 0.0) m[c] = fma(w, d, m[c]);
    });
  });
}

template <class L>
__global__ void k_diag(const double* __restrict__ f, const double* __restrict__ Me,
                       DiagPart* __restrict__ part, int64_t V) {
  constexpr int D = L::D, Q = L::Q;
  __shared__ DiagPart sh[256];
  DiagPart p = {0.0, 0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    double fa[Q];
    int bad = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      fa[q] = f[q * V + i];
      bad += nonfinite(fa[q]) ? 1 : 0;
    }
    double rh = fa[0];
#pragma unroll
    for (int q = 1; q < Q; ++q) rh += fa[q];
    double m[D];
    pair_momentum<L>(fa, m);
    // |u|^2 = S^2 |m|^2 / rho^2 and KE = rho |u|^2 / 2, with one division
    double m2 = m[0] * m[0];
#pragma unroll
    for (int c = 1; c < D; ++c) m2 = fma(m[c], m[c], m2);
    const double inv = L::S / rh;
    const double u2 = m2 * inv * inv;
    const double ke = 0.5 * rh * u2;
    const double me = Me[i];
    p.mass = fma(me, rh, p.mass);
    p.ke_int = fma(me, ke, p.ke_int);
    p.ke_max = fmax(p.ke_max, ke);
    p.u2max = fmax(p.u2max, u2);
    p.rho_min = fmin(p.rho_min, rh);
    p.rho_max = fmax(p.rho_max, rh);
    if (bad) p.nonfinite += bad;
  }
  sh[threadIdx.x] = p;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) diag_combine(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// the per-block partials combined in a fixed order: thread t folds partials
// t, t + T, t + 2T, ... in turn, then a fixed tree over the T threads.  The
// result does not depend on scheduling, and the work is spread over the
// threads (one thread folding the 1,184 partials of a 884,736-node mesh in
// turn took 0.4 ms)
constexpr int kCombineThreads = 128;

template <class P, class F>
__device__ __forceinline__ void combine_fixed_order(const P* __restrict__ part, int n,
                                                    P* __restrict__ out, F combine) {
  __shared__ P sh[kCombineThreads];
  const int t = threadIdx.x;
  if (t < n) {
    P a = part[t];
    for (int i = t + kCombineThreads; i < n; i += kCombineThreads) combine(a, part[i]);
    sh[t] = a;
  }
  __syncthreads();
  const int m = min(n, kCombineThreads);
  for (int s = kCombineThreads / 2; s > 0; s >>= 1) {
    if (t < s && t + s < m) combine(sh[t], sh[t + s]);
    __syncthreads();
  }
  if (t == 0) *out = sh[0];
}

static __global__ void __launch_bounds__(kCombineThreads)
    k_diag_final(const DiagPart* __restrict__ part, int n, DiagPart* __restrict__ out) {
  combine_fixed_order(part, n, out, [](DiagPart& a, const DiagPart& b) { diag_combine(a, b); });
}

// ---------------------------------------------------------------------------
// contact-angle measurement (Sec. 3.1, 3.2): moments of the liquid fraction
// phi = (rho - rho_v)/(rho_l - rho_v) over the domain (GLL mass quadrature; the
// copies of a shared node together carry its assembled mass) and over the wall
// faces of one tag (face quadrature w |a|); per-block partials combined in a
// fixed order, so the result does not depend on scheduling
// ---------------------------------------------------------------------------
struct WetPart {
  double vol, vx[3], wall, wet, wx[3];
  double mv, rv, ml, rl;   // mass and mass-weighted rho of nodes with phi < 0.02 / phi > 0.98
};

template <class L>
__global__ void k_wet(const double* __restrict__ f, const double* __restrict__ Me,
                      const double* __restrict__ xyz, const int* __restrict__ rec_elem,
                      const int* __restrict__ rec_node, const int* __restrict__ rec_mask,
                      const int* __restrict__ rec_tag, const double* __restrict__ wsf, int R,
                      int tag, int NL, double rho_v, double inv_drho, WetPart* __restrict__ part,
                      int64_t V) {
  constexpr int D = L::D, Q = L::Q;
  __shared__ WetPart sh[256];
  WetPart p = {};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += stride) {
    double rh = 0.0;
    for (int q = 0; q < Q; ++q) rh += f[q * V + i];
    const double phi = (rh - rho_v) * inv_drho;
    const double me = Me[i];
    const double m = me * phi;
    p.vol += m;
    for (int c = 0; c < D; ++c) p.vx[c] += m * xyz[i * D + c];
    if (phi < 0.02) {
      p.mv += me;
      p.rv += me * rh;
    } else if (phi > 0.98) {
      p.ml += me;
      p.rl += me * rh;
    }
  }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += stride) {
    const int64_t i = (int64_t)rec_elem[r] * NL + rec_node[r];
    const int mask = rec_mask[r];
    double rh = 0.0;
    for (int q = 0; q < Q; ++q) rh += f[q * V + i];
    const double phi = (rh - rho_v) * inv_drho;
    for (int fc = 0; fc < 2 * D; ++fc) {
      if (!((mask >> fc) & 1) || (tag >= 0 && rec_tag[r * 2 * D + fc] != tag)) continue;
      const double w = wsf[r * 2 * D + fc];
      p.wall += w;
      p.wet += w * phi;
      for (int c = 0; c < D; ++c) p.wx[c] += w * phi * xyz[i * D + c];
    }
  }
  sh[threadIdx.x] = p;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      WetPart& a = sh[threadIdx.x];
      const WetPart& b = sh[threadIdx.x + s];
      a.vol += b.vol;
      a.wall += b.wall;
      a.wet += b.wet;
      for (int c = 0; c < 3; ++c) {
        a.vx[c] += b.vx[c];
        a.wx[c] += b.wx[c];
      }
      a.mv += b.mv;
      a.rv += b.rv;
      a.ml += b.ml;
      a.rl += b.rl;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

static __global__ void __launch_bounds__(kCombineThreads)
    k_wet_final(const WetPart* __restrict__ part, int n, WetPart* __restrict__ out) {
  combine_fixed_order(part, n, out, [](WetPart& a, const WetPart& b) {
    a.vol += b.vol;
    a.wall += b.wall;
    a.wet += b.wet;
    for (int c = 0; c < 3; ++c) {
      a.vx[c] += b.vx[c];
      a.wx[c] += b.wx[c];
    }
    a.mv += b.mv;
    a.rv += b.rv;
    a.ml += b.ml;
    a.rl += b.rl;
  });
}

// initial state fbar = t_a rho (f^eq at u = 0)
template <class L>
__global__ void k_init(const double* __restrict__ rho_in, double* __restrict__ f,
                       double* __restrict__ rho, int64_t V) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V) return;
  const double r = rho_in[i];
  rho[i] = r;
  for (int q = 0; q < L::Q; ++q) f[q * V + i] = L::t(q) * r;
}

// rho = sum_a fbar_a (after set_state)
template <class L>
__global__ void k_density(const double* __restrict__ f, double* __restrict__ rho, int64_t V) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V) return;
  double s = 0.0;
  for (int q = 0; q < L::Q; ++q) s += f[q * V + i];
  rho[i] = s;
}

// u = sum_a fbar_a e_a / rho, [D][V]
template <class L>
__global__ void k_velocity(const double* __restrict__ f, double* __restrict__ u, int64_t V) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V) return;
  double rh = 0.0;
  for (int q = 0; q < L::Q; ++q) rh += f[q * V + i];
  for (int a = 0; a < L::D; ++a) {
    double m = 0.0;
    for (int q = 1; q < L::Q; ++q) m += L::C(q, a) * f[q * V + i];
    u[a * V + i] = m * L::S / rh;
  }
}

}  // namespace semlbm
