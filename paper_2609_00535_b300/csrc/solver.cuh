// Private to libsemlbm: the solver object shared by the single-solve C ABI
// (sem_lbm.cu) and the batch engine (batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "kernels.cuh"
#include "sem_lbm.h"

namespace semlbm {

// records a message for sem_lbm_last_error() and returns code
int fail(int code, const char* fmt, ...);

constexpr int kDssThreads = 128;   // threads per CTA of the gather-scatter kernels

inline int grid_of(int64_t work, int threads) { return (int)((work + threads - 1) / threads); }

// Launches a kernel, optionally as a programmatic dependent launch: the kernel
// may then be scheduled while the previous kernel on the stream finishes, and
// it waits for that kernel's completion (and the visibility of its writes) in
// pdl_wait() before touching any data (kernels.cuh).  Inside a captured graph
// the dependency becomes a programmatic edge.
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                   cudaStream_t stream, bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Makes `device` current for the lifetime of the guard and restores the
// caller's device afterwards, so that a call on a solver or batch launches on
// the device the object was created on, whatever device the caller has current.
class DeviceGuard {
 public:
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev_) == cudaSuccess && prev_ != device && cudaSetDevice(device) == cudaSuccess)
      switched_ = true;
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;

 private:
  int prev_ = 0;
  bool switched_ = false;
};

}  // namespace semlbm

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return semlbm::fail(SEMLBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));           \
  } while (0)

struct sem_lbm_batch;

struct sem_lbm {
  int D, N, n, NL, Q, EPB;
  int device = 0;
  sem_lbm_lattice lat;
  int64_t E, V, G, R;
  double beta, kappa, tau, theta_w, rho_l, rho_v, dt, mu0f;
  int force_split;   // 0: F** from c_s^2 grad rho - rho grad mu; 1: -rho grad mu
  cudaStream_t stream;
  bool own_stream = false;
  void* ws = nullptr;
  bool own_ws = false;
  size_t ws_bytes = 0;
  // device arrays
  double *f, *fs, *g, *r, *rho, *mu, *lapr, *Fp, *drho, *MJ, *Gm, *Me, *invMg, *xyz, *Dm, *wg;
  double* CJ = nullptr;   // stored pair coefficients of the streaming kernel (D3Q13)
  int *off, *idx, *slot, *rec_elem, *rec_node, *rec_mask, *flags;
  double *wet, *ae, *rec_cos, *rec_ub, *wub;
  int* rec_tag;                         // [R][2D] wall tag per face (-1: not a wall face)
  double* wsf;                          // [R][2D] face quadrature weight w |a|
  semlbm::WetPart *wparts, *wout;       // wetting-moment partials
  bool moving = false;   // some wall has a non-zero velocity
  semlbm::DiagPart *parts, *dout;
  int diag_blocks = 0;
  int n_sm = 148;                       // SMs of the device (grid sizing)
  bool state_ready = false;
  int64_t step = 0;
  semlbm::View view{};                   // device pointers + parameters, for the kernels
  cudaGraphExec_t graph = nullptr;
  int kernels_per_step = 0;
  bool prof_on = false;
  bool pdl = false;                     // launch the step's kernels as programmatic dependents
  bool graph_pdl = false;               // the captured step has programmatic edges
  sem_lbm_batch* batch = nullptr;     // set while a batch steps this solver
  cudaStream_t home_stream = nullptr; // the solver's own stream while it is in a batch
  std::vector<int> first_copy;   // [G] element-local index of each node group's first copy
  std::vector<cudaEvent_t> ev;   // event pool; ev[0..nev) recorded since the last read
  std::vector<int> ev_cls;       // class of the kernel that ends at ev[i] (i >= 1)
  size_t nev = 0;
  struct Ops* ops = nullptr;
};

struct Ops {
  void (*geom)(sem_lbm&);
  void (*wall)(sem_lbm&);
  void (*lap)(sem_lbm&);
  void (*mu)(sem_lbm&);
  void (*force)(sem_lbm&);
  void (*rhs)(sem_lbm&, const double* g);
  void (*collide)(sem_lbm&);
  void (*rk)(sem_lbm&, int stage, const double* gcur, double* out);
  void (*diag)(sem_lbm&);
  void (*init)(sem_lbm&, const double* rho);
  void (*density)(sem_lbm&);
  void (*velocity)(sem_lbm&, double* u);
  int (*prepare)();
  void (*lap_into)(sem_lbm&, const double* rho, double* partial);
  void (*mu_from)(sem_lbm&, const double* partial, const double* rho, double* mu);
  void (*wet)(sem_lbm&, int tag, double rho_v_ref, double rho_l_ref);
  int (*rhs_split)(const sem_lbm&);   // CTAs sharing one element batch's velocity pairs
  int epb;                            // elements per CTA of the element kernels
};

