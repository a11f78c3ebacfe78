/*
 * sem_lbm.h - C ABI of the B300 (sm_103a) FP64 spectral element lattice
 * Boltzmann step for non-ideal gases with partial wetting.
 *
 * The method is that of "Spectral element lattice Boltzmann method for
 * non-ideal gases with partial wetting boundary condition" (Zhao, Patel, Lee):
 *   - chemical potential mu = mu0(rho) - kappa lap(rho), Eq. (chemi), with the
 *     Laplacian in the weak form of Eq. (weak) whose wall integral carries the
 *     wetting gradient n.grad(rho) = cos(theta) sqrt(2 e0/kappa) (Sec. 2.2);
 *   - BGK collision with the higher-order force F** (Sec. 2.1, Appendix A);
 *   - SSP-RK3 streaming in the weak form Eq. (advection)/(spetrum), force-split
 *     as in Sec. 3.3, with the flux bounce-back wall flux J (Sec. 2.2, Eq. 9);
 *   - direct-stiffness summation (gather-scatter) of every element-local
 *     contribution across shared GLL nodes.
 *
 * Conventions common to every call
 *   - Every function returns SEMLBM_OK (0) or a negative SEMLBM_E* code and,
 *     on error, leaves a message readable with sem_lbm_last_error() (per
 *     calling thread).  No call aborts the process.
 *   - All floating-point data is IEEE binary64.
 *   - Element-local node order: k = i + n j (+ n^2 l), n = N+1, i along the
 *     first reference axis (fastest).  Faces: f = 2 b + s, b = reference axis,
 *     s = 0 for xi_b = -1 and 1 for xi_b = +1.
 *   - Field layout: scalar fields [E][n^d]; the state fbar [Q][E][n^d]
 *     (structure of arrays per velocity).  Shared nodes are stored once per
 *     element; the library keeps the copies equal.
 *   - Velocity order.  D2Q9: 0 rest, 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1),
 *     5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1); weights 4/9, 1/9, 1/36.
 *     D3Q13: 0 rest, then s*(0,1,phi), s*(0,-1,phi), s*(1,phi,0),
 *     s*(-1,phi,0), s*(phi,0,1), s*(phi,0,-1) and e_{a+6} = -e_a, with
 *     phi the golden ratio and |e| = sqrt(5/3); weights 2/5 and 1/20.
 *     D3Q19: 0 rest, 1-3 (1,0,0) (0,1,0) (0,0,1), 4-9 (1,1,0) (1,-1,0) (1,0,1)
 *     (1,0,-1) (0,1,1) (0,1,-1), e_{a+9} = -e_a; weights 1/3, 1/18, 1/36.
 *     D3Q27: as D3Q19 for 1-9, then 10-13 (1,1,1) (1,1,-1) (1,-1,1) (1,-1,-1),
 *     e_{a+13} = -e_a; weights 8/27, 2/27, 1/54, 1/216.
 *     c_s^2 = 1/3 for all.
 *   - Calls on one solver are not thread safe; distinct solvers are
 *     independent.  Work is enqueued on the solver's stream (params.stream,
 *     else a stream the solver owns).
 *   - A solver (and a batch) lives on the device that was current when it was
 *     created.  Every later call makes that device current for its own
 *     duration and restores the caller's current device before returning, so
 *     callers that switch devices need not switch back first.
 */
#ifndef SEM_LBM_H
#define SEM_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SEMLBM_OK = 0,
  SEMLBM_EINVAL = -1,      /* bad argument (null pointer, size, range, state) */
  SEMLBM_ENOMEM = -2,      /* device memory or caller workspace too small     */
  SEMLBM_ECUDA = -3,       /* a CUDA runtime call failed                       */
  SEMLBM_ENONFINITE = -4,  /* the state holds NaN/Inf (diagnostics status)      */
  SEMLBM_ETIMEOUT = -5,    /* a bounded device-side wait gave up                */
  SEMLBM_EUNSUPPORTED = -6 /* order N or lattice/dimension pair not built       */
};

typedef enum {
  SEMLBM_D2Q9 = 0,   /* 2D, Sec. 2.1                                        */
  SEMLBM_D3Q13 = 1,  /* 3D, Sec. 3.2 (rest + icosahedron)                   */
  SEMLBM_D3Q19 = 2,  /* 3D cubic, faces + edges                             */
  SEMLBM_D3Q27 = 3   /* 3D cubic, faces + edges + corners                   */
} sem_lbm_lattice;

/* Mesh (host memory; copied by sem_lbm_create, the caller keeps ownership).
 *   node_xyz  [n_elem][(N+1)^dim][dim]  GLL node coordinates of each element
 *             (isoparametric: geometry order = N).  Elements must have a
 *             positive Jacobian at every node.
 *   global_id [n_elem][(N+1)^dim]  equal ids <=> the same mesh node (periodic
 *             gluing is expressed by equal ids).  Any int64 values.
 *   face_kind [n_elem][2 dim]  0 interior or periodic, 1 wall.
 *   face_tag  [n_elem][2 dim]  wall contact-angle tag: < 0 neutral wall
 *             (90 degrees), 0 -> theta_w, k >= 1 -> params->theta_tag[k-1]. */
typedef struct {
  int dim;
  int64_t n_elem;
  const double* node_xyz;
  const int64_t* global_id;
  const uint8_t* face_kind;
  const int32_t* face_tag;
} sem_lbm_mesh;

/* Optional parameters; a zeroed struct (or a NULL pointer) gives defaults. */
typedef struct {
  double rho_l, rho_v;    /* phase densities (0 -> 1.0 and 0.1; Appendix A)       */
  double dt;              /* time step; <= 0 -> min(cfl h_min / max|e_alpha|,
                             0.1 h_min^2 / sqrt(rho_l kappa)), h_min the smallest
                             distance between neighbouring GLL nodes              */
  double cfl;             /* used when dt <= 0; 0 -> 0.4                            */
  double mu0_factor;      /* mu0 = factor*beta(rho-rl)(rho-rv)(2rho-rl-rv); 0 -> 2  */
  int n_tags;             /* entries in theta_tag                                   */
  const double* theta_tag;/* contact angles (radians) of wall tags 1..n_tags        */
  void* stream;           /* cudaStream_t to run on; NULL -> solver-owned stream    */
  void* workspace;        /* caller device memory (e.g. from PyTorch) or NULL       */
  size_t workspace_bytes; /* its size; must be >= sem_lbm_workspace_bytes()         */
  const double* wall_velocity; /* [n_tags + 1][dim]: velocity u_b of the walls with
                             tag 0..n_tags, entering the flux bounce-back term
                             -2 t_a rho e_a.u_b / c_s^2 (Sec. 2.2); NULL = static.
                             Walls with tag < 0 are static.                          */
  int force_split;        /* which force enters F** of the collision (Sec. 2.1):
                             0 = F = c_s^2 grad rho - rho grad mu, as printed;
                             1 = its potential part -rho grad mu alone.  The two
                             have the same equilibria (F** vanishes at u = 0);
                             with 0, long runs of isolated drops develop a growing
                             mode whose rate per unit time falls with dt, with 1
                             they stay bounded.  Other values: SEMLBM_EINVAL.      */
} sem_lbm_params;

typedef struct sem_lbm sem_lbm_t;

typedef struct {
  int64_t step;       /* completed time steps                                  */
  double time;        /* step * dt                                             */
  double mass;        /* sum_e sum_i M_e,i rho_i (integral of rho)             */
  double ke_max;      /* max over nodes of 0.5 rho |u|^2 (Sec. 3.3)           */
  double ke_int;      /* integral of 0.5 rho |u|^2                             */
  double umax;        /* max |u|                                               */
  double rho_min, rho_max;
  int64_t n_nonfinite;/* non-finite entries of fbar                            */
  int status;         /* SEMLBM_OK, SEMLBM_ENONFINITE, or SEMLBM_ETIMEOUT when a
                         streaming kernel's bounded wait for its bulk-copied tiles
                         gave up (the step's results are then not valid)      */
} sem_lbm_diag;

typedef struct {
  int dim, N, Q;
  int64_t n_elem, n_local;   /* n_local = n_elem (N+1)^dim                     */
  int64_t n_global;          /* distinct global nodes                           */
  int64_t n_wall_nodes;      /* element-local nodes on a wall face              */
  double dt, kappa, beta, tau;
  size_t workspace_bytes;
  int graph_launches;        /* 1 if steps replay a captured CUDA graph         */
  int kernels_per_step;      /* kernel launches in one time step                */
  int elements_per_cta;      /* elements per CTA of the element kernels         */
  int rhs_pair_groups;       /* CTAs that share the velocity pairs of one element
                                batch in the streaming right-hand side: 1 = one
                                CTA per element batch (meshes that fill the GPU),
                                > 1 = the pair-split form for small meshes      */
  int graph_pdl;             /* 1 once the captured step launches each kernel after
                                the first as a programmatic dependent of the one
                                before (its launch overlaps the predecessor's end;
                                its data accesses still follow it), 0 otherwise  */
} sem_lbm_info_t;

/* Device bytes sem_lbm_create needs for this mesh (for admission control and
 * for callers that pass their own workspace).  0 on invalid input. */
size_t sem_lbm_workspace_bytes(const sem_lbm_mesh* mesh, int N, sem_lbm_lattice lattice);

/* Build a solver: validates the mesh, builds GLL tables, the gather-scatter
 * map and the wall records on the host, uploads the mesh and computes the
 * geometry (Jacobians, metrics, masses, wall area vectors) in kernels.
 *   N        polynomial order: 2..16 for D2Q9, 2..8 for the 3D sets
 *   beta     bulk free-energy coefficient of e0 = beta (rho-rl)^2 (rho-rv)^2
 *   kappa    gradient-energy coefficient (Appendix A: beta delta^2 (rl-rv)^2/8)
 *   tau      relaxation time in units of dt; collision rate 1/(tau + 1/2)
 *   theta_w  contact angle (radians, measured through the liquid) of tag 0
 * The state is undefined until sem_lbm_set_density or sem_lbm_set_state. */
int sem_lbm_create(const sem_lbm_mesh* mesh, int N, sem_lbm_lattice lattice, double beta,
                   double kappa, double tau, double theta_w, const sem_lbm_params* params,
                   sem_lbm_t** out);

/* fbar = f^eq(rho, u = 0) = t_alpha rho (Appendix A initial state).
 * rho [n_elem][(N+1)^dim]; copies of a shared node must be equal. */
int sem_lbm_set_density(sem_lbm_t* s, const double* rho, int rho_on_device);

/* Advance n_steps >= 0 full time steps (collision + 3 SSP-RK3 stages).
 * Asynchronous on the solver's stream; returns the launch status. */
int sem_lbm_step(sem_lbm_t* s, int64_t n_steps);

/* Reduce the diagnostics of the current state (synchronises the stream). */
int sem_lbm_diagnostics(sem_lbm_t* s, sem_lbm_diag* out);

/* Moments of the liquid fraction phi = (rho - rho_v)/(rho_l - rho_v) of the
 * current state, from which the static contact angle of a drop is measured
 * (Sec. 3.1 and 3.2 measure it on the equilibrium cap; the paper states no
 * procedure).  On a flat wall the cap's liquid volume and wetted base give the
 * angle (paper_2609_00535_b300/wetting.py).  Volume integrals use the GLL mass
 * quadrature, wall integrals the face quadrature w |a| of the wetting term. */
typedef struct {
  double volume;          /* int phi dV (an area in 2D)                              */
  double centroid[3];     /* int phi x dV / volume (components >= dim are 0)          */
  double wall;            /* int dS over the selected wall faces (a length in 2D)     */
  double wetted;          /* int phi dS over the selected wall faces                  */
  double wet_centroid[3]; /* int phi x dS / wetted (0 when wetted == 0)               */
  double rho_v_ref, rho_l_ref; /* the reference densities that defined phi            */
} sem_lbm_wetting;

/* tag >= 0 selects the wall faces with that tag, tag < 0 every wall face.
 * rho_v_ref, rho_l_ref: the phase densities that define phi.  A drop in a closed
 * domain settles with both phases off rho_v and rho_l (its Laplace pressure and
 * the conserved mass shift them), and the vapour filling the domain then adds
 * to int phi dV; pass the bulk densities, or a value <= 0 for either to have
 * them measured: phi is first taken on the state's density range [min, max],
 * and the references become the mass-weighted mean densities of the nodes
 * with phi < 0.02 (vapour) and phi > 0.98 (liquid).  Runs its kernels on the
 * solver's stream and synchronises it; the reduction order is fixed, so
 * repeated calls give the same bits.  Errors: SEMLBM_EINVAL (NULL argument,
 * state not set, rho_l_ref <= rho_v_ref), SEMLBM_ECUDA. */
int sem_lbm_wetting_moments(sem_lbm_t* s, int tag, double rho_v_ref, double rho_l_ref,
                            sem_lbm_wetting* out);

/* Copy a field out.  which: 0 fbar [Q][E][n^d], 1 rho [E][n^d],
 * 2 u [dim][E][n^d], 3 mu [E][n^d] (of the last computed stage-1 state).
 * dst is host memory unless dst_on_device; host copies synchronise. */
int sem_lbm_get_field(sem_lbm_t* s, int which, double* dst, int dst_on_device);

/* Checkpoint: fbar [Q][E][n^d] plus the step counter. */
int sem_lbm_get_state(sem_lbm_t* s, double* fbar, int on_device, int64_t* step);
int sem_lbm_set_state(sem_lbm_t* s, const double* fbar, int on_device, int64_t step);

/* Compact checkpoint: fbar on the mesh's global nodes, [Q][G] with
 * G = sem_lbm_info_t.n_global, one value per node instead of one per element
 * copy.  The copies of a shared node are equal after every step (the direct
 * stiffness summation of Sec. 2.2 writes one value to all of them), so the
 * compact state carries the whole state in G/V of the bytes (0.6 on hex meshes
 * at N = 5).  Nodes are in the library's node-group order:
 * sem_lbm_get_global_nodes gives, for each, the element-local index (into
 * [E][n^d]) of its first copy, so mesh.global_id[first_copy[g]] names node g.
 *   get: reads each node's first copy into fbar_g (device memory when on_device,
 *        else host memory; a host copy synchronises the stream).  Errors:
 *        SEMLBM_EINVAL (NULL argument, state not set), SEMLBM_ECUDA.
 *   set: writes value [q][g] to every copy of node g, recomputes rho and sets
 *        the step counter; a host source is copied (and the stream synchronised)
 *        before the call returns, a device source is read in stream order on the
 *        solver's stream.  The library keeps no pointer to either buffer.
 *        Errors: SEMLBM_EINVAL (NULL argument), SEMLBM_ECUDA.
 *   get_global_nodes: fills first_copy[G] (host memory, caller-owned). */
int sem_lbm_get_state_global(sem_lbm_t* s, double* fbar_g, int on_device, int64_t* step);
int sem_lbm_set_state_global(sem_lbm_t* s, const double* fbar_g, int on_device, int64_t step);
int sem_lbm_get_global_nodes(const sem_lbm_t* s, int64_t* first_copy);

int sem_lbm_get_info(const sem_lbm_t* s, sem_lbm_info_t* out);

/* Per-kernel device timing, for measurement.  While enabled, sem_lbm_step
 * issues the step's kernels directly (not as a graph replay) and records a
 * CUDA event on the solver's stream after each launch, so that consecutive
 * events bracket exactly one kernel.  sem_lbm_profile_read synchronises the
 * stream and returns, per kernel class, the summed milliseconds and launch
 * counts recorded since the last read (or since enabling), then resets them.
 * Classes: 0 k_lap (weak Laplacian), 1 k_dss_mu (gather-scatter + mu),
 * 2 k_force, 3 k_dss_collide (force average + collision), 4 k_rhs (streaming
 * right-hand side), 5 k_dss_rk (gather-scatter + SSP-RK3 update). */
#define SEMLBM_N_KERNEL_CLASSES 6
typedef struct {
  double ms[8];
  int64_t launches[8];
  double total_ms;    /* first to last event */
} sem_lbm_profile_t;

int sem_lbm_profile(sem_lbm_t* s, int enable);
int sem_lbm_profile_read(sem_lbm_t* s, sem_lbm_profile_t* out);

/* Allocation-free chemical potential.  Computes mu = mu0(rho) - kappa lap(rho)
 * for a caller-supplied density field on this solver's mesh, like
 * sem_lbm_get_field(s, 3, ...), but without using any device memory beyond
 * what already exists: the element-local Laplacian partials (the one piece of
 * scratch this computation needs) live in a fixed array compiled into the
 * library, not in the solver workspace, and the call performs no cudaMalloc,
 * cudaFree or other allocation.  It is meant for callers that must not
 * allocate device memory while they run: serving loops that reserve every
 * byte at admission time (an allocation there can fail or stall under memory
 * pressure), and programs whose device memory is owned by another allocator
 * (a raw cudaMalloc would bypass its accounting).  The paper has no
 * counterpart; this is an integration feature.
 *   rho  device pointer, [n_elem][(N+1)^dim], copies of shared nodes equal
 *   mu   device pointer, same layout, written at every copy
 * Runs on the solver's stream and returns without synchronising.
 * Limit: n_elem (N+1)^dim <= SEMLBM_NOALLOC_MAX_NODES; larger meshes are
 * rejected with SEMLBM_EINVAL.  The array (8 MiB) is held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call reuses
 * the same array: each call overwrites all entries it reads, so nothing
 * carries over between calls, but calls whose work overlaps on the GPU (other
 * streams, other solvers, other host threads) race on it and must be
 * serialised by the caller. */
#define SEMLBM_NOALLOC_MAX_NODES (1 << 20)
int sem_lbm_chemical_potential_noalloc(sem_lbm_t* s, const double* rho, double* mu);

/* ---------------------------------------------------------------------------
 * Batches: many independent solves (uneven meshes, orders, angles) advanced
 * together.  The paper runs one solve at a time; batching serves its parameter
 * sweeps (contact angles, geometries).
 *
 * A batch owns no solve: sem_lbm_batch_add takes a created, initialised
 * solver and steps it (sem_lbm_step on it then fails) until it is removed.
 * While a member, the solver's calls run on the batch's stream.  Solves are
 * grouped by (velocity set, N), N <= 8; one batch step replays one CUDA graph
 * whose branches are the groups' persistent kernels over device-resident slot
 * tables, so adding or removing a member between steps does not re-capture it.
 * Each member computes exactly the same bits as it would alone.
 * --------------------------------------------------------------------------- */
typedef struct sem_lbm_batch sem_lbm_batch_t;

typedef struct {
  int lattice, N, n_members, epb;     /* epb: elements per CTA in use          */
  int64_t elem_items, node_items;     /* work-list lengths                      */
  int grid_elem, grid_node;           /* persistent grid sizes                  */
  int capture_failures;               /* batch steps run as direct launches     */
  int n_candidates;                   /* tile shapes the tuner can choose from  */
  int candidate_epb[4];
  double candidate_ms[4];             /* measured ms per step (0 until tuned)   */
} sem_lbm_batch_group_info;

/* stream: cudaStream_t or NULL for a batch-owned stream. */
int sem_lbm_batch_create(void* stream, sem_lbm_batch_t** out);
/* The stream the batch steps on (the one given to sem_lbm_batch_create, or the
 * batch's own when that was NULL); NULL for a NULL batch.  A batch captures its
 * step into a CUDA graph on this stream, so no other thread may use the stream
 * meanwhile: give each batch a stream of its own. */
void* sem_lbm_batch_stream(const sem_lbm_batch_t* b);
/* Adds s (state set, same device, N <= 8); returns its slot index. */
int sem_lbm_batch_add(sem_lbm_batch_t* b, sem_lbm_t* s, int* slot);
/* Removes the solver in `slot` (after the batch's pending work). */
int sem_lbm_batch_remove(sem_lbm_batch_t* b, int slot);
/* Advances every member n_steps full steps (asynchronous). */
int sem_lbm_batch_step(sem_lbm_batch_t* b, int64_t n_steps);
/* Autotuner: for each group and every compiled tile shape, runs one warm-up
 * step (drained before timing) and two timed runs of steps_per_candidate - 1
 * (>= 1) real steps, and keeps the shape with the fastest run (remembered for
 * later groups of the same velocity set, N and size in this process).  All
 * shapes give identical results; the tuning steps (2 steps_per_candidate - 1
 * per shape) advance the members like any step. */
int sem_lbm_batch_tune(sem_lbm_batch_t* b, int steps_per_candidate);
/* Diagnostics of slots 0..n-1 (one synchronisation); empty slots get
 * step = -1 and status = SEMLBM_EINVAL. */
int sem_lbm_batch_diagnostics(sem_lbm_batch_t* b, sem_lbm_diag* out, int n);
int sem_lbm_batch_info(sem_lbm_batch_t* b, sem_lbm_batch_group_info* out, int max_groups,
                       int* n_groups);
/* Slot of a solver in its batch, or -1. */
int sem_lbm_batch_slot_of(const sem_lbm_t* s);
/* Removes every member (returning them to their own streams) and frees the batch. */
void sem_lbm_batch_destroy(sem_lbm_batch_t* b);

/* Releases device memory the solver allocated (never the caller's workspace)
 * and the stream it owns, after removing it from its batch.  NULL is ignored. */
void sem_lbm_destroy(sem_lbm_t* s);

/* Message of the calling thread's last failed call ("" if none). */
const char* sem_lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_LBM_H */
