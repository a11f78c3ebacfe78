"""Thin Python binding of libsemlbm (ctypes): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
only fills the C structs of ``include/sem_lbm.h``, hands PyTorch device memory
and a PyTorch stream to the library, and converts errors into exceptions.  It
fails loudly when the shared library is missing: there is no fallback.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsemlbm.so")

D2Q9, D3Q13, D3Q19, D3Q27 = 0, 1, 2, 3
LATTICES = {"D2Q9": D2Q9, "D3Q13": D3Q13, "D3Q19": D3Q19, "D3Q27": D3Q27}
Q_OF = {D2Q9: 9, D3Q13: 13, D3Q19: 19, D3Q27: 27}

ERRORS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "EUNSUPPORTED"}

EXPORTED = ["sem_lbm_workspace_bytes", "sem_lbm_create", "sem_lbm_set_density", "sem_lbm_step",
            "sem_lbm_diagnostics", "sem_lbm_wetting_moments", "sem_lbm_get_field", "sem_lbm_get_state", "sem_lbm_set_state",
            "sem_lbm_get_state_global", "sem_lbm_set_state_global", "sem_lbm_get_global_nodes",
            "sem_lbm_get_info", "sem_lbm_destroy", "sem_lbm_last_error", "sem_lbm_profile",
            "sem_lbm_profile_read", "sem_lbm_chemical_potential_noalloc",
            "sem_lbm_batch_create", "sem_lbm_batch_add", "sem_lbm_batch_remove",
            "sem_lbm_batch_step", "sem_lbm_batch_tune", "sem_lbm_batch_diagnostics",
            "sem_lbm_batch_info", "sem_lbm_batch_slot_of", "sem_lbm_batch_stream",
            "sem_lbm_batch_destroy"]
NOALLOC_MAX_NODES = 1 << 20
KERNEL_CLASSES = ["k_lap", "k_dss_mu", "k_force", "k_dss_collide", "k_rhs", "k_dss_rk"]
PEAK_PATH = os.path.join(_HERE, "libsemlbm_peak.so")


class SemLbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class MeshC(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_elem", ctypes.c_int64), ("node_xyz", ctypes.c_void_p),
                ("global_id", ctypes.c_void_p), ("face_kind", ctypes.c_void_p),
                ("face_tag", ctypes.c_void_p)]


class ParamsC(ctypes.Structure):
    _fields_ = [("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double), ("dt", ctypes.c_double),
                ("cfl", ctypes.c_double), ("mu0_factor", ctypes.c_double),
                ("n_tags", ctypes.c_int), ("theta_tag", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("wall_velocity", ctypes.c_void_p),
                ("force_split", ctypes.c_int)]


class WettingC(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_double), ("centroid", ctypes.c_double * 3),
                ("wall", ctypes.c_double), ("wetted", ctypes.c_double),
                ("wet_centroid", ctypes.c_double * 3), ("rho_v_ref", ctypes.c_double),
                ("rho_l_ref", ctypes.c_double)]


class DiagC(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("time", ctypes.c_double), ("mass", ctypes.c_double),
                ("ke_max", ctypes.c_double), ("ke_int", ctypes.c_double),
                ("umax", ctypes.c_double), ("rho_min", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("n_nonfinite", ctypes.c_int64),
                ("status", ctypes.c_int)]


class ProfileC(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8),
                ("total_ms", ctypes.c_double)]


class InfoC(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("N", ctypes.c_int), ("Q", ctypes.c_int),
                ("n_elem", ctypes.c_int64), ("n_local", ctypes.c_int64),
                ("n_global", ctypes.c_int64), ("n_wall_nodes", ctypes.c_int64),
                ("dt", ctypes.c_double), ("kappa", ctypes.c_double), ("beta", ctypes.c_double),
                ("tau", ctypes.c_double), ("workspace_bytes", ctypes.c_size_t),
                ("graph_launches", ctypes.c_int), ("kernels_per_step", ctypes.c_int),
                ("elements_per_cta", ctypes.c_int), ("rhs_pair_groups", ctypes.c_int),
                ("graph_pdl", ctypes.c_int)]


class GroupInfoC(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("N", ctypes.c_int), ("n_members", ctypes.c_int),
                ("epb", ctypes.c_int), ("elem_items", ctypes.c_int64),
                ("node_items", ctypes.c_int64), ("grid_elem", ctypes.c_int),
                ("grid_node", ctypes.c_int), ("capture_failures", ctypes.c_int),
                ("n_candidates", ctypes.c_int),
                ("candidate_epb", ctypes.c_int * 4), ("candidate_ms", ctypes.c_double * 4)]


_lib = None


def load():
    """Load libsemlbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsemlbm.so is missing at %s; build it with "
                           "paper_2609_00535_b300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    L.sem_lbm_workspace_bytes.argtypes = [ctypes.POINTER(MeshC), I, I]
    L.sem_lbm_workspace_bytes.restype = SZ
    L.sem_lbm_create.argtypes = [ctypes.POINTER(MeshC), I, I, D, D, D, D, ctypes.POINTER(ParamsC),
                                 ctypes.POINTER(P)]
    L.sem_lbm_create.restype = I
    L.sem_lbm_set_density.argtypes = [P, P, I]
    L.sem_lbm_step.argtypes = [P, I64]
    L.sem_lbm_diagnostics.argtypes = [P, ctypes.POINTER(DiagC)]
    L.sem_lbm_wetting_moments.argtypes = [P, I, D, D, ctypes.POINTER(WettingC)]
    L.sem_lbm_get_field.argtypes = [P, I, P, I]
    L.sem_lbm_get_state.argtypes = [P, P, I, ctypes.POINTER(I64)]
    L.sem_lbm_set_state.argtypes = [P, P, I, I64]
    L.sem_lbm_get_state_global.argtypes = [P, P, I, ctypes.POINTER(I64)]
    L.sem_lbm_set_state_global.argtypes = [P, P, I, I64]
    L.sem_lbm_get_global_nodes.argtypes = [P, P]
    L.sem_lbm_get_info.argtypes = [P, ctypes.POINTER(InfoC)]
    L.sem_lbm_destroy.argtypes = [P]
    L.sem_lbm_destroy.restype = None
    L.sem_lbm_last_error.restype = ctypes.c_char_p
    L.sem_lbm_profile.argtypes = [P, I]
    L.sem_lbm_profile_read.argtypes = [P, ctypes.POINTER(ProfileC)]
    L.sem_lbm_chemical_potential_noalloc.argtypes = [P, P, P]
    L.sem_lbm_chemical_potential_noalloc.restype = I
    L.sem_lbm_batch_create.argtypes = [P, ctypes.POINTER(P)]
    L.sem_lbm_batch_add.argtypes = [P, P, ctypes.POINTER(I)]
    L.sem_lbm_batch_remove.argtypes = [P, I]
    L.sem_lbm_batch_step.argtypes = [P, I64]
    L.sem_lbm_batch_tune.argtypes = [P, I]
    L.sem_lbm_batch_diagnostics.argtypes = [P, ctypes.POINTER(DiagC), I]
    L.sem_lbm_batch_info.argtypes = [P, ctypes.POINTER(GroupInfoC), I, ctypes.POINTER(I)]
    L.sem_lbm_batch_slot_of.argtypes = [P]
    L.sem_lbm_batch_stream.argtypes = [P]
    L.sem_lbm_batch_stream.restype = P
    L.sem_lbm_batch_destroy.argtypes = [P]
    L.sem_lbm_batch_destroy.restype = None
    for name in ("sem_lbm_batch_create", "sem_lbm_batch_add", "sem_lbm_batch_remove",
                 "sem_lbm_batch_step", "sem_lbm_batch_tune", "sem_lbm_batch_diagnostics",
                 "sem_lbm_batch_info", "sem_lbm_batch_slot_of"):
        getattr(L, name).restype = I
    for name in ("sem_lbm_set_density", "sem_lbm_step", "sem_lbm_diagnostics", "sem_lbm_get_field",
                 "sem_lbm_get_state", "sem_lbm_set_state", "sem_lbm_get_info", "sem_lbm_profile",
                 "sem_lbm_profile_read", "sem_lbm_get_state_global", "sem_lbm_set_state_global",
                 "sem_lbm_get_global_nodes"):
        getattr(L, name).restype = I
    _lib = L
    return L


def fp64_peak_tflops(device=0, iters=20000):
    """Measured FP64 FMA throughput of the GPU (TFLOP/s) and the probe's duration."""
    if not os.path.exists(PEAK_PATH):
        raise RuntimeError("libsemlbm_peak.so is missing; run paper_2609_00535_b300.build.build()")
    P = ctypes.CDLL(PEAK_PATH)
    P.semlbm_fp64_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
    t, ms = ctypes.c_double(), ctypes.c_double()
    rc = P.semlbm_fp64_peak(device, iters, ctypes.byref(t), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError("semlbm_fp64_peak failed (%d)" % rc)
    return t.value, ms.value


def check(rc):
    if rc != 0:
        raise SemLbmError(rc, load().sem_lbm_last_error().decode())
    return rc


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def mesh_struct(mesh):
    """Contiguous copies of the mesh arrays and the C struct pointing at them."""
    keep = (np.ascontiguousarray(mesh.node_xyz, dtype=np.float64),
            np.ascontiguousarray(mesh.global_id, dtype=np.int64),
            np.ascontiguousarray(mesh.face_kind, dtype=np.uint8),
            np.ascontiguousarray(mesh.face_tag, dtype=np.int32))
    m = MeshC(mesh.dim, mesh.n_elem, keep[0].ctypes.data, keep[1].ctypes.data,
              keep[2].ctypes.data, keep[3].ctypes.data)
    return m, keep


def workspace_bytes(mesh, N, lattice):
    m, keep = mesh_struct(mesh)
    return int(load().sem_lbm_workspace_bytes(ctypes.byref(m), N, LATTICES.get(lattice, lattice)))


class Solver:
    """One SEM-LBM solve on one GPU: create / set_density / step / diagnostics."""

    def __init__(self, mesh, lattice, beta, kappa, tau, theta_w, theta_tag=(), rho_l=1.0,
                 rho_v=0.1, dt=0.0, cfl=0.0, mu0_factor=0.0, stream=None, device=0,
                 wall_velocity=None, force_split=0):
        import torch
        L = load()
        self.lattice = LATTICES.get(lattice, lattice)
        self.Q = Q_OF[self.lattice]
        self.mesh = mesh
        self.N = mesh.N
        self.dim = mesh.dim
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        m, keep = mesh_struct(mesh)
        nbytes = int(L.sem_lbm_workspace_bytes(ctypes.byref(m), self.N, self.lattice))
        if nbytes == 0:
            raise SemLbmError(-1, L.sem_lbm_last_error().decode())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._tags = np.ascontiguousarray(np.asarray(theta_tag, dtype=np.float64).reshape(-1))
        self._ub = None
        if wall_velocity:   # {tag: u_b} for tags 0..len(theta_tag)
            self._ub = np.zeros((len(self._tags) + 1, self.dim))
            for tag, u in dict(wall_velocity).items():
                if 0 <= int(tag) <= len(self._tags):
                    self._ub[int(tag)] = u
        p = ParamsC(rho_l, rho_v, dt, cfl, mu0_factor, len(self._tags),
                    self._tags.ctypes.data if len(self._tags) else None,
                    self.stream.cuda_stream, self.workspace.data_ptr(), nbytes,
                    self._ub.ctypes.data if self._ub is not None else None, int(force_split))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(L.sem_lbm_create(ctypes.byref(m), self.N, self.lattice, beta, kappa, tau,
                                   theta_w, ctypes.byref(p), ctypes.byref(h)))
        self.h = h
        self.info = self.get_info()
        self.V = self.info["n_local"]

    @classmethod
    def from_case(cls, case, **kw):
        kw.setdefault("wall_velocity", getattr(case, "wall_velocity", None))
        kw.setdefault("force_split", getattr(case, "force_split", 0))
        return cls(case.mesh, case.lattice, case.beta, case.kappa, case.tau, case.theta_w,
                   case.theta_tag, case.rho_l, case.rho_v, dt=case.dt, **kw)

    # -- state -------------------------------------------------------------
    def set_density(self, rho):
        import torch
        if isinstance(rho, torch.Tensor):
            assert rho.dtype == torch.float64 and rho.is_contiguous() and rho.numel() == self.V
            self.stream.wait_stream(torch.cuda.current_stream(rho.device))
            check(load().sem_lbm_set_density(self.h, ctypes.c_void_p(rho.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
            assert a.size == self.V
            check(load().sem_lbm_set_density(self.h, _ptr(a), 0))

    def set_state(self, fbar, step=0):
        import torch
        if isinstance(fbar, torch.Tensor):
            assert fbar.dtype == torch.float64 and fbar.is_contiguous()
            assert fbar.numel() == self.Q * self.V
            if fbar.is_cuda:
                self.stream.wait_stream(torch.cuda.current_stream(fbar.device))
                check(load().sem_lbm_set_state(self.h, ctypes.c_void_p(fbar.data_ptr()), 1, step))
            else:   # host memory (pinned for full-speed copies)
                check(load().sem_lbm_set_state(self.h, ctypes.c_void_p(fbar.data_ptr()), 0, step))
        else:
            a = np.ascontiguousarray(fbar, dtype=np.float64).reshape(-1)
            assert a.size == self.Q * self.V
            check(load().sem_lbm_set_state(self.h, _ptr(a), 0, step))

    def set_state_global(self, fbar_g, step=0):
        """Compact state [Q, G] on the global nodes (sem_lbm_set_state_global), in
        the order of global_nodes(); a CUDA tensor, a host tensor (pinned for
        full-speed copies) or a numpy array."""
        import torch
        n = self.Q * self.info["n_global"]
        if isinstance(fbar_g, torch.Tensor):
            assert fbar_g.dtype == torch.float64 and fbar_g.is_contiguous() and fbar_g.numel() == n
            if fbar_g.is_cuda:
                self.stream.wait_stream(torch.cuda.current_stream(fbar_g.device))
                check(load().sem_lbm_set_state_global(self.h, ctypes.c_void_p(fbar_g.data_ptr()),
                                                      1, step))
            else:
                check(load().sem_lbm_set_state_global(self.h, ctypes.c_void_p(fbar_g.data_ptr()),
                                                      0, step))
        else:
            a = np.ascontiguousarray(fbar_g, dtype=np.float64).reshape(-1)
            assert a.size == n
            check(load().sem_lbm_set_state_global(self.h, _ptr(a), 0, step))

    def get_state_global(self, out=None):
        """(fbar on the global nodes [Q, G], step); into a CUDA tensor when out is given."""
        step = ctypes.c_int64()
        if out is not None:
            import torch
            assert isinstance(out, torch.Tensor) and out.dtype == torch.float64 and out.is_cuda
            assert out.is_contiguous() and out.numel() == self.Q * self.info["n_global"]
            check(load().sem_lbm_get_state_global(self.h, ctypes.c_void_p(out.data_ptr()), 1,
                                                  ctypes.byref(step)))
            torch.cuda.current_stream(out.device).wait_stream(self.stream)
            return out, step.value
        a = np.empty((self.Q, self.info["n_global"]), dtype=np.float64)
        check(load().sem_lbm_get_state_global(self.h, _ptr(a), 0, ctypes.byref(step)))
        return a, step.value

    def global_nodes(self):
        """Element-local index of each global node's first copy, [G] int64: node g
        of the compact state is mesh.global_id[global_nodes()[g]]."""
        a = np.empty(self.info["n_global"], dtype=np.int64)
        check(load().sem_lbm_get_global_nodes(self.h, _ptr(a)))
        return a

    def step(self, n=1):
        check(load().sem_lbm_step(self.h, int(n)))

    def diagnostics(self):
        d = DiagC()
        check(load().sem_lbm_diagnostics(self.h, ctypes.byref(d)))
        return {k: getattr(d, k) for k, _ in DiagC._fields_}

    def wetting_moments(self, tag=0, rho_v=0.0, rho_l=0.0):
        """Liquid-fraction moments of the current state (sem_lbm_wetting_moments):
        volume, centroid, wall, wetted, wet_centroid; tag < 0 = every wall;
        rho_v / rho_l <= 0: the state's bulk phase densities define phi."""
        w = WettingC()
        check(load().sem_lbm_wetting_moments(self.h, int(tag), float(rho_v), float(rho_l),
                                             ctypes.byref(w)))
        return {"volume": w.volume, "centroid": list(w.centroid)[:self.dim], "wall": w.wall,
                "wetted": w.wetted, "wet_centroid": list(w.wet_centroid)[:self.dim],
                "rho_v_ref": w.rho_v_ref, "rho_l_ref": w.rho_l_ref}

    def field(self, which, out=None):
        """which: 'fbar' [Q,V], 'rho' [V], 'u' [dim,V], 'mu' [V]; numpy, or into a CUDA tensor."""
        import torch
        code = {"fbar": 0, "rho": 1, "u": 2, "mu": 3}[which]
        shape = {"fbar": (self.Q, self.V), "rho": (self.V,), "u": (self.dim, self.V),
                 "mu": (self.V,)}[which]
        if out is not None:
            assert isinstance(out, torch.Tensor) and out.dtype == torch.float64
            check(load().sem_lbm_get_field(self.h, code, ctypes.c_void_p(out.data_ptr()), 1))
            torch.cuda.current_stream(out.device).wait_stream(self.stream)
            return out
        a = np.empty(shape, dtype=np.float64)
        check(load().sem_lbm_get_field(self.h, code, _ptr(a), 0))
        return a

    def get_state(self):
        a = np.empty((self.Q, self.V), dtype=np.float64)
        step = ctypes.c_int64()
        check(load().sem_lbm_get_state(self.h, _ptr(a), 0, ctypes.byref(step)))
        return a, step.value

    def get_info(self):
        i = InfoC()
        check(load().sem_lbm_get_info(self.h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in InfoC._fields_}

    def profile(self, enable=True):
        """Per-kernel CUDA-event timing of subsequent steps (see sem_lbm_profile)."""
        check(load().sem_lbm_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        p = ProfileC()
        check(load().sem_lbm_profile_read(self.h, ctypes.byref(p)))
        return {"ms": {k: p.ms[i] for i, k in enumerate(KERNEL_CLASSES)},
                "launches": {k: p.launches[i] for i, k in enumerate(KERNEL_CLASSES)},
                "total_ms": p.total_ms}

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None):
            load().sem_lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several solves stepped together (see sem_lbm_batch_* in sem_lbm.h)."""

    def __init__(self, stream=None, device=0):
        # without a caller stream the batch uses one the library creates for it:
        # torch's pooled streams repeat, and a solver built on another thread on
        # the same stream would collide with the batch's graph capture
        import torch
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(load().sem_lbm_batch_create(stream.cuda_stream if stream is not None else None,
                                              ctypes.byref(h)))
        self.h = h
        self.stream = stream if stream is not None else torch.cuda.ExternalStream(
            load().sem_lbm_batch_stream(h), device=self.device)
        self.members = {}

    def add(self, solver):
        slot = ctypes.c_int()
        check(load().sem_lbm_batch_add(self.h, solver.h, ctypes.byref(slot)))
        self.members[slot.value] = solver
        solver.batch = self
        return slot.value

    def remove(self, slot):
        check(load().sem_lbm_batch_remove(self.h, int(slot)))
        s = self.members.pop(slot)
        s.batch = None
        return s

    def step(self, n=1):
        check(load().sem_lbm_batch_step(self.h, int(n)))

    def tune(self, steps_per_candidate=3):
        check(load().sem_lbm_batch_tune(self.h, int(steps_per_candidate)))

    def diagnostics(self):
        n = max(self.members) + 1 if self.members else 0
        arr = (DiagC * max(n, 1))()
        check(load().sem_lbm_batch_diagnostics(self.h, arr, n))
        return {i: {k: getattr(arr[i], k) for k, _ in DiagC._fields_} for i in self.members}

    def info(self):
        arr = (GroupInfoC * 32)()
        ng = ctypes.c_int()
        check(load().sem_lbm_batch_info(self.h, arr, 32, ctypes.byref(ng)))
        out = []
        for i in range(min(ng.value, 32)):
            g = arr[i]
            out.append({"lattice": g.lattice, "N": g.N, "n_members": g.n_members, "epb": g.epb,
                        "elem_items": g.elem_items, "node_items": g.node_items,
                        "grid_elem": g.grid_elem, "grid_node": g.grid_node,
                        "capture_failures": g.capture_failures,
                        "candidates": [(g.candidate_epb[c], g.candidate_ms[c])
                                       for c in range(g.n_candidates)]})
        return out

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None):
            load().sem_lbm_batch_destroy(self.h)
            for s in self.members.values():
                s.batch = None
            self.members = {}
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
