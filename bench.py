#!/usr/bin/env python
"""Benchmark: FP64 GLL node-updates/s of the SEM-LBM wetting step on B300.

One "step" is one full time step of the method (collision + three SSP-RK3
streaming stages, every kernel of the hot path) over the whole mesh.  Default
workload: the 3D droplet on a sphere-cap wall, 16^3 curved hexes, N = 5,
D3Q13, 884,736 element-local GLL nodes (synthetic mesh and tanh-initialised
density; the paper's GMSH meshes are not available).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun each rank advances its own independent solve (the paper's
sweeps are independent problems): weak scaling, no collective on the data
path; the timing is bracketed by barriers and the max over ranks is taken.
Prints one JSON line on rank 0.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_00535_b300 import flops as flopcount  # noqa: E402
from paper_2609_00535_b300 import inputs  # noqa: E402

import hashlib  # noqa: E402

METRIC = "FP64 GLL node-updates/s (3D droplet)"

# DRAM traffic of one k_rhs launch from an ncu capture of the 12^3-hex
# sphere-cap mesh at N = 5 (373,248 nodes: 108.96 MB read + 8.81 MB written, the
# mean of two launches); the traffic grows with the node count, so it is scaled
# per node.  Valid only while the kernel sources are the ones profiled.
RHS_TRAFFIC = {"kernels.cuh": "323819fc1b0f7d76", "lattice.cuh": "5fa95228ce9be598",
               "bytes_per_node": (108.96e6 + 8.81e6) / 373248, "lattice": "D3Q13", "N": 5}


def rhs_traffic_per_launch(lattice, N, n_local):
    csrc = os.path.join(ROOT, "paper_2609_00535_b300", "csrc")
    for name in ("kernels.cuh", "lattice.cuh"):
        h = hashlib.sha256(open(os.path.join(csrc, name), "rb").read()).hexdigest()[:16]
        if h != RHS_TRAFFIC[name]:
            return None
    if (lattice, N) != (RHS_TRAFFIC["lattice"], RHS_TRAFFIC["N"]):
        return None
    return RHS_TRAFFIC["bytes_per_node"] * n_local


UNIT = "node-updates/s"
L2_BYTES = 126 * 2 ** 20


def make_case(name, ne=None):
    if name == "sphere3d":
        return inputs.sphere_3d(ne=(ne, ne, ne)) if ne else inputs.sphere_3d()
    if name == "flat2d":
        return inputs.flat_wall_2d()
    if name == "cylinder2d":
        return inputs.cylinder_2d()
    raise SystemExit("unknown config %s" % name)


def sample_case(name):
    """Bounded sample of the workload for the CPU oracle: same mesh family, N,
    velocity set and parameters, fewer elements."""
    if name == "sphere3d":
        return inputs.sphere_3d(ne=(4, 4, 4)), "sphere-cap mesh 4x4x4 elements, N=5, D3Q13 (13,824 nodes)"
    if name == "flat2d":
        return inputs.flat_wall_2d(), "the full 1,600-node mesh"
    return inputs.cylinder_2d(n_theta=16, n_r=4), "cylinder O-grid 16x4 elements, N=6"


def max_over_ranks(x, device=None):
    """Max of a float over all ranks (identity at world size 1)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, seconds_per_rank, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / max_over_ranks(seconds_per_rank)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock and throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def oracle_rate(case, steps, warmup=0):
    """Time the CPU oracle (as it stands) on a case: node-updates/s, threads."""
    from tests.helpers import oracle_of
    om, orc = oracle_of(case)
    f = orc.initial_state(case.rho0.reshape(om.shape))
    for _ in range(warmup):
        f = orc.step(f)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = orc.step(f)
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = 1
    return case.nodes * steps / dt, dt, cores


def _oracle_worker(job):
    """One host core: the oracle on its own copy of the sample (spawned process)."""
    name, steps = job
    sys.path.insert(0, ROOT)
    case, _ = sample_case(name)
    rate, secs, _ = oracle_rate(case, steps, warmup=1)
    return case.nodes * steps, secs


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_all_cores(name, steps):
    """The oracle as it stands on every host core at once: one independent replica
    of the bounded sample per core (spawned processes, one BLAS thread each);
    throughput = the node-updates of all replicas / the slowest replica's time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(name, steps)] * cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(u for u, _ in res)
    return units / max(t for _, t in res), cores


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    case, what = sample_case(args.config)
    steps = max(1, args.steps)
    rate, secs, cores = oracle_rate(case, steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "%s (oracle sample: %s)" % (args.config, what), "nodes": case.nodes},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d steps of %s" % (steps, what)},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def small_solves(n=64, seed=9):
    """The paper's own problem sizes: the flat-wall drop (8x8 quads, N = 4, 1,600
    nodes) at angles uniform in 15-165 degrees and the isolated periodic drop of
    Sec. 3.3 (4x4 quads, N = 8, 1,296 nodes, force_split 1), half and half."""
    import math
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if i % 2 == 0:
            out.append(inputs.flat_wall_2d(theta=math.radians(rng.uniform(15.0, 165.0))))
        else:
            c = inputs.periodic_droplet(dim=2, ne=4, N=8, D=0.5 * rng.uniform(0.9, 1.1))
            c.force_split = 1
            out.append(c)
    return out


def batched_section(args, device, cases=None):
    """64 solves of uneven E, N and angle: 64 sequential plain solves against one
    autotuned batch (every solve advances the same number of steps in both)."""
    import torch
    from paper_2609_00535_b300 import semlbm
    if cases is None:
        cases = inputs.batch_mix(n=args.batch_solves, seed=4)
    solvers = []
    for c in cases:
        s = semlbm.Solver.from_case(c, device=device)
        s.set_density(c.rho0)
        solvers.append(s)
    nodes = sum(s.info["n_local"] for s in solvers)
    K = args.batch_steps
    for s in solvers:                       # warm-up, graph capture
        s.step(2)
        s.synchronize()
    t0 = time.perf_counter()
    for s in solvers:                       # plain: one solve after the other
        s.step(K)
        s.synchronize()
    t_plain = time.perf_counter() - t0
    b = semlbm.Batch(device=device)
    for s in solvers:
        b.add(s)
    t0 = time.perf_counter()
    b.tune(3)
    t_tune = time.perf_counter() - t0
    b.step(2)
    b.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(b.stream)
    b.step(K)
    e1.record(b.stream)
    b.synchronize()
    t_batch_host = time.perf_counter() - t0
    t_batch = e0.elapsed_time(e1) * 1e-3
    groups = b.info()
    diag = b.diagnostics()
    ok = all(d["status"] == 0 for d in diag.values())
    b.close()
    for s in solvers:
        s.close()
    return {"solves": len(cases), "nodes": nodes, "steps": K,
            "plain_node_updates_per_s": nodes * K / t_plain,
            "batched_node_updates_per_s": nodes * K / t_batch,
            "batched_host_clock_node_updates_per_s": nodes * K / t_batch_host,
            "speedup": t_plain / t_batch, "tune_s": t_tune, "all_finite": ok,
            "groups": [{"lattice": ["D2Q9", "D3Q13"][g["lattice"]], "N": g["N"],
                        "members": g["n_members"], "epb": g["epb"],
                        "candidates": g["candidates"]} for g in groups]}


def serving_section(args, device, capacity):
    """Poisson stream of relaxing requests through the continuous-batching server,
    each run until KE_max < 1e-20 or its step budget: a quarter each of drops on
    a flat wall, a cylinder and the sphere wall of Sec. 3.2, and periodic drops
    (2D/3D); p50/p99 time to a converged answer and the aggregate rate."""
    from paper_2609_00535_b300 import serve
    n = args.serve_requests
    probe = inputs.relaxing_request_stream(n=n, rate=1.0, seed=8)
    nodes = [r.case().nodes for r in probe]
    # mean work per request: its nodes times the mean steps to converge (the
    # kinds' medians, 5e3 to 1.2e5 steps, average about a quarter of the budget)
    work = sum(nodes) / len(nodes) * 0.25 * args.serve_max_steps
    rate = 1.2 * capacity / work              # offered load ~1.2x the measured capacity
    reqs = inputs.relaxing_request_stream(n=n, rate=rate, seed=8)
    srv = serve.Server(hbm_budget_bytes=int(args.serve_budget_gb * 2 ** 30),
                       epoch_steps=args.serve_epoch, ke_tol=1e-20,
                       max_steps=args.serve_max_steps, min_steps=args.serve_epoch)
    st = srv.run(reqs)
    out = st.summary()
    conv = sorted(r.finished - r.arrival for r in st.records if r.converged)
    by_kind = {}
    for q, r in zip(sorted(reqs, key=lambda x: x.arrival), st.records):
        e = by_kind.setdefault(q.kind, {"requests": 0, "converged": 0, "steps": [], "ke_capped": []})
        e["requests"] += 1
        if r.converged:
            e["converged"] += 1
            e["steps"].append(r.steps)
        elif r.ke_max is not None:
            e["ke_capped"].append(r.ke_max)
    for e in by_kind.values():
        st_ = sorted(e.pop("steps"))
        ke = sorted(e.pop("ke_capped"))
        e["median_steps_to_converge"] = st_[len(st_) // 2] if st_ else None
        e["median_ke_when_capped"] = ke[len(ke) // 2] if ke else None
    out.update({"workload": "relaxing requests: drops on a flat wall, a cylinder and a sphere "
                            "wall, periodic drops 2D/3D; E %s, N 4; beta 0.1, force_split 1"
                            % {k: list(v) for k, v in inputs.RELAX_SIZES.items()},
                "by_kind": by_kind,
                "converged_p50_s": conv[len(conv) // 2] if conv else None,
                "converged_p99_s": conv[min(len(conv) - 1, int(round(0.99 * (len(conv) - 1))))]
                if conv else None,
                "arrival_rate_per_s": rate, "offered_load": 1.2, "ke_tol": 1e-20,
                "max_steps": args.serve_max_steps, "epoch_steps": args.serve_epoch,
                "hbm_budget_gb": args.serve_budget_gb})
    return out


def serving_c5_sizes_section(args, device, capacity):
    """Admission and continuous batching at the mesh sizes of the survey's C5
    stream (E log-uniform in [256, 8192], N in 4..7; a quarter each flat wall,
    cylinder, sphere cap and periodic drop 2D/3D), each request capped at a few
    hundred steps: these sizes relax too slowly to run to KE_max < 1e-20 here, so
    this measures admission by HBM budget and throughput under load, not
    time-to-converged."""
    from paper_2609_00535_b300 import serve
    n = args.c5_requests
    probe = inputs.request_stream(n=n, rate=1.0, seed=5)
    nodes = [r.E * (r.N + 1) ** (3 if "3d" in r.kind else 2) for r in probe]
    rate = 1.2 * capacity / (sum(nodes) / len(nodes) * args.c5_steps)
    reqs = inputs.request_stream(n=n, rate=rate, seed=5)
    srv = serve.Server(hbm_budget_bytes=int(args.serve_budget_gb * 2 ** 30), epoch_steps=50,
                       ke_tol=1e-20, max_steps=args.c5_steps, min_steps=50)
    out = srv.run(reqs).summary()
    out.update({"workload": "C5 sizes: E log-uniform in [256, 8192], N 4..7, capped at %d "
                            "steps (admission and throughput, not convergence)" % args.c5_steps,
                "arrival_rate_per_s": rate, "offered_load": 1.2, "max_steps": args.c5_steps,
                "hbm_budget_gb": args.serve_budget_gb})
    return out


def angle_sweep_section(args, device):
    """Contact-angle sweep through the server: drops on a flat wall run until
    KE_max < 1e-20, each started at its equilibrium cap and, as a comparison
    stream with the same angles and sizes, as a half-disc; every converged
    result's angle is measured from the device's wetting moments."""
    import math
    from paper_2609_00535_b300 import serve, wetting
    out = {"workload": "flat-wall drops 2D, 16x8 quads, N 4, beta 0.1, delta 0.1, "
                       "angles 20-100 deg, R 0.225-0.275",
           "requests": args.sweep_requests, "ke_tol": 1e-20, "max_steps": args.sweep_max_steps}
    steps_by = {}
    for init in ("cap", "disc"):
        reqs = inputs.angle_sweep_stream(n=args.sweep_requests, rate=50.0, seed=7,
                                         angles=(20.0, 100.0), init=init)
        srv = serve.Server(hbm_budget_bytes=int(args.serve_budget_gb * 2 ** 30), epoch_steps=1000,
                           ke_tol=1e-20, max_steps=args.sweep_max_steps, min_steps=1000,
                           measure_tag=0)
        st = srv.run(reqs)
        summ = st.summary()
        by = {r.rid: r for r in st.records}
        errs = []
        steps_by[init] = {}
        for q in reqs:
            r = by[q.rid]
            if r.converged and r.moments:
                steps_by[init][q.rid] = r.steps
                try:
                    errs.append(wetting.contact_angle(r.moments, 2, delta=0.1) - math.degrees(q.theta))
                except ValueError:
                    pass
        steps = sorted(steps_by[init].values())
        errs.sort(key=abs)
        out[init] = {"converged": summ["converged"], "capped": summ["capped"],
                     "failed": summ["failed"], "p50_s": summ["p50_s"], "p99_s": summ["p99_s"],
                     "node_updates_per_s": summ["node_updates_per_s"],
                     "median_steps_to_converge": steps[len(steps) // 2] if steps else None,
                     "angle_err_deg_median": errs[len(errs) // 2] if errs else None,
                     "angle_err_deg_max_abs": abs(errs[-1]) if errs else None}
    both = [q for q in steps_by["cap"] if q in steps_by["disc"]]
    if both:
        out["steps_cap_over_disc"] = (sum(steps_by["cap"][q] for q in both)
                                      / sum(steps_by["disc"][q] for q in both))
    return out


def config_lines_section(args, device):
    """Plain single-solve lines of the two 2D workloads: the flat-wall droplet
    (8x8 quads, N = 4, 1,600 nodes) and the droplet on a cylinder (1,024 curved
    quads, N = 6, 50,176 nodes); node-updates/s and the k_rhs FP64 roofline."""
    import torch
    from paper_2609_00535_b300 import semlbm
    peak, _ = semlbm.fp64_peak_tflops(device)
    out = {}
    for name in ("flat2d", "cylinder2d"):
        case = make_case(name)
        s = semlbm.Solver.from_case(case, device=device)
        s.set_density(case.rho0)
        s.step(5)
        s.synchronize()
        K = args.config_steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(K)                            # graph replay, as a user runs it
        e1.record(s.stream)
        s.synchronize()
        ms = e0.elapsed_time(e1)
        s.profile(True)                      # per-kernel events on a second run
        s.step(K)
        prof = s.profile_read()
        s.profile(False)
        info = s.info
        rhs_ms = prof["ms"]["k_rhs"] / max(prof["launches"]["k_rhs"], 1)
        work = flopcount.rhs_work(case.lattice, case.mesh.N, info["n_local"], info["n_wall_nodes"])
        ach = work["flops"] / (rhs_ms * 1e-3) / 1e12
        out[name] = {"mesh": "%d quads, N=%d" % (case.mesh.n_elem, case.mesh.N),
                     "nodes": info["n_local"], "steps": K,
                     "node_updates_per_s": info["n_local"] * K / (ms * 1e-3),
                     "ms_per_step": ms / K, "us_per_step": 1e3 * ms / K,
                     "k_rhs_ms": rhs_ms, "k_rhs_tflops": ach, "k_rhs_frac": ach / peak,
                     "k_rhs_pair_groups": info["rhs_pair_groups"],
                     "status": s.diagnostics()["status"]}
        s.close()
        if not args.no_cpu_baseline:   # the oracle on one core, on the same mesh
            steps = 20 if name == "flat2d" else 4
            rate, secs, _ = oracle_rate(case, steps, warmup=1)
            out[name]["oracle_1core"] = {"node_updates_per_s": rate, "steps": steps,
                                         "seconds": secs}
    return out


def angle_resolution_section(args, device):
    """Static contact angle on a flat wall against the interface width: the drop
    of the angle sweep (area of a half-disc of radius R = 0.25 on the wall y = 0 of
    [0, 2] x [0, 1], beta 0.1, tau 1, started at its equilibrium cap) at
    delta / R = 0.4, 0.2 and 0.1 with delta = 3.2 node spacings (16x8, 32x16 and
    64x32 quads at N = 4), and at delta / R = 0.4 with N = 8 (the same width over
    twice the nodes).  Each solve runs in one batch until KE_max < 1e-14 or its
    step budget; the angle comes from the device wetting moments with the
    diffuse-interface correction (wetting.contact_angle)."""
    import math
    from paper_2609_00535_b300 import semlbm, wetting
    meshes = [(8, 4, 0.1), (16, 4, 0.05), (32, 4, 0.025), (8, 8, 0.1)]
    angles = [float(a) for a in args.angle_study_degrees.split(",")]
    b = semlbm.Batch(device=device)
    live = {}
    for ne, N, delta in meshes:
        for deg in angles:
            c = inputs.cap_on_wall_2d(math.radians(deg), N=N, ne=ne, delta=delta)
            c.force_split = 1
            s = semlbm.Solver.from_case(c, device=device)
            s.set_density(c.rho0)
            live[b.add(s)] = (ne, N, delta, deg, s)
    out = []
    done = 0
    while live and done < args.angle_study_max_steps:
        b.step(args.angle_study_epoch)
        done += args.angle_study_epoch
        diag = b.diagnostics()
        for slot in list(live):
            ne, N, delta, deg, s = live[slot]
            d = diag[slot]
            if d["status"] == 0 and d["ke_max"] >= 1e-14 and done < args.angle_study_max_steps:
                continue
            b.remove(slot)
            row = {"mesh": "%dx%d quads, N=%d" % (2 * ne, ne, N), "delta_over_R": delta / 0.25,
                   "theta_deg": deg, "steps": done, "ke_max": d["ke_max"], "status": d["status"]}
            row["rho_min"], row["rho_max"] = d["rho_min"], d["rho_max"]
            if d["status"] == 0:
                m = s.wetting_moments(0)
                row["volume"], row["wetted"] = m["volume"], m["wetted"]
                try:
                    row["measured_deg"] = wetting.contact_angle(m, 2, delta=delta)
                    row["error_deg"] = row["measured_deg"] - deg
                except ValueError as exc:       # no drop left on the wall
                    row["error"] = str(exc)
            out.append(row)
            s.close()
            del live[slot]
    b.close()
    return out


def angle_kelvin_section(args, device):
    """Static contact angle on a flat wall with and without the Kelvin shift:
    the angle-sweep drop (area of a half-disc of radius 0.25 on the wall y = 0
    of [0, 2] x [0, 1], beta 0.1, tau 1, force_split 1, equilibrium-cap start)
    at 30, 60, 90 and 120 degrees on 16x8 and 32x16 quads at N = 4 (delta / R =
    0.4 and 0.2), started between the bulk densities and between both shifted by
    inputs.kelvin_shift of the cap's radius.  Each solve runs in one batch until
    KE_max < 1e-14 or 3e5 steps; the angle comes from the device wetting moments
    with the diffuse-interface correction."""
    import math
    from paper_2609_00535_b300 import semlbm, wetting
    b = semlbm.Batch(device=device)
    live = {}
    for saturated in (False, True):
        for ne, delta in ((8, 0.1), (16, 0.05)):
            for deg in (30.0, 60.0, 90.0, 120.0):
                c = inputs.cap_on_wall_2d(math.radians(deg), N=4, ne=ne, delta=delta,
                                          saturate=saturated)
                c.force_split = 1
                s = semlbm.Solver.from_case(c, device=device)
                s.set_density(c.rho0)
                live[b.add(s)] = (ne, delta, deg, s, saturated)
    out = []
    done = 0
    while live and done < 300000:
        b.step(2000)
        done += 2000
        diag = b.diagnostics()
        for slot in list(live):
            ne, delta, deg, s, saturated = live[slot]
            d = diag[slot]
            if d["status"] == 0 and d["ke_max"] >= 1e-14 and done < 300000:
                continue
            b.remove(slot)
            m = s.wetting_moments(0)
            row = {"mesh": "%dx%d quads, N=4" % (2 * ne, ne), "delta_over_R": delta / 0.25,
                   "saturated": saturated, "theta_deg": deg, "steps": done,
                   "ke_max": d["ke_max"], "status": d["status"], "area": m["volume"],
                   "wetted": m["wetted"]}
            try:
                row["measured_deg"] = wetting.contact_angle(m, 2, delta=delta)
                row["error_deg"] = row["measured_deg"] - deg
            except ValueError as exc:       # no drop left on the wall
                row["error"] = str(exc)
            out.append(row)
            s.close()
            del live[slot]
    b.close()
    return out


def angle_resolution_3d_section(args, device):
    """Static contact angle on the sphere wall of the Sec. 3.2 box (radius 0.7)
    against the interface width: the relaxing sphere-wall request (drop radius
    0.13 at its equilibrium position, beta 0.1, interface 2.5 node spacings,
    force_split 1, tau from inputs.viscous_tau) on ne^3 curved hexes at N = 4,
    so delta / R = 0.4, 0.3 and 0.2 for ne = 6, 8 and 12.  Each drop starts
    between the bulk densities rho_l, rho_v, and again between the densities
    shifted by inputs.kelvin_shift for its radius ("saturated": the vapour
    already at the density a drop of that size holds at rest, so the drop does
    not evaporate to reach it).  Each solve runs in one batch until
    KE_max < 1e-12 or the step budget; the angle comes from the device wetting
    moments with the sphere-sphere lens geometry."""
    import math
    from paper_2609_00535_b300 import semlbm, wetting
    angles = [float(a) for a in args.angle_study_degrees.split(",")]
    b = semlbm.Batch(device=device)
    live = {}
    for saturated in (False, True):
        for ne in (6, 8, 12):
            for deg in angles:
                c = inputs.relaxing_case("relaxsphere3d", ne ** 3, 4, math.radians(deg),
                                         saturate=saturated)
                s = semlbm.Solver.from_case(c, device=device)
                s.set_density(c.rho0)
                live[b.add(s)] = (ne, c, deg, s, saturated)
    out = []
    done = 0
    while live and done < args.angle_study_3d_max_steps:
        b.step(args.angle_study_epoch)
        done += args.angle_study_epoch
        diag = b.diagnostics()
        for slot in list(live):
            ne, c, deg, s, saturated = live[slot]
            d = diag[slot]
            if d["status"] == 0 and d["ke_max"] >= 1e-12 and done < args.angle_study_3d_max_steps:
                continue
            b.remove(slot)
            delta = c.extra["delta"]
            row = {"mesh": "%d^3 hexes, N=4" % ne, "delta": delta, "delta_over_R": delta / 0.13,
                   "saturated": saturated, "tau": c.tau, "theta_deg": deg, "steps": done,
                   "ke_max": d["ke_max"], "status": d["status"],
                   "rho_min": d["rho_min"], "rho_max": d["rho_max"]}
            if d["status"] == 0:
                m = s.wetting_moments(0)
                row["volume"], row["wetted"] = m["volume"], m["wetted"]
                try:
                    row["measured_deg"] = wetting.contact_angle(m, 3, delta=delta, wall_radius=0.7)
                    row["error_deg"] = row["measured_deg"] - deg
                except ValueError as exc:       # no drop left on the wall
                    row["error"] = str(exc)
                try:   # independent estimate: sphere fitted to the mid-density contour
                    row["contour_deg"] = wetting.contour_angle_on_curved_wall(
                        c.mesh.node_xyz, s.field("rho").reshape(c.mesh.n_elem, -1), 5, 3,
                        (0.25, 0.25, -0.7), 0.7, delta)
                except ValueError as exc:
                    row["contour_error"] = str(exc)
            out.append(row)
            s.close()
            del live[slot]
    b.close()
    return out


def lattice_section(args, device):
    """The sphere workload with the cubic velocity sets D3Q19 and D3Q27 (same mesh,
    N and parameters): node-updates/s and the k_rhs FP64 roofline of each."""
    import torch
    from paper_2609_00535_b300 import semlbm
    peak, _ = semlbm.fp64_peak_tflops(device)
    out = {}
    for lat in ("D3Q19", "D3Q27"):
        case = inputs.sphere_3d(ne=(args.ne,) * 3 if args.ne else (16, 16, 16), lattice=lat)
        s = semlbm.Solver.from_case(case, device=device)
        s.set_density(case.rho0)
        s.step(3)
        s.synchronize()
        s.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(args.lattice_steps)
        e1.record(s.stream)
        s.synchronize()
        ms = e0.elapsed_time(e1)
        prof = s.profile_read()
        s.profile(False)
        info = s.info
        rhs_ms = prof["ms"]["k_rhs"] / max(prof["launches"]["k_rhs"], 1)
        work = flopcount.rhs_work(lat, case.mesh.N, info["n_local"], info["n_wall_nodes"])
        ach = work["flops"] / (rhs_ms * 1e-3) / 1e12
        out[lat] = {"node_updates_per_s": info["n_local"] * args.lattice_steps / (ms * 1e-3),
                    "ms_per_step": ms / args.lattice_steps, "k_rhs_ms": rhs_ms,
                    "k_rhs_tflops": ach, "k_rhs_frac": ach / peak,
                    "status": s.diagnostics()["status"]}
        s.close()
    return out


def native_arm(args):
    import numpy as np
    import torch
    from paper_2609_00535_b300 import semlbm

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = local
    torch.cuda.set_device(device)

    case = make_case(args.config, args.ne)
    solver = semlbm.Solver.from_case(case, device=device)
    info = solver.info
    solver.set_density(case.rho0)
    stream = solver.stream

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (graph capture happens on the first step)
    solver.step(args.warmup)
    solver.synchronize()

    # timed region: K steps, every kernel bracketed by CUDA events on the
    # solver's stream (per-kernel durations for the roofline)
    # timed region: K steps replayed from the captured graph, as a user's
    # sem_lbm_step runs them (programmatic launches, no events between kernels),
    # bracketed by CUDA events on the solver's stream
    clocks = Clocks(device)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    # the same K steps again with a CUDA event after every kernel
    # (sem_lbm_profile): the per-kernel durations of the roofline and the shares
    solver.profile(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        solver.step(1)
    p1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof_ms = p0.elapsed_time(p1) / args.steps
    prof = solver.profile_read()
    solver.profile(False)
    ms = max_over_ranks(ms, device="cuda")
    value = info["n_local"] * args.steps * ws / (ms * 1e-3)
    d = solver.diagnostics()

    # roofline of the dominant kernel (k_rhs)
    rhs_ms = prof["ms"]["k_rhs"] / max(prof["launches"]["k_rhs"], 1)
    work = flopcount.rhs_work(case.lattice, case.mesh.N, info["n_local"], info["n_wall_nodes"])
    peak, _ = semlbm.fp64_peak_tflops(device)
    achieved = work["flops"] / (rhs_ms * 1e-3) / 1e12
    total_kernel_ms = sum(prof["ms"].values())
    sw = flopcount.step_work(case.lattice, case.mesh.N, info["n_local"], info["n_global"],
                             info["n_wall_nodes"])
    step_s = (ms / args.steps) * 1e-3
    shares = {k: round(v / total_kernel_ms, 4) for k, v in prof["ms"].items()}

    # end to end through the public API with host buffers: every step's input
    # state is uploaded from pinned host memory, the step advances it and its
    # diagnostics are read back to the host.  The input is the compact state,
    # one value per global node and velocity (sem_lbm_set_state_global): the
    # copies of a shared node are equal, so it holds the whole state in G/V of
    # the element-local bytes.  The upload of step k+1's input (a copy stream,
    # into the other of two device staging buffers) overlaps step k's compute;
    # set_state_global then scatters it to the element copies on the device.
    # The same loop with the element-local state (set_state) is reported too.
    Q, V, G = info["Q"], info["n_local"], info["n_global"]
    e2e_steps = max(1, min(args.steps, 100))

    def e2e_measure(n_values, set_fn, state):
        host = torch.empty(n_values, dtype=torch.float64).pin_memory()
        host.copy_(torch.from_numpy(state.reshape(-1)))
        stage = [torch.empty(n_values, dtype=torch.float64, device=device) for _ in range(2)]
        copy = torch.cuda.Stream(device=device)

        def run(n):
            with torch.cuda.stream(copy):
                stage[0].copy_(host, non_blocking=True)
            for k in range(n):
                with torch.cuda.stream(copy):
                    set_fn(stage[k % 2], 0)                    # waits for this input's upload
                    if k + 1 < n:                              # buffer last read by step k-1
                        stage[(k + 1) % 2].copy_(host, non_blocking=True)
                solver.step(1)
                solver.diagnostics()                           # device-to-host read, synchronises

        run(2)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(e2e_steps)
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, device="cuda")

    st_local, _ = solver.get_state()
    st_global, _ = solver.get_state_global()
    e2e_s = e2e_measure(Q * G, solver.set_state_global, st_global)
    e2e_value = V * e2e_steps * ws / e2e_s
    e2e_local_s = e2e_measure(Q * V, solver.set_state, st_local)
    e2e_local_value = V * e2e_steps * ws / e2e_local_s

    line = None
    if rank == 0:
        cpu = cpu1 = None
        if not args.no_cpu_baseline:
            cpu_steps = args.cpu_steps
            rate, secs, cores = oracle_rate(case, cpu_steps)
            cpu1 = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": "%d time steps of the full %s mesh (%d nodes), %.1f s" %
                              (cpu_steps, args.config, case.nodes, secs),
                    "cpu": cpu_model()}
            scase, what = sample_case(args.config)
            rate_all, ncores = oracle_all_cores(args.config, args.cpu_sample_steps)
            cpu = {"value": rate_all, "unit": UNIT, "cores": ncores, "kind": "oracle",
                   "sample": "one replica per core of %d time steps of %s" %
                             (args.cpu_sample_steps, what),
                   "nproc": os.cpu_count(), "cpu": cpu_model(),
                   "single_core_full_mesh": rate}
        batched = batched_small = serving = None
        if not args.no_batched:
            batched = batched_section(args, device)
            batched_small = batched_section(args, device, small_solves())
        lattices = None if args.no_lattices else lattice_section(args, device)
        angle_study = angle_resolution_section(args, device) if args.angle_study else None
        angle_study_3d = (angle_resolution_3d_section(args, device)
                          if args.angle_study_3d else None)
        angle_kelvin = angle_kelvin_section(args, device) if args.angle_study_kelvin else None
        configs = None if args.no_configs else config_lines_section(args, device)
        sweep = serving_c5 = None
        if not args.no_serving:
            cap = batched["batched_node_updates_per_s"] if batched else value
            serving = serving_section(args, device, cap)
            serving_c5 = serving_c5_sizes_section(args, device, cap)
            sweep = angle_sweep_section(args, device)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {
                "workload": args.config, "model": None,
                "mesh": "%d curved hexes, N=%d" % (case.mesh.n_elem, case.mesh.N)
                if case.mesh.dim == 3 else "%d quads, N=%d" % (case.mesh.n_elem, case.mesh.N),
                "lattice": case.lattice, "nodes": V, "global_nodes": info["n_global"],
                "dt": info["dt"], "tau": case.tau, "parallelism": "replicas" if ws > 1 else "1gpu",
                "l2": "inputs larger than L2 (%.0f MB state+geometry vs 126 MB)" %
                      (info["workspace_bytes"] / 1e6),
            },
            "roofline": {"bound": "alu", "kernel": "k_rhs", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": rhs_traffic_per_launch(case.lattice, case.mesh.N, V),
                         "traffic_unit": "bytes per launch",
                         "peak_source": "measured live: FP64 DFMA probe (libsemlbm_peak)",
                         "fp64_op_frac": work["ops"] / (rhs_ms * 1e-3) / (peak * 1e12 / 2),
                         "kernel_ms": rhs_ms, "flops_per_launch": work["flops"]},
            "step_roofline": {"bound": "alu", "ops_per_step": sw["ops"],
                              "flops_per_step": sw["flops"],
                              "achieved": sw["flops"] / step_s / 1e12, "peak": peak,
                              "unit": "TFLOP/s", "frac": sw["flops"] / step_s / 1e12 / peak,
                              "fp64_op_frac": sw["ops"] / step_s / (peak * 1e12 / 2),
                              "note": "all 14 kernels of a step; counts from flops.step_work"},
            "kernel_share": shares,
            "kernel_ms_per_launch": {k: round(prof["ms"][k] / max(1, prof["launches"][k]), 4)
                                     for k in prof["ms"]},
            "gpu_launches": int(info["kernels_per_step"] * args.steps),
            "graph_programmatic_launches": bool(solver.get_info()["graph_pdl"]),
            "instrumented": {"ms_per_step": prof_ms, "node_updates_per_s": V / (prof_ms * 1e-3),
                             "note": "the same K steps issued kernel by kernel with a CUDA event "
                                     "after each (source of the roofline and the kernel shares)"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": Q * G * 8,
                    "d2h_bytes_per_step": 80, "steps": e2e_steps,
                    "input": "compact state on the global nodes (sem_lbm_set_state_global)"},
            "e2e_element_local": {"value": e2e_local_value, "unit": UNIT,
                                  "h2d_bytes_per_step": Q * V * 8, "d2h_bytes_per_step": 80,
                                  "steps": e2e_steps,
                                  "input": "element-local state (sem_lbm_set_state)"},
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
            "configs": configs,
            "batched": batched,
            "batched_small": batched_small,
            "serving": serving,
            "serving_c5_sizes": serving_c5,
            "angle_sweep": sweep,
            "lattices": lattices,
            "angle_resolution": angle_study,
            "angle_resolution_3d": angle_study_3d,
            "angle_kelvin": angle_kelvin,
            "final_diag": {"ke_max": d["ke_max"], "mass": d["mass"], "status": d["status"]},
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--config", default="sphere3d", choices=["sphere3d", "flat2d", "cylinder2d"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-solves", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--config-steps", type=int, default=200,
                    help="steps of the flat-wall and cylinder plain lines")
    ap.add_argument("--no-configs", action="store_true", help="skip the 2D plain lines")
    ap.add_argument("--cpu-sample-steps", type=int, default=60,
                    help="oracle steps per core replica of the bounded sample")
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--serve-max-steps", type=int, default=200000)
    ap.add_argument("--serve-epoch", type=int, default=500)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--sweep-requests", type=int, default=16)
    ap.add_argument("--c5-requests", type=int, default=60)
    ap.add_argument("--c5-steps", type=int, default=300)
    ap.add_argument("--lattice-steps", type=int, default=50)
    ap.add_argument("--angle-study", action="store_true",
                    help="flat-wall contact angle at three interface widths (minutes)")
    ap.add_argument("--angle-study-3d", action="store_true",
                    help="add the sphere-wall contact angle at four interface widths")
    ap.add_argument("--angle-study-3d-max-steps", type=int, default=200000)
    ap.add_argument("--angle-study-kelvin", action="store_true",
                    help="add the flat-wall angle with and without the Kelvin shift")
    ap.add_argument("--angle-study-degrees", default="60,90,120")
    ap.add_argument("--angle-study-epoch", type=int, default=2000)
    ap.add_argument("--angle-study-max-steps", type=int, default=600000)
    ap.add_argument("--no-lattices", action="store_true", help="skip the D3Q19/D3Q27 lines")
    ap.add_argument("--sweep-max-steps", type=int, default=100000)
    ap.add_argument("--ne", type=int, default=None,
                    help="elements per axis of the sphere-cap mesh (profiling cases only)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return native_arm(args)


if __name__ == "__main__":
    sys.exit(main())
