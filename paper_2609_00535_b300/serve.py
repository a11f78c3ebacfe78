"""Continuous-batching server for contact-angle and geometry sweep requests.

Requests arrive over time (e.g. a Poisson stream); each asks for one solve to
be run until its maximum kinetic energy falls below a threshold, or until a
step budget is spent.  The server keeps one batch (libsemlbm's
sem_lbm_batch_*) stepping on the GPU, and three kinds of work overlap:

* a dispatcher thread follows the arrival schedule and hands each arrived
  request to a worker pool;
* a worker builds the request's mesh and initial density on the host, then
  reserves its device memory (sem_lbm_workspace_bytes) against the HBM budget
  - first come, first served, waiting while the budget is full - and creates
  the solver in PyTorch memory;
* the main loop, between epochs of `epoch_steps` steps, adds every ready
  solver to the batch as a new slot (the running CUDA graph is not
  re-captured), reads all slots' diagnostics with one synchronisation, and
  retires the slots that converged (KE_max < ke_tol after min_steps), failed
  (non-finite state), were cancelled (Server.cancel) or used max_steps,
  returning their memory to the budget.

Every solve computes the same bits as it would alone (the batch kernels are
the single-solve kernels over a slot table), so admission order and the mix
change latency, never results.
"""
import concurrent.futures as cf
import queue
import threading
import time
from dataclasses import dataclass, field

from . import semlbm


@dataclass
class Record:
    rid: int
    arrival: float
    ready: float = None
    admitted: float = None
    finished: float = None
    steps: int = 0
    ke_max: float = None
    converged: bool = False
    failed: bool = False
    cancelled: bool = False
    nodes: int = 0
    bytes: int = 0
    name: str = ""
    error: str = ""
    state: object = None
    moments: dict = None   # wetting moments at retirement (Server(measure_tag=...))


@dataclass
class Stats:
    records: list = field(default_factory=list)
    wall_s: float = 0.0
    node_updates: int = 0
    epochs: int = 0
    max_slots: int = 0
    max_bytes: int = 0
    overlapped_admissions: int = 0     # admitted while other slots were running

    def latencies(self):
        return sorted(r.finished - r.arrival for r in self.records if r.finished is not None)

    def percentile(self, p):
        lat = self.latencies()
        if not lat:
            return None
        k = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
        return lat[k]

    def summary(self):
        done = [r for r in self.records if r.finished is not None]
        return {
            "requests": len(self.records), "completed": len(done),
            "converged": sum(r.converged for r in done),
            "capped": sum((not r.converged and not r.failed and not r.cancelled) for r in done),
            "failed": sum(r.failed for r in done),
            "cancelled": sum(r.cancelled for r in done),
            "p50_s": self.percentile(50), "p99_s": self.percentile(99),
            "node_updates_per_s": self.node_updates / self.wall_s if self.wall_s else None,
            "wall_s": self.wall_s, "epochs": self.epochs, "max_slots": self.max_slots,
            "max_bytes": self.max_bytes, "overlapped_admissions": self.overlapped_admissions,
            "failures": [{"name": r.name, "steps": r.steps, "error": r.error}
                         for r in done if r.failed],
        }


class Budget:
    """Device-memory budget handed out first come, first served."""

    def __init__(self, total):
        self.total = int(total)
        self.used = 0
        self.cv = threading.Condition()
        self.next_ticket = 0
        self.serving = 0

    def acquire(self, nbytes, stop):
        with self.cv:
            ticket = self.next_ticket
            self.next_ticket += 1
            while not stop.is_set() and (ticket != self.serving or
                                         (self.used + nbytes > self.total and self.used > 0)):
                self.cv.wait(0.05)
            if stop.is_set():
                return False
            self.used += nbytes
            self.serving += 1
            self.cv.notify_all()
            return True

    def release(self, nbytes):
        with self.cv:
            self.used -= nbytes
            self.cv.notify_all()


class Server:
    def __init__(self, hbm_budget_bytes, epoch_steps=50, ke_tol=1e-20, max_steps=2000,
                 min_steps=100, keep_state=False, workers=4, device=0, clock=time.perf_counter,
                 measure_tag=None):
        self.budget_bytes = int(hbm_budget_bytes)
        self.epoch_steps = int(epoch_steps)
        self.ke_tol = ke_tol
        self.max_steps = int(max_steps)
        self.min_steps = int(min_steps)
        self.keep_state = keep_state
        self.workers = workers
        self.device = device
        self.clock = clock
        self.measure_tag = measure_tag   # wall tag whose wetting moments each result carries
        self._cancel = set()
        self._cancel_lock = threading.Lock()

    def cancel(self, rid):
        """Withdraw a request (from any thread): one not yet built is never built,
        a running one is retired at the next epoch boundary; others are unaffected."""
        with self._cancel_lock:
            self._cancel.add(rid)

    def _cancelled(self, rid):
        with self._cancel_lock:
            return rid in self._cancel

    def run(self, requests):
        """Serve the requests; returns Stats (one Record per request)."""
        import torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        stats = Stats()
        budget = Budget(self.budget_bytes)
        ready = queue.Queue()
        stop = threading.Event()
        t0 = self.clock()
        records = {r.rid: Record(r.rid, r.arrival) for r in reqs}
        stats.records = [records[r.rid] for r in reqs]

        def prepare(req):
            torch.cuda.set_device(self.device)
            rec = records[req.rid]
            if self._cancelled(req.rid):
                rec.cancelled = True
                rec.finished = self.clock() - t0
                ready.put((req.rid, None))
                return
            try:
                case = req.case()
                need = semlbm.workspace_bytes(case.mesh, case.mesh.N, case.lattice)
                rec.nodes, rec.bytes, rec.name = case.nodes, need, case.name
                if not budget.acquire(need, stop):
                    return
                s = semlbm.Solver.from_case(case, device=self.device)
                s.set_density(case.rho0)
                s.synchronize()
                rec.ready = self.clock() - t0
                ready.put((req.rid, s))
            except Exception as exc:   # a request that cannot be built fails alone
                rec.failed = True
                rec.finished = self.clock() - t0
                rec.error = repr(exc)[:200]
                ready.put((req.rid, None))

        pool = cf.ThreadPoolExecutor(max_workers=self.workers)

        def dispatch():
            for req in reqs:
                while not stop.is_set():
                    wait = req.arrival - (self.clock() - t0)
                    if wait <= 0:
                        break
                    time.sleep(min(wait, 0.01))
                if stop.is_set():
                    return
                pool.submit(prepare, req)

        dispatcher = threading.Thread(target=dispatch, daemon=True)
        batch = semlbm.Batch(device=self.device)
        active = {}
        finished = 0
        dispatcher.start()
        try:
            while finished < len(reqs):
                # admit every solver that is ready
                while True:
                    try:
                        rid, s = ready.get(timeout=0.0 if active else 0.02)
                    except queue.Empty:
                        break
                    rec = records[rid]
                    if s is None:
                        finished += 1
                        continue
                    if self._cancelled(rid):          # withdrawn while it was being built
                        rec.cancelled = True
                        rec.finished = self.clock() - t0
                        s.close()
                        budget.release(rec.bytes)
                        finished += 1
                        continue
                    if active:
                        stats.overlapped_admissions += 1
                    slot = batch.add(s)
                    rec.admitted = self.clock() - t0
                    active[slot] = (s, rec)
                stats.max_slots = max(stats.max_slots, len(active))
                stats.max_bytes = max(stats.max_bytes, budget.used)
                if not active:
                    continue
                batch.step(self.epoch_steps)
                stats.epochs += 1
                stats.node_updates += self.epoch_steps * sum(r.nodes for _, r in active.values())
                diag = batch.diagnostics()
                now = self.clock() - t0
                for slot in list(active):
                    s, rec = active[slot]
                    d = diag[slot]
                    rec.steps, rec.ke_max = d["step"], d["ke_max"]
                    if d["status"] != 0:
                        rec.failed = True
                        rec.error = "status %d at step %d" % (d["status"], d["step"])
                    elif self._cancelled(rec.rid):
                        rec.cancelled = True
                    elif d["step"] >= self.min_steps and d["ke_max"] < self.ke_tol:
                        rec.converged = True
                    elif d["step"] < self.max_steps:
                        continue
                    rec.finished = now
                    batch.remove(slot)
                    if self.keep_state:
                        rec.state = s.get_state()[0]
                    if self.measure_tag is not None and not (rec.failed or rec.cancelled):
                        rec.moments = s.wetting_moments(self.measure_tag)
                    s.close()
                    budget.release(rec.bytes)
                    del active[slot]
                    finished += 1
        finally:
            stop.set()
            stats.wall_s = self.clock() - t0
            dispatcher.join(timeout=5)
            pool.shutdown(wait=True)
            while not ready.empty():
                _, s = ready.get()
                if s is not None:
                    s.close()
            for s, _ in active.values():
                s.close()
            batch.close()
        return stats
