"""Continuous-batching solve service on top of the C ABI's batch sessions.

Requests (mesh size n, rho, target, tolerance) are grouped by (n, rho-bucket).  Buckets
are decades of rho, floor(log10 rho), grouped per mesh into two regimes: stiffness-
dominated (rho >= h^2) and mass-dominated (rho < h^2).  With the prolongators fixed, a
bucket's operators are the pencil rho K_l + M_l, and prolongators set up at the largest
rho of a regime serve every rho of it (coarse correction matters in the stiff regime and
little in the mass regime, where the smoother does the work).  Per n there is one
assembled system that keeps its pencil (K and M); per (n, regime) a smoothed-aggregation
hierarchy is built once and cached; per (n, regime) one batch session with a fixed
number of slots runs on its own CUDA stream,
so sessions of different keys overlap on the device.  Every tick advances each busy
session by a few CG iterations, retires the slots that finished, and admits waiting
requests into free slots; a session is created only if its bytes fit in the HBM budget
(idle sessions are evicted first, least recently used).  Each request's result depends
only on its own slot: the same request solved alone or among others gives the same bits.

All arithmetic runs in the CUDA library; this module only schedules calls.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import torch

from . import _binding as fa


@dataclass
class Request:
    id: int
    n: int
    rho: float
    target: dict
    t_arrival: float = 0.0
    tol: float = 1e-8
    # filled in by the service
    t_admit: float = -1.0
    t_done: float = -1.0
    iterations: int = 0
    status: int = -1
    relres: float = float("nan")
    u: torch.Tensor | None = None


@dataclass
class ServeConfig:
    slots: int = 4                # slots per (n, bucket) session
    steps_per_tick: int = 1       # CG iterations per session per tick
    hbm_budget: int = 160 << 30   # bytes the service may hold on the device
    precision: int = fa.AMG_PREC_FP32
    keep_solutions: bool = False  # keep each request's solution on the device
    max_iter: int = 500
    coarse_max: int = 256


def rho_bucket(rho: float) -> int:
    return int(math.floor(math.log10(rho) + 1e-12))


def regime(n: int, bucket: int) -> int:
    """1 for decades whose rho reaches h^2 = 1/n^2 or more (stiffness-dominated), 0 below."""
    return 1 if 10.0 ** (bucket + 1) > 1.0 / n ** 2 else 0


def regime_rho_setup(n: int, reg: int, rho_max: float = 1.0) -> float:
    """Set-up rho of a regime: its largest rho (rho_max for the stiff regime, h^2 below)."""
    return rho_max if reg == 1 else 1.0 / n ** 2


@dataclass
class _Session:
    key: tuple
    handle: object
    stream: torch.cuda.Stream
    slots: int
    bytes: int
    members: dict = field(default_factory=dict)   # slot -> Request
    last_used: float = 0.0


class SolveService:
    def __init__(self, cfg: ServeConfig | None = None, device: int = 0):
        self.cfg = cfg or ServeConfig()
        self.device = torch.device("cuda", device)
        self.systems: dict[int, object] = {}
        self.hier: dict[tuple, object] = {}
        self.sessions: "collections.OrderedDict[tuple, _Session]" = collections.OrderedDict()
        self.queue: "collections.deque[Request]" = collections.deque()
        self.done: list[Request] = []
        self.bytes_in_use = 0
        self.stats = collections.Counter()
        self._t0 = time.perf_counter()

    # ------------------------------------------------------------------ resources
    def now(self) -> float:
        return time.perf_counter() - self._t0

    def _system(self, n: int):
        s = self.systems.get(n)
        if s is None:
            s = fa.fem_assemble(n, 1.0 / n ** 2, {"kind": "sine"}, keep_pencil=True)
            info = fa.fem_system_get_info(s)
            self.bytes_in_use += info["nnz"] * 28 + info["N"] * 24
            self.systems[n] = s
        return s

    def _hierarchy(self, n: int, reg: int):
        key = (n, reg)
        h = self.hier.get(key)
        if h is None:
            self.stats["hierarchy_builds"] += 1
            h = fa.amg_setup(self._system(n), precision=self.cfg.precision,
                             coarse_max=self.cfg.coarse_max, rho_setup=regime_rho_setup(n, reg))
            self.bytes_in_use += self._hier_bytes(h)
            self.hier[key] = h
        else:
            self.stats["hierarchy_hits"] += 1
        return h

    def _hier_bytes(self, h) -> int:
        return sum(fa.amg_hier_get_info(h)["nnz"]) * 20

    def _evict_idle(self, need: int, keep: tuple) -> bool:
        """Free idle sessions (least recently used first), then hierarchies that no session
        uses, until `need` more bytes fit in the budget."""
        for key in list(self.sessions.keys()):
            if self.bytes_in_use + need <= self.cfg.hbm_budget:
                return True
            sess = self.sessions[key]
            if not sess.members:
                fa.pcg_batch_destroy(sess.handle)
                self.bytes_in_use -= sess.bytes
                del self.sessions[key]
                self.stats["evictions"] += 1
        for key in list(self.hier.keys()):
            if self.bytes_in_use + need <= self.cfg.hbm_budget:
                return True
            if key != keep and key not in self.sessions:
                h = self.hier.pop(key)
                self.bytes_in_use -= self._hier_bytes(h)
                fa.amg_hier_destroy(h)
                self.stats["hierarchy_evictions"] += 1
        return self.bytes_in_use + need <= self.cfg.hbm_budget

    def _session(self, n: int, bucket: int):
        key = (n, regime(n, bucket))
        sess = self.sessions.get(key)
        if sess is not None:
            self.sessions.move_to_end(key)
            self.stats["hierarchy_hits"] += 1
            return sess
        sys_ = self._system(n)
        h = self._hierarchy(*key)
        need = fa.pcg_batch_footprint(sys_, h, self.cfg.slots)
        if need < 0:
            raise fa.FemError(fa.FEM_EINVAL, "no footprint for this session")
        if not self._evict_idle(need, key):
            if not any(s.members for s in self.sessions.values()):
                raise MemoryError("a (n=%d, regime=%d) session does not fit in the budget" % key)
            return None
        stream = torch.cuda.Stream(device=self.device)
        handle = fa.pcg_batch_create(sys_, h, self.cfg.slots, stream=stream,
                                     tol=1e-8, max_iter=self.cfg.max_iter)
        sess = _Session(key, handle, stream, self.cfg.slots, need)
        self.bytes_in_use += need
        self.sessions[key] = sess
        return sess

    # ------------------------------------------------------------------ requests
    def submit(self, req: Request):
        self.queue.append(req)

    def _admit_waiting(self):
        waiting = collections.deque()
        while self.queue:
            req = self.queue.popleft()
            try:
                sess = self._session(req.n, rho_bucket(req.rho))
            except MemoryError:
                req.status = 2  # rejected: can never fit
                req.t_done = self.now()
                self.done.append(req)
                self.stats["rejected"] += 1
                continue
            if sess is None or len(sess.members) >= sess.slots:
                waiting.append(req)
                continue
            N = (req.n - 1) ** 3
            f = torch.empty(N, dtype=torch.float64, device=self.device)
            with torch.cuda.stream(sess.stream):
                fa.fem_assemble_rhs(self._system(req.n), req.target, f, stream=sess.stream)
                slot = fa.pcg_batch_admit(sess.handle, f, req.rho, stream=sess.stream)
            sess.members[slot] = req
            req.t_admit = self.now()
            self.stats["admitted"] += 1
        self.queue = waiting

    def tick(self):
        """Admit, advance every busy session, retire finished slots."""
        self._admit_waiting()
        busy = [s for s in self.sessions.values() if s.members]
        for s in busy:
            fa.pcg_batch_step(s.handle, self.cfg.steps_per_tick, stream=s.stream)
        for s in busy:
            st, it, rr = fa.pcg_batch_poll(s.handle, s.slots, stream=s.stream)
            t = self.now()
            s.last_used = t
            for slot in [k for k in s.members if st[k] != 0]:
                req = s.members.pop(slot)
                N = (req.n - 1) ** 3
                u = torch.empty(N, dtype=torch.float64, device=self.device)
                fa.pcg_batch_retire(s.handle, slot, u, stream=s.stream)
                req.t_done = t
                req.iterations = int(it[slot])
                req.status = int(st[slot])
                req.relres = float(rr[slot])
                if self.cfg.keep_solutions:
                    req.u = u
                self.done.append(req)
                self.stats["retired"] += 1
        return len(busy)

    def idle(self) -> bool:
        return not self.queue and all(not s.members for s in self.sessions.values())

    def run(self, requests, realtime: bool = True, time_limit: float = 1e9):
        """Serve requests whose t_arrival are seconds after the start (realtime) or all at
        once (realtime=False).  Returns the summary of run_stats()."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        self._t0 = time.perf_counter()
        while pending or not self.idle():
            t = self.now()
            if t > time_limit:
                break
            while pending and (not realtime or pending[0].t_arrival <= t):
                r = pending.popleft()
                if not realtime:
                    r.t_arrival = t
                self.submit(r)
            if self.tick() == 0 and not self.queue and pending:
                time.sleep(max(0.0, min(0.002, pending[0].t_arrival - self.now())))
        torch.cuda.synchronize(self.device)
        return self.run_stats()

    def run_stats(self) -> dict:
        lat = sorted(r.t_done - r.t_arrival for r in self.done if r.t_done >= 0)
        if not lat:
            return {"solved": 0}
        span = max(r.t_done for r in self.done) - min(r.t_arrival for r in self.done)

        def pct(p):
            return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)]
        ok = sum(1 for r in self.done if r.status == 1)
        hits = self.stats["hierarchy_hits"]
        builds = self.stats["hierarchy_builds"]
        return {"solved": len(lat), "converged": ok, "p50_ms": pct(50) * 1e3,
                "p99_ms": pct(99) * 1e3, "mean_ms": sum(lat) / len(lat) * 1e3,
                "solves_per_s": len(lat) / span if span > 0 else float("nan"),
                "hierarchy_builds": builds,
                "cache_hit_rate": hits / (hits + builds) if hits + builds else 0.0,
                "evictions": self.stats["evictions"]}

    def close(self):
        torch.cuda.synchronize(self.device)
        for s in self.sessions.values():
            fa.pcg_batch_destroy(s.handle)
        for h in self.hier.values():
            fa.amg_hier_destroy(h)
        for s in self.systems.values():
            fa.fem_system_destroy(s)
        self.sessions.clear()
        self.hier.clear()
        self.systems.clear()
