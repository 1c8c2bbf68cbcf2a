"""Host logic of the serving loop with a fake library (no GPU): sessions are created only when
their bytes fit the HBM budget, idle sessions are evicted least recently used first and then
hierarchies no session uses, a session that can never fit is refused, and requests wait for
free slots and join a busy session as soon as one frees up (continuous batching)."""
import contextlib
import types

import pytest
import torch

from paper_2102_03515_gb300 import serving


class FakeLib:
    """The calls serving makes, with sizes chosen by the test: a session costs `session`
    bytes, a hierarchy 20, a system nothing; every request converges after `iters` steps."""

    AMG_PREC_FP32 = 1
    FEM_EINVAL = 1
    FemError = RuntimeError

    def __init__(self, session=100, iters=3):
        self.session, self.iters = session, iters
        self.next = 0
        self.batches = {}
        self.log = []

    def _new(self, kind):
        self.next += 1
        self.log.append(("new", kind, self.next))
        return (kind, self.next)

    def fem_assemble(self, n, rho, target, keep_pencil=False):
        return self._new("sys")

    def fem_system_get_info(self, s):
        return {"nnz": 0, "N": 0}

    def amg_setup(self, sys_, **kw):
        return self._new("hier")

    def amg_hier_get_info(self, h):
        return {"nnz": [1]}

    def pcg_batch_footprint(self, sys_, h, slots):
        return self.session

    def pcg_batch_create(self, sys_, h, slots, stream=None, **kw):
        b = self._new("batch")
        self.batches[b] = [None] * slots
        return b

    def pcg_batch_destroy(self, b):
        self.log.append(("free", "batch", b[1]))
        del self.batches[b]

    def amg_hier_destroy(self, h):
        self.log.append(("free", "hier", h[1]))

    def fem_system_destroy(self, s):
        pass

    def fem_assemble_rhs(self, sys_, target, f, stream=None):
        pass

    def pcg_batch_admit(self, b, f, rho, stream=None):
        slots = self.batches[b]
        k = slots.index(None)
        slots[k] = 0
        return k

    def pcg_batch_step(self, b, iters, stream=None):
        slots = self.batches[b]
        for k, v in enumerate(slots):
            if v is not None:
                slots[k] = v + iters

    def pcg_batch_poll(self, b, nslots, stream=None):
        slots = self.batches[b]
        st = [-1 if v is None else (1 if v >= self.iters else 0) for v in slots]
        it = [0 if v is None else v for v in slots]
        return st, it, [0.0] * nslots

    def pcg_batch_retire(self, b, slot, u, stream=None):
        self.batches[b][slot] = None


FAKE_TORCH = types.SimpleNamespace(
    float64=torch.float64, device=torch.device, Tensor=torch.Tensor,
    empty=lambda *a, dtype=None, device=None: torch.empty(*a, dtype=dtype),
    cuda=types.SimpleNamespace(Stream=lambda device=None: object(),
                               stream=lambda s: contextlib.nullcontext(),
                               synchronize=lambda *a, **k: None))


@pytest.fixture
def service(monkeypatch):
    def make(budget, session=100, iters=3, slots=2):
        lib = FakeLib(session, iters)
        monkeypatch.setattr(serving, "fa", lib)
        monkeypatch.setattr(serving, "torch", FAKE_TORCH)
        cfg = serving.ServeConfig(slots=slots, hbm_budget=budget)
        return serving.SolveService(cfg), lib
    return make


def _req(i, n, rho=1.0):
    return serving.Request(id=i, n=n, rho=rho, target={"kind": "sine"})


def _serve(s, reqs, budget, ticks=50):
    for r in reqs:
        s.submit(r)
    for _ in range(ticks):
        s.tick()
        assert s.bytes_in_use <= budget
        if s.idle():
            return
    raise AssertionError("service did not drain")


def test_idle_sessions_are_evicted_least_recently_used_first(service):
    s, lib = service(budget=280)
    _serve(s, [_req(0, 32)], 280)            # session (32) + hierarchy: 120 bytes
    _serve(s, [_req(1, 64)], 280)            # 240
    _serve(s, [_req(2, 32)], 280)            # reuses (32): now the most recently used
    b64 = s.sessions[(64, 1)].handle
    _serve(s, [_req(3, 96)], 280)            # 260 + 100 > 280: evict one idle session
    assert (64, 1) not in s.sessions and (32, 1) in s.sessions and (96, 1) in s.sessions
    assert ("free", "batch", b64[1]) in lib.log
    assert s.stats["evictions"] == 1 and s.stats["hierarchy_evictions"] == 0
    assert all(r.status == 1 for r in s.done)


def test_unused_hierarchies_go_when_idle_sessions_are_not_enough(service):
    s, lib = service(budget=130)
    _serve(s, [_req(0, 32)], 130)            # 120
    _serve(s, [_req(1, 64)], 130)            # needs the (32) session and its hierarchy freed
    assert s.stats["evictions"] == 1 and s.stats["hierarchy_evictions"] == 1
    assert list(s.hier.keys()) == [(64, 1)] and list(s.sessions.keys()) == [(64, 1)]
    assert [r.status for r in s.done] == [1, 1]


def test_a_session_that_can_never_fit_is_refused(service):
    s, _ = service(budget=110)                # hierarchy 20 + session 100 > 110
    _serve(s, [_req(0, 32)], 110)
    assert [r.status for r in s.done] == [2] and s.stats["rejected"] == 1


def test_requests_wait_for_slots_and_join_busy_sessions(service):
    s, _ = service(budget=1 << 20, iters=3, slots=2)
    first = _req(0, 48)
    s.submit(first)
    s.tick()                                  # admitted, one CG step done
    late = [_req(1, 48), _req(2, 48)]
    for r in late:
        s.submit(r)
    s.tick()                                  # one free slot: the first late request joins
    sess = s.sessions[(48, 1)]
    assert sorted(r.id for r in sess.members.values()) == [0, 1] and len(s.queue) == 1
    for _ in range(10):
        s.tick()
        if s.idle():
            break
    assert s.idle() and sorted(r.id for r in s.done) == [0, 1, 2]
    assert all(r.status == 1 and r.iterations == 3 for r in s.done)
    assert late[0].t_admit < first.t_done <= late[1].t_admit
