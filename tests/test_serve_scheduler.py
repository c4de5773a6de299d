"""Host logic of the serving loop (``serve.CNServer``) on the CPU.

The scheduler's policy is host code: admission by HBM budget, eviction of
the least recently used idle operator, and at most one request per operator
per batch, in arrival order. It also handles cancellation and surfaces a
failed step to every waiting client. Here it runs against a fake of the
binding (same calls, CPU tensors). Faults are injected on the host: a step
that raises, and a request cancelled while queued. The fake step is the affine
map u <- dt u + 1 of each operator, so after k steps every entry of u equals
x_k = dt x_{k-1} + 1. The closed form checks that states survive batching,
eviction and re-admission.
"""

import threading

import numpy as np
import pytest
import torch

from paper_2004_05566_gb300 import serve as S

BYTES = 100_000  # device bytes the fake hif_query reports per operator


class _FakeHandle:
    def __init__(self, fake, dt):
        self.fake, self.dt, self.closed, self.reaction = fake, dt, False, None

    def close(self):
        assert not self.closed
        self.closed = True
        self.fake.live -= 1


class _FakeBinding:
    HIF_FP64 = 0
    HIF_FP32 = 1

    def __init__(self, poison_dt=None, hold_dt=None):
        self.hold_dt = hold_dt  # steps of operators with this dt wait for hold
        self.hold = threading.Event()
        self.held = threading.Event()  # set when such a step waits
        self.setups = 0
        self.live = 0
        self.batch_sizes = []
        self.poison_dt = poison_dt
        self.entered = threading.Event()  # set when a step starts
        self.gate = threading.Event()     # a step waits for it
        self.gate.set()

    def default_options(self, eps, precision, cg_tol):
        return (eps, precision, cg_tol)

    def hif_setup(self, dim, n, leaf, a, dt, opt):
        assert a.shape == (n + 1,) * dim
        self.setups += 1
        self.live += 1
        return _FakeHandle(self, dt)

    def hif_set_reaction(self, h, kind, k1, k2):
        h.reaction = (kind, k1, k2)

    def hif_query(self, h):
        return {"device_bytes": BYTES}

    def cn_step_batched(self, hs, us, outs):
        if self.hold_dt is not None and any(h.dt == self.hold_dt for h in hs):
            self.held.set()
            assert self.hold.wait(30)
        self.entered.set()
        assert self.gate.wait(30)
        assert len({id(h) for h in hs}) == len(hs)  # one request per operator
        self.batch_sizes.append(len(hs))
        for h, u, o in zip(hs, us, outs):
            assert not h.closed
            if h.dt == self.poison_dt:
                raise RuntimeError("injected step failure")
            o.copy_(h.dt * u + 1.0)
        return outs, [2] * len(hs)


@pytest.fixture
def fake(monkeypatch):
    f = _FakeBinding(poison_dt=0.875)
    monkeypatch.setattr(S, "H", f)
    return f


def _spec(dt, n=8):
    return S.OperatorSpec(dim=2, n=n, leaf=4, a_nodes=np.ones((n + 1, n + 1)), dt=dt, eps=1e-6,
                          u0=np.zeros((n - 1, n - 1)), reaction=(1, 1.0, 10.0), precision=1)


def _expected(dt, k):
    x = 0.0
    for _ in range(k):
        x = dt * x + 1.0
    return x


def _server(budget, **kw):
    return S.CNServer(hbm_budget_bytes=budget, device=torch.device("cpu"), **kw)


def test_budget_admission_lru_eviction_and_state(fake):
    srv = _server(int(2.5 * BYTES))  # room for two resident operators
    dts = {"A": 0.5, "B": 0.25, "C": 0.125}
    for k, dt in dts.items():
        srv.register(k, _spec(dt))
    try:
        for k in ("A", "B", "C"):  # C's admission evicts A (least recently used)
            r = srv.submit(k).result(30)
            assert r.step == 1 and r.iters == 2
        assert srv.evictions == 1 and srv.setups("A") == 1
        assert srv.resident_bytes() == 2 * BYTES
        assert srv.submit("A").result(30).step == 2  # re-admitted: B is now the oldest
        assert srv.setups("A") == 2 and srv.evictions == 2
        for _ in range(3):
            srv.submit("B").result(30)
        steps = {"A": 2, "B": 4, "C": 1}
        for k, dt in dts.items():
            assert srv.step_count(k) == steps[k]
            assert np.all(srv.state(k) == _expected(dt, steps[k])), k
        assert srv.resident_bytes() <= srv.budget
        assert fake.live == 2
    finally:
        srv.close()
    assert fake.live == 0


def test_one_request_per_operator_per_batch_in_order(fake):
    srv = _server(10 * BYTES)
    srv.register("A", _spec(0.5))
    srv.register("B", _spec(0.25))
    try:
        fake.gate.clear()
        f1 = srv.submit("A")
        assert fake.entered.wait(30)  # the first batch is running (held at the gate)
        f2, f3, g1 = srv.submit("A"), srv.submit("A"), srv.submit("B")
        fake.gate.set()
        res = [f.result(30) for f in (f1, f2, f3, g1)]
        assert [r.step for r in res[:3]] == [1, 2, 3]
        assert res[3].step == 1
        assert fake.batch_sizes == [1, 2, 1]
        assert res[1].batch_size == 2 and res[2].batch_size == 1
        assert np.all(srv.state("A") == _expected(0.5, 3))
    finally:
        srv.close()


def test_cancelled_request_is_not_stepped(fake):
    srv = _server(10 * BYTES)
    for k, dt in (("A", 0.5), ("B", 0.25), ("C", 0.125)):
        srv.register(k, _spec(dt))
    try:
        fake.gate.clear()
        fa = srv.submit("A")
        assert fake.entered.wait(30)
        fb = srv.submit("B")
        assert fb.cancel()  # still queued: cancellable
        fc = srv.submit("C")
        fake.gate.set()
        assert fa.result(30).step == 1 and fc.result(30).step == 1
        assert fb.cancelled()
        assert srv.step_count("B") == 0 and srv.setups("B") == 0
        assert srv.submit("B").result(30).step == 1  # the server is still serving
        assert not fa.cancel()  # a completed request cannot be cancelled
    finally:
        srv.close()


def test_failed_step_reaches_every_waiting_client(fake):
    srv = _server(10 * BYTES)
    srv.register("ok", _spec(0.5))
    srv.register("bad", _spec(fake.poison_dt))
    try:
        fake.gate.clear()
        f0 = srv.submit("ok")
        assert fake.entered.wait(30)
        f_bad, f_ok, f_later = srv.submit("bad"), srv.submit("ok"), srv.submit("ok")
        f_cancel = srv.submit("ok")
        assert f_cancel.cancel()
        fake.gate.set()
        assert f0.result(30).step == 1
        for f in (f_bad, f_ok, f_later):
            with pytest.raises(RuntimeError, match="injected step failure"):
                f.result(30)
        assert f_cancel.cancelled()
        with pytest.raises(RuntimeError, match="server stopped"):
            srv.submit("ok")
    finally:
        srv.close()
    assert fake.live == 0


def test_size_lanes_small_operators_pass_a_held_large_batch(monkeypatch):
    """Two size lanes: while a step of a large operator is held on the GPU
    side, requests of small operators are still stepped (their own lane), and
    every trajectory is the closed form afterwards."""
    f = _FakeBinding(hold_dt=0.75)
    monkeypatch.setattr(S, "H", f)
    srv = _server(10 * BYTES, lanes=[100])  # N <= 100: lane 0 (n = 8: N = 49); n = 16: N = 225
    srv.register("big", _spec(0.75, n=16))
    srv.register("s1", _spec(0.5))
    srv.register("s2", _spec(0.25))
    try:
        assert srv.lane_of("big") == 1 and srv.lane_of("s1") == 0
        fb = srv.submit("big")
        assert f.held.wait(30)  # the large lane's batch is running (held)
        small = [srv.submit("s1"), srv.submit("s2"), srv.submit("s1")]
        res = [r.result(30) for r in small]  # completes while "big" is still held
        assert not fb.done()
        assert [r.step for r in res] == [1, 1, 2]
        f.hold.set()
        assert fb.result(30).step == 1
        assert np.all(srv.state("s1") == _expected(0.5, 2))
        assert np.all(srv.state("big") == _expected(0.75, 1))
    finally:
        f.hold.set()
        srv.close()
    assert f.live == 0


class _OffloadBinding(_FakeBinding):
    """The fake with hif_offload / hif_reload: an offloaded handle refuses steps."""

    def __init__(self):
        super().__init__()
        self.offloads = 0

    def hif_offload(self, h):
        assert not h.closed and not getattr(h, "off", False)
        h.off = True
        self.offloads += 1

    def hif_reload(self, h):
        assert h.off
        h.off = False

    def cn_step_batched(self, hs, us, outs):
        assert not any(getattr(h, "off", False) for h in hs)
        return super().cn_step_batched(hs, us, outs)


def test_eviction_offloads_and_readmission_reloads(monkeypatch):
    """With offload available, an evicted operator keeps its handle (moved to
    host memory) and is reloaded instead of factored again; states continue."""
    f = _OffloadBinding()
    monkeypatch.setattr(S, "H", f)
    srv = _server(int(2.5 * BYTES))
    dts = {"A": 0.5, "B": 0.25, "C": 0.125}
    for k, dt in dts.items():
        srv.register(k, _spec(dt))
    try:
        for k in ("A", "B", "C", "A", "B"):
            srv.submit(k).result(30)
        assert f.offloads >= 2 and srv.evictions == f.offloads
        assert all(srv.setups(k) == 1 for k in dts)  # never factored twice
        assert srv.reload_count("A") == 1
        steps = {"A": 2, "B": 2, "C": 1}
        for k, dt in dts.items():
            assert np.all(srv.state(k) == _expected(dt, steps[k])), k
        assert f.live == 3  # offloaded handles are kept
    finally:
        srv.close()
    assert f.live == 0


class _SlowOffloadBinding(_OffloadBinding):
    """Offload takes a while, so another lane's request for the operator being
    evicted arrives while the eviction runs."""

    def __init__(self):
        super().__init__()
        self.offloading = threading.Event()

    def hif_offload(self, h):
        self.offloading.set()
        import time
        time.sleep(0.3)
        super().hif_offload(h)


def test_lane_waits_for_an_eviction_by_another_lane(monkeypatch):
    """Lane 1's admission evicts lane 0's idle operator; a request for that
    operator arriving during the eviction waits for it to finish and then
    reloads the operator (it is never stepped half-evicted)."""
    f = _SlowOffloadBinding()
    monkeypatch.setattr(S, "H", f)
    srv = _server(int(1.5 * BYTES), lanes=[100])
    srv.register("small", _spec(0.5))          # lane 0
    srv.register("big", _spec(0.75, n=16))     # lane 1
    try:
        assert srv.submit("small").result(30).step == 1
        fb = srv.submit("big")                 # admission evicts "small" (slowly)
        assert f.offloading.wait(30)
        fs = srv.submit("small")               # arrives during the eviction
        assert fb.result(30).step == 1
        assert fs.result(30).step == 2         # stepped after the eviction, reloaded
        assert srv.reload_count("small") == 1
        assert np.all(srv.state("small") == _expected(0.5, 2))
    finally:
        srv.close()
