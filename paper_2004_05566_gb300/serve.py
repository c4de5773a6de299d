"""Continuous-batching service of Crank-Nicolson steps over resident operators.

Each registered operator is one CN problem (grid, coefficient a(x), dt, eps,
reaction) whose HIF factor and state u live on the GPU while it is resident.
Clients submit step requests; a scheduler thread repeatedly takes every
pending request whose operator is not already in the running batch, admits
the operators it needs (factoring them on the GPU, evicting the least
recently used idle operators when the HBM budget would be exceeded), and runs
the whole batch with one ``cn_step_batched`` call, whose steps overlap on the
device.  Requests that arrive while a batch runs join the next one
(step-level continuous batching).  Each request completes with the new step
index, the PCG iteration count and its latency (arrival to result ready).  A
client may cancel a request's future while it is still queued; the step is then
not taken.  Once a request joins a batch its future can no longer be cancelled.

Eviction keeps the operator's handle when the library can offload it: its
large device allocations (factor, indices, work vectors) move to host memory
(``hif_offload``) and come back at the same device addresses on re-admission
(``hif_reload``), a copy instead of a new factorization; the trajectory
continues bit for bit.  Reduced-precision operators drop their FP64 factor
copy after the setup (``hif_release_fp64``, on by default), which the steps
never read.

Size lanes: with ``lanes`` (increasing unknown-count bounds) the operators
are split into size classes, each served by its own scheduler thread and
CUDA stream, so that a batch of large operators (a 3D 127^3 step takes tens
of milliseconds) does not hold back the requests of small ones (2D steps of
about a millisecond): a request joins the next batch of its own lane, and
the lanes' batches overlap on the GPU.  Admission and eviction are shared by
the lanes; an operator in a running batch of any lane is never evicted.

Determinism: every kernel of the library reduces in a fixed order and the
factorization is deterministic, so an operator's trajectory is the same
whether it is stepped alone, in any mix, or after an eviction and re-factor.
"""

from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch

from . import hifcn as H

# device bytes per unknown of a resident 2D operator with FP64 + FP32 factors
# (measured with hif_query on 2D leaf-16 problems); used before the first setup
_BYTES_PER_DOF_ESTIMATE = {2: 2300, 3: 12000}


@dataclass
class OperatorSpec:
    dim: int
    n: int
    leaf: int
    a_nodes: np.ndarray
    dt: float
    eps: float
    u0: np.ndarray
    reaction: tuple = (0, 0.0, 0.0)
    precision: int = H.HIF_FP32
    release_fp64: bool = True  # FP32 / BF16TOP: free the FP64 factor copy after the setup
    lane: int | None = None    # size lane; None: chosen from N by the server's bounds

    @property
    def N(self) -> int:
        return (self.n - 1) ** self.dim


@dataclass
class _Resident:
    handle: H.Handle
    u: torch.Tensor
    out: torch.Tensor
    bytes: int
    last_used: float = 0.0


@dataclass
class _State:
    spec: OperatorSpec
    lane: int = 0
    step: int = 0
    u_host: np.ndarray | None = None  # state while not resident
    resident: _Resident | None = None
    parked: H.Handle | None = None    # offloaded handle while not resident
    setups: int = 0
    reloads: int = 0


@dataclass
class StepResult:
    op_id: object
    step: int
    iters: int
    latency_s: float
    batch_size: int


@dataclass
class _Request:
    op_id: object
    arrival: float
    future: Future = field(default_factory=Future)


class CNServer:
    """Step-level continuous batching of CN steps on one GPU (see module doc)."""

    def __init__(self, hbm_budget_bytes: int, device=0, max_batch: int = 256, lanes=None):
        self.budget = int(hbm_budget_bytes)
        self.device = device if isinstance(device, torch.device) else torch.device("cuda", device)
        self.max_batch = max_batch
        self._bounds = sorted(int(b) for b in lanes) if lanes else []
        nlanes = len(self._bounds) + 1
        self._ops: dict = {}
        self._pending = [collections.deque() for _ in range(nlanes)]
        self._busy: set = set()  # operators in a running batch (never evicted)
        self._cv = threading.Condition()
        self._stop = False
        self._resident_bytes = 0
        self.batches = 0
        self.evictions = 0
        self.reloads = 0
        self._error: BaseException | None = None
        self._threads = [threading.Thread(target=self._loop, args=(i,), name=f"cn-server-{i}", daemon=True)
                         for i in range(nlanes)]
        for t in self._threads:
            t.start()

    def lane_of(self, op_id) -> int:
        """Size lane of a registered operator."""
        return self._ops[op_id].lane

    def _lane_for(self, spec: OperatorSpec) -> int:
        if spec.lane is not None:
            return max(0, min(int(spec.lane), len(self._bounds)))
        for i, b in enumerate(self._bounds):
            if spec.N <= b:
                return i
        return len(self._bounds)

    # -------------------------------------------------------------- client API
    def register(self, op_id, spec: OperatorSpec) -> None:
        with self._cv:
            if op_id in self._ops:
                raise KeyError(f"operator {op_id!r} already registered")
            self._ops[op_id] = _State(spec=spec, lane=self._lane_for(spec),
                                      u_host=np.array(spec.u0, dtype=np.float64).ravel())

    def submit(self, op_id) -> Future:
        req = _Request(op_id, time.perf_counter())
        with self._cv:
            if self._error is not None:
                raise RuntimeError("server stopped after an error") from self._error
            if op_id not in self._ops:
                raise KeyError(op_id)
            self._pending[self._ops[op_id].lane].append(req)
            self._cv.notify_all()
        return req.future

    def state(self, op_id) -> np.ndarray:
        """Current u of an operator (host copy; call when its requests are done)."""
        with self._cv:
            st = self._ops[op_id]
            if st.resident is not None:
                self._sync()
                return st.resident.u.cpu().numpy().copy()
            return st.u_host.copy()

    def setups(self, op_id) -> int:
        with self._cv:
            return self._ops[op_id].setups

    def reload_count(self, op_id) -> int:
        with self._cv:
            return self._ops[op_id].reloads

    def step_count(self, op_id) -> int:
        with self._cv:
            return self._ops[op_id].step

    def resident_bytes(self) -> int:
        return self._resident_bytes

    def close(self) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        for st in self._ops.values():
            if st.resident is not None:
                st.resident.handle.close()
                st.resident = None
            if st.parked is not None:
                st.parked.close()
                st.parked = None

    # -------------------------------------------------------------- scheduler
    def _sync(self) -> None:
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)

    def _estimate(self, spec: OperatorSpec) -> int:
        return _BYTES_PER_DOF_ESTIMATE[spec.dim] * spec.N

    def _evict_one(self, keep: set) -> bool:
        with self._cv:
            cands = [(st.resident.last_used, oid) for oid, st in self._ops.items()
                     if st.resident is not None and oid not in keep and oid not in self._busy]
            if not cands:
                return False
            _, oid = min(cands, key=lambda t: t[0])
            self._busy.add(oid)  # no other lane picks or steps it meanwhile
        st = self._ops[oid]
        self._sync()
        u_host = st.resident.u.cpu().numpy().copy()
        res = st.resident
        parked = None
        offload = getattr(H, "hif_offload", None)
        if offload is not None:
            try:
                offload(res.handle)
                parked = res.handle
            except Exception:  # no virtual memory management: discard the factor
                parked = None
        if parked is None:
            res.handle.close()
        with self._cv:
            st.resident, st.u_host, st.parked = None, u_host, parked
            self._resident_bytes -= res.bytes
            self.evictions += 1
            self._busy.discard(oid)
            self._cv.notify_all()  # a lane may be waiting for this operator
        return True

    def _admit(self, oid, keep: set) -> None:
        st = self._ops[oid]
        if st.resident is not None:
            return
        spec = st.spec
        need = self._estimate(spec)
        while self._resident_bytes + need > self.budget:
            if not self._evict_one(keep):
                break  # admit anyway when nothing else can be evicted
        reloaded = False
        if st.parked is not None:
            h, st.parked = st.parked, None
            H.hif_reload(h)
            reloaded = True
        else:
            a = torch.from_numpy(spec.a_nodes).to(self.device)
            opt = H.default_options(eps=spec.eps, precision=spec.precision, cg_tol=1e-10)
            h = H.hif_setup(spec.dim, spec.n, spec.leaf, a, spec.dt, opt)
            if spec.reaction[0]:
                H.hif_set_reaction(h, *spec.reaction)
            if spec.release_fp64 and spec.precision != H.HIF_FP64 and hasattr(H, "hif_release_fp64"):
                H.hif_release_fp64(h)
        info = H.hif_query(h)
        u = torch.from_numpy(st.u_host).to(self.device)
        with self._cv:
            st.resident = _Resident(h, u, torch.empty_like(u), int(info["device_bytes"]))
            if reloaded:
                st.reloads += 1
                self.reloads += 1
            else:
                st.setups += 1
            self._resident_bytes += st.resident.bytes
        while self._resident_bytes > self.budget and self._evict_one(keep | {oid}):
            pass

    def _take_batch(self, lane: int) -> list:
        """Pending requests of a lane, at most one per operator (the rest stay
        queued).  Cancelled requests are dropped; the ones taken are marked
        running and their operators busy.  An operator that is busy (being
        evicted by another lane) keeps its requests queued."""
        pend = self._pending[lane]
        batch, seen, rest = [], set(), collections.deque()
        while pend and len(batch) < self.max_batch:
            r = pend.popleft()
            if r.future.cancelled():
                continue
            if r.op_id in seen or r.op_id in self._busy:
                rest.append(r)
            elif r.future.set_running_or_notify_cancel():
                seen.add(r.op_id)
                batch.append(r)
        while rest:
            pend.appendleft(rest.pop())
        self._busy |= seen
        return batch

    def _fail_all(self, exc: BaseException) -> None:
        """(lock held) every waiting request of every lane gets the error."""
        self._error = exc
        for pend in self._pending:
            while pend:
                f = pend.popleft().future
                if not f.done():  # a cancelled request stays cancelled
                    f.set_exception(exc)
        self._cv.notify_all()

    def _loop(self, lane: int = 0) -> None:
        stream = None
        if self.device.type == "cuda":
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
        with torch.cuda.stream(stream) if stream is not None else _nullctx():
            self._serve_lane(lane)

    def _serve_lane(self, lane: int) -> None:
        pend = self._pending[lane]
        while True:
            with self._cv:
                while not pend and not self._stop and self._error is None:
                    self._cv.wait()
                if self._error is not None:
                    return
                if self._stop and not pend:
                    return
                batch = self._take_batch(lane)
                if not batch and pend:  # only operators that another lane is evicting
                    self._cv.wait(0.001)
            if not batch:  # everything taken was cancelled
                continue
            try:
                keep = {r.op_id for r in batch}
                for r in batch:
                    self._admit(r.op_id, keep)
                res = [self._ops[r.op_id].resident for r in batch]
                outs, iters = H.cn_step_batched([x.handle for x in res], [x.u for x in res],
                                                outs=[x.out for x in res])
                now = time.perf_counter()
                done = []
                with self._cv:
                    self.batches += 1
                    for r, x, it in zip(batch, res, iters):
                        x.u, x.out = x.out, x.u
                        x.last_used = now
                        st = self._ops[r.op_id]
                        st.step += 1
                        done.append((r, StepResult(r.op_id, st.step, it, now - r.arrival, len(batch))))
                    self._busy -= {r.op_id for r in batch}
                for r, out in done:
                    r.future.set_result(out)
            except BaseException as exc:  # surface to every waiting client
                with self._cv:
                    for r in batch:
                        if not r.future.done():
                            r.future.set_exception(exc)
                    self._busy -= {r.op_id for r in batch}
                    self._fail_all(exc)
                return


class _nullctx:
    def __enter__(self):
        return None

    def __exit__(self, *a):
        return False
