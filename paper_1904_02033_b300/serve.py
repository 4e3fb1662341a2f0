"""Continuous-batching server for encrypted distance queries.

Keeps keys-independent state resident (each database's encoded plaintexts
and, for the tensor-core path, its digit layout) and serves a stream of
encrypted queries.  Requests that arrive while other batches are on the GPU
wait until an execution slot and device memory free up; then every waiting
request of one database (up to `max_batch`, FIFO) is admitted as one batch
and launched on its own stream, so batches overlap on the device.  A batch
of `batched_min` or more queries may run on the tensor-core path, smaller
ones run on the per-query path; once the executor is calibrated, a batch
takes whichever path its measured service times say is faster for that
database and batch size (the tensor path's per-call query expansion only
pays back over enough blocks).  Both give bit-identical ciphertexts, so a
request's result does not depend on what it was batched with.

The scheduler is plain host logic over an `Executor` interface, which makes
it testable without a GPU (tests drive it with a fake executor and a fake
clock).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Protocol


@dataclasses.dataclass
class Request:
    rid: int
    db: str
    arrival: float              # seconds on the scheduler clock
    payload: object = None      # executor-specific (query ciphertext, qid)
    start: float | None = None
    done: float | None = None
    result: object = None
    error: str | None = None    # set when the request cannot be served

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


class Executor(Protocol):
    def bytes_for(self, db: str, n_queries: int) -> int: ...
    def launch(self, db: str, reqs: list[Request], slot: int) -> object: ...
    def ready(self, handle: object) -> bool: ...
    def finish(self, handle: object, reqs: list[Request]) -> None: ...


@dataclasses.dataclass
class Stats:
    latencies: list = dataclasses.field(default_factory=list)
    batches: list = dataclasses.field(default_factory=list)   # (db, size, t_launch)
    deferred: int = 0                                          # admissions held back for memory
    rejected: int = 0                                          # requests larger than the whole budget

    def percentile(self, p: float) -> float:
        xs = sorted(self.latencies)
        if not xs:
            return float("nan")
        k = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
        return xs[k]


class Scheduler:
    """Admission by free execution slots and a device-memory budget."""

    def __init__(self, executor: Executor, max_batch: int = 128, slots: int = 3,
                 mem_budget: int = 1 << 40, clock: Callable[[], float] = time.perf_counter,
                 batch_window: float = 0.0):
        self.ex = executor
        self.max_batch = max_batch
        self.slots = slots
        self.mem_budget = mem_budget
        self.clock = clock
        # a database's queue is admitted once it holds max_batch requests or
        # its oldest request has waited batch_window seconds (0: at once)
        self.batch_window = batch_window
        self.waiting: dict[str, collections.deque] = collections.defaultdict(collections.deque)
        self.inflight: list[tuple[object, list[Request], int, int]] = []  # handle, reqs, bytes, slot
        self.mem_used = 0
        self.stats = Stats()

    def submit(self, req: Request):
        self.waiting[req.db].append(req)

    def _free_slot(self) -> int | None:
        used = {s for _, _, _, s in self.inflight}
        for s in range(self.slots):
            if s not in used:
                return s
        return None

    def poll(self) -> int:
        """Retire finished batches, then admit as many waiting batches as slots
        and memory allow.  Returns the number of requests retired."""
        retired = 0
        still = []
        for h, reqs, nbytes, slot in self.inflight:
            if self.ex.ready(h):
                self.ex.finish(h, reqs)
                now = self.clock()
                for r in reqs:
                    r.done = now
                    self.stats.latencies.append(r.latency)
                self.mem_used -= nbytes
                retired += len(reqs)
            else:
                still.append((h, reqs, nbytes, slot))
        self.inflight = still
        while True:
            slot = self._free_slot()
            if slot is None:
                break
            # oldest waiting request decides which database goes next, among
            # the queues that are full or have waited out the batching window
            now = self.clock()
            cands = [(q[0].arrival, db) for db, q in self.waiting.items()
                     if q and (self.batch_window <= 0 or len(q) >= self.max_batch
                               or now - q[0].arrival >= self.batch_window)]
            if not cands:
                break
            _, db = min(cands)
            q = self.waiting[db]
            if self.ex.bytes_for(db, 1) > self.mem_budget:
                # no amount of retiring frees enough memory for this request
                # alone: it is rejected rather than held at the queue's head
                r = q.popleft()
                r.done = self.clock()
                r.error = "needs more device memory than the admission budget"
                self.stats.rejected += 1
                continue
            nq = min(len(q), self.max_batch)
            while nq > 0 and self.mem_used + self.ex.bytes_for(db, nq) > self.mem_budget:
                nq //= 2
            if nq == 0:
                self.stats.deferred += 1
                break
            reqs = [q.popleft() for _ in range(nq)]
            now = self.clock()
            for r in reqs:
                r.start = now
            nbytes = self.ex.bytes_for(db, nq)
            h = self.ex.launch(db, reqs, slot)
            self.mem_used += nbytes
            self.inflight.append((h, reqs, nbytes, slot))
            self.stats.batches.append((db, nq, now))
        return retired

    def idle(self) -> bool:
        return not self.inflight and not any(self.waiting.values())


def run_open_loop(sched: Scheduler, arrivals: list[Request], poll_sleep: float = 0.0,
                  clock: Callable[[], float] | None = None) -> Stats:
    """Replay requests at their arrival times (relative to the start) and keep
    polling until every one of them has been served."""
    clock = clock or sched.clock
    t0 = clock()
    i = 0
    pending = sorted(arrivals, key=lambda r: r.arrival)
    for r in pending:
        r.arrival += t0
    while i < len(pending) or not sched.idle():
        now = clock()
        while i < len(pending) and pending[i].arrival <= now:
            sched.submit(pending[i])
            i += 1
        sched.poll()
        if poll_sleep:
            time.sleep(poll_sleep)
    return sched.stats


def interpolate_ms(table: list[tuple[int, float]], n: int) -> float:
    """Service time of a batch of n queries from measured (batch size, ms)
    points: piecewise linear between them, linear beyond the ends."""
    pts = sorted(table)
    if len(pts) == 1:
        b, ms = pts[0]
        return ms * n / b
    # the first segment whose right end reaches n, else the last one
    i = next((i for i in range(1, len(pts)) if n <= pts[i][0]), len(pts) - 1)
    (b0, m0), (b1, m1) = pts[i - 1], pts[i]
    return m0 + (m1 - m0) * (n - b0) / (b1 - b0)


def tensor_path_is_faster(per_query: list[tuple[int, float]], tensor: list[tuple[int, float]],
                          n: int) -> bool:
    """The path decision of a calibrated executor for a batch of n queries."""
    return interpolate_ms(tensor, n) < interpolate_ms(per_query, n)


class GpuExecutor:
    """Executor over libsanns: one CUDA stream and one output buffer set per
    slot; databases and their contexts stay resident."""

    def __init__(self, dbs: dict, slots: int, max_batch: int, batched_min: int = 8,
                 mask_seed: int = 5, keep: Callable[[Request], bool] | None = None):
        import torch

        from . import sanns as S
        self.S, self.torch = S, torch
        self.dbs = dbs                      # name -> (ctx, db)
        self.batched_min = batched_min
        self.mask_seed = mask_seed
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.max_batch = max_batch
        self.tensor_batches = 0             # batches launched on the tensor-core path
        # which finished requests keep their result tensors (all by default);
        # a result is a view of its whole batch's buffers, so keeping one
        # keeps the batch's responses in device memory
        self.keep = keep
        # db -> {"per_query": [(B, ms)], "tensor": [(B, ms)]} once calibrated
        self.costs: dict = {}

    def uses_tensor_path(self, db: str, n_queries: int) -> bool:
        if n_queries < self.batched_min or not getattr(self.dbs[db][1], "batched", False):
            return False
        c = self.costs.get(db)
        return c is None or tensor_path_is_faster(c["per_query"], c["tensor"], n_queries)

    def calibrate(self, pools: dict, per_query_sizes=(1, 2, 4), tensor_sizes=(8, 32, 128),
                  reps: int = 3) -> dict:
        """Time both paths on every database at a few batch sizes (queries
        taken cyclically from pools[db] = (ct, qids)), keep the tables and
        route each later batch to the faster path.  Synchronous; call it
        before serving."""
        torch, S = self.torch, self.S
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = self.streams[0]
        for name, (ctx, d) in self.dbs.items():
            ct, qids = pools[name]
            table = {"per_query": [], "tensor": []}
            paths = [("per_query", per_query_sizes, S.sanns_distances)]
            if getattr(d, "batched", False):
                paths.append(("tensor", [b for b in tensor_sizes if b >= self.batched_min],
                              S.sanns_distances_batched))
            for key, sizes, fn in paths:
                for b in sizes:
                    idx = torch.arange(b, device=ct.device) % ct.shape[0]
                    x, qx = ct.index_select(0, idx).contiguous(), qids.index_select(0, idx).contiguous()
                    with torch.cuda.stream(st):
                        out, srv = fn(ctx, d, x, self.mask_seed, qx, stream=st)
                        ev0.record(st)
                        for _ in range(reps):
                            fn(ctx, d, x, self.mask_seed, qx, out, srv, stream=st)
                        ev1.record(st)
                    ev1.synchronize()
                    table[key].append((b, ev0.elapsed_time(ev1) / reps))
                    del out, srv
            if not table["tensor"]:
                table["tensor"] = [(1, float("inf"))]   # no tensor path on this database
            self.costs[name] = table
        return self.costs

    def bytes_for(self, db: str, n_queries: int) -> int:
        """Device memory one batch holds while in flight: its responses and
        server shares, the concatenated query ciphertexts, and the scratch
        the library allocates for the call (the tensor-core path's query
        multiples)."""
        ctx, d = self.dbs[db]
        per_q = d.K * 2 * ctx.L * ctx.N * 8 + d.n * 4 + ctx.d * 2 * ctx.L * ctx.N * 8
        scratch = self.S.sanns_distances_scratch_bytes(ctx, n_queries,
                                                       self.uses_tensor_path(db, n_queries))
        return n_queries * per_q + scratch

    def launch(self, db: str, reqs: list[Request], slot: int):
        torch, S = self.torch, self.S
        ctx, d = self.dbs[db]
        st = self.streams[slot]
        with torch.cuda.stream(st):
            ct = torch.cat([r.payload[0] for r in reqs]) if len(reqs) > 1 else reqs[0].payload[0]
            qids = torch.cat([r.payload[1] for r in reqs]) if len(reqs) > 1 else reqs[0].payload[1]
            if self.uses_tensor_path(db, len(reqs)):
                self.tensor_batches += 1
                out, srv = S.sanns_distances_batched(ctx, d, ct, self.mask_seed, qids, stream=st)
            else:
                out, srv = S.sanns_distances(ctx, d, ct, self.mask_seed, qids, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, out, srv)

    def ready(self, handle) -> bool:
        return handle[0].query()

    def finish(self, handle, reqs):
        _, out, srv = handle
        for i, r in enumerate(reqs):
            if self.keep is None or self.keep(r):
                r.result = (out[i:i + 1], srv[i:i + 1])
