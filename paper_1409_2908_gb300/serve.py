"""Serving loop for GEMM requests of mixed shapes: continuous batching with
admission by device memory, operands kept on the device, requests grouped by
plan and launched as captured CUDA graphs, latency percentiles beside
throughput.

  * A request brings its operands (device tensors) and an arrival time.
  * Requests are admitted in arrival order while their output and workspace
    fit the memory budget and a stream slot is free; a request arriving while
    others run is admitted as soon as slots and memory free up.
  * Admitted requests that share a plan and a shape form a group.  A shape
    that recurs is replayed from a CUDA graph captured once per plan, shape
    and slot (fixed operand buffers; capture runs on the slot's stream
    without a device-wide synchronisation); a shape's first occurrence runs
    directly.
  * With group_shapes, admitted requests of DIFFERENT shapes whose plans are
    emulated FP64 with at most one recursive level go out together as one
    fmm_gemm_grouped call (up to max_group per call): their residue GEMMs run
    as one grouped tensor-core launch, which fills the GPU where a single
    small product cannot.  Shapes with a captured graph keep the graph path.
  * Groups on different streams overlap on the device; completion is polled
    with CUDA events.

Every product runs through the library's C ABI (fmm_gemm); the plans come
from the autotuner.  Plans are deterministic (stored-product or emulated
schemes), so a result does not depend on what else is running.
"""
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np

import paper_1409_2908_gb300 as fmm


@dataclass
class Request:
    rid: int
    A: object                 # device tensor m x k (float64)
    B: object                 # device tensor k x n
    arrival: float            # seconds from the start of the run
    C: object = None
    t_admit: float = -1.0
    t_done: float = -1.0

    @property
    def shape(self):
        return (self.A.shape[0], self.A.shape[1], self.B.shape[1])

    @property
    def flops(self):
        m, k, n = self.shape
        return 2.0 * m * k * n


@dataclass
class _Graph:
    graph: object
    A: object
    B: object
    C: object
    ws: object
    nbytes: int
    done: object = None       # event after the last replay (its buffers are free once it has passed)


@dataclass
class _Group:
    reqs: list
    event: object
    stream: object
    nbytes: int


@dataclass
class Stats:
    completed: int = 0
    wall_s: float = 0.0
    flops: float = 0.0
    latencies: list = field(default_factory=list)
    waits: list = field(default_factory=list)       # admission minus arrival (queueing)
    services: list = field(default_factory=list)    # completion minus admission
    max_waiting: int = 0                            # most requests arrived but not admitted
    graphs_captured: int = 0
    graph_replays: int = 0
    max_inflight: int = 0
    grouped_calls: int = 0                          # fmm_gemm_grouped calls
    grouped_requests: int = 0                       # requests they carried

    def summary(self):
        lat = np.array(self.latencies) * 1e3
        wt = np.array(self.waits) * 1e3
        sv = np.array(self.services) * 1e3

        def pct(x, q):
            return float(np.percentile(x, q)) if len(x) else None
        return {"requests": self.completed, "wall_s": self.wall_s,
                "effective_tflops": self.flops / self.wall_s / 1e12 if self.wall_s else 0.0,
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "wait_p50_ms": pct(wt, 50), "wait_p99_ms": pct(wt, 99),
                "service_p50_ms": pct(sv, 50), "service_p99_ms": pct(sv, 99),
                "max_waiting": self.max_waiting,
                "graphs_captured": self.graphs_captured, "graph_replays": self.graph_replays,
                "max_inflight_groups": self.max_inflight, "grouped_calls": self.grouped_calls,
                "grouped_requests": self.grouped_requests,
                "mean_group_size": (self.grouped_requests / self.grouped_calls) if self.grouped_calls else None}


class Server:
    def __init__(self, tuner, memory_budget_bytes, slots=4, graph_cache_bytes=None, use_graphs=True,
                 keep_results=True, group_shapes=False):
        import torch
        self.tuner = tuner
        self.budget = int(memory_budget_bytes)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_slots = deque(range(slots))
        self.use_graphs = use_graphs
        self.keep_results = keep_results   # False: a result is dropped once complete (handed off)
        self.graph_cache_bytes = graph_cache_bytes if graph_cache_bytes is not None else self.budget // 2
        self._graphs = OrderedDict()      # (plan key, shape, slot) -> _Graph
        self._graph_bytes = 0
        self._seen = {}
        self._slot_ws = [None] * slots     # per-slot workspace, grown on demand
        self._slot_wss = [[] for _ in range(slots)]   # per-slot workspaces of grouped calls
        self.group_shapes = group_shapes
        self.used = 0
        self.stats = Stats()

    # ------------------------------------------------------------ memory
    def _bytes(self, plan, m, k, n):
        return 8 * m * n + plan.workspace_size(m, k, n)

    def _plan(self, m, k, n):
        p = self.tuner.plan(m, k, n)
        if not getattr(p, "_prepared", False):
            p.prepare()
            p._prepared = True
        return p

    # ------------------------------------------------------------ launch
    def _graph_for(self, plan, shape, slot):
        """The graph of (plan, shape), captured on first use; None while its
        previous replay (on any stream) may still be using its buffers."""
        import torch
        key = (id(plan), shape)
        g = self._graphs.get(key)
        if g is not None:
            if g.done is not None and not g.done.query():
                return None
            self._graphs.move_to_end(key)
            return g
        m, k, n = shape
        nbytes = 8 * (m * k + k * n + m * n) + plan.workspace_size(m, k, n)
        # evict least recently used graphs that are idle (a graph whose last
        # replay has not passed may still be reading its buffers)
        for old_key in list(self._graphs):
            if self._graph_bytes + nbytes <= self.graph_cache_bytes:
                break
            old = self._graphs[old_key]
            if old.done is None or old.done.query():
                self._graph_bytes -= self._graphs.pop(old_key).nbytes
        A = torch.empty((m, k), dtype=torch.float64, device="cuda")
        B = torch.empty((k, n), dtype=torch.float64, device="cuda")
        C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        wsz = plan.workspace_size(m, k, n)
        ws = torch.empty(wsz, dtype=torch.uint8, device="cuda") if wsz else None
        stream = self.streams[slot]
        graph = torch.cuda.CUDAGraph()
        # capture on the slot's own stream: no device-wide synchronisation, so
        # groups running on the other streams keep going
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            graph.capture_begin(capture_error_mode="relaxed")
            try:
                fmm.gemm(plan, A, B, C=C, workspace=ws, stream=stream)
            finally:
                graph.capture_end()
        g = _Graph(graph, A, B, C, ws, nbytes)
        self._graphs[key] = g
        self._graph_bytes += nbytes
        self.stats.graphs_captured += 1
        return g

    def _workspace(self, slot, nbytes):
        """The slot's workspace, grown to `nbytes` if needed.  It is allocated
        on the slot's stream, so work queued there uses it in order and a
        replaced buffer is only reused by later work on that stream."""
        import torch
        if not nbytes:
            return None
        ws = self._slot_ws[slot]
        if ws is None or ws.numel() < nbytes:
            with torch.cuda.stream(self.streams[slot]):
                ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self._slot_ws[slot] = ws
        return ws

    @staticmethod
    def _groupable(plan, shape, sms=152):
        """Emulated products (at most one level) whose residue GEMM alone has
        fewer tiles than the GPU has SMs: grouping several such products into
        one launch fills the GPU; larger products run better on their own
        streams, where one product's memory passes overlap another's GEMM."""
        if plan.precision != "ozaki_bf16" or plan.levels > 1 or (plan.flags & fmm.FLAG_TC_FUSED_S):
            return False
        m, k, n = shape
        M, K, N = (plan.dims if plan.levels else (1, 1, 1))
        R = plan.rank if plan.levels else 1
        mL, nL = m // M, n // N
        tiles = R * (plan.moduli or 15) * -(-mL // 128) * -(-nL // (256 if nL >= 256 else 128))
        return tiles < sms

    def _workspaces(self, slot, sizes):
        """One workspace per product of a grouped call on this slot (grown on
        demand, allocated on the slot's stream like _workspace)."""
        import torch
        wss = self._slot_wss[slot]
        out = []
        for i, nb in enumerate(sizes):
            if not nb:
                out.append(None)
                continue
            while len(wss) <= i:
                wss.append(None)
            if wss[i] is None or wss[i].numel() < nb:
                with torch.cuda.stream(self.streams[slot]):
                    wss[i] = torch.empty(nb, dtype=torch.uint8, device="cuda")
            out.append(wss[i])
        return out

    def _launch_grouped(self, reqs, plans, slot):
        import torch
        stream = self.streams[slot]
        with torch.cuda.stream(stream):
            Cs = [torch.empty((r.shape[0], r.shape[2]), dtype=torch.float64, device="cuda") for r in reqs]
            wss = self._workspaces(slot, [p.workspace_size(*r.shape) for p, r in zip(plans, reqs)])
            fmm.gemm_grouped(plans, [r.A for r in reqs], [r.B for r in reqs], Cs=Cs, workspaces=wss, stream=stream)
            for r, C in zip(reqs, Cs):
                r.C = C
            ev = torch.cuda.Event()
            ev.record(stream)
        self.stats.grouped_calls += 1
        self.stats.grouped_requests += len(reqs)
        return _Group(reqs, ev, stream, sum(self._bytes(p, *r.shape) for p, r in zip(plans, reqs)))

    def _launch(self, group_reqs, plan, slot):
        import torch
        stream = self.streams[slot]
        m, k, n = group_reqs[0].shape
        nbytes = 0
        with torch.cuda.stream(stream):
            for r in group_reqs:
                r.C = torch.empty((m, n), dtype=torch.float64, device="cuda")
                shape_key = (id(plan), (m, k, n))
                self._seen[shape_key] = self._seen.get(shape_key, 0) + 1
                # a shape seen before is replayed from a captured graph; the
                # first occurrence runs directly (capturing a one-off shape buys nothing)
                g = self._graph_for(plan, (m, k, n), slot) if (self.use_graphs and self._seen[shape_key] > 1) else None
                if g is not None:
                    g.A.copy_(r.A, non_blocking=True)
                    g.B.copy_(r.B, non_blocking=True)
                    g.graph.replay()
                    r.C.copy_(g.C, non_blocking=True)
                    g.done = torch.cuda.Event()
                    g.done.record(stream)
                    self.stats.graph_replays += 1
                else:
                    fmm.gemm(plan, r.A, r.B, C=r.C, workspace=self._workspace(slot, plan.workspace_size(m, k, n)),
                             stream=stream)
                nbytes += self._bytes(plan, m, k, n)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _Group(group_reqs, ev, stream, nbytes)

    # ------------------------------------------------------------ loop
    def run(self, requests, max_group=8):
        """Serve `requests` (sorted by arrival); returns the stats summary."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue = deque()                 # admission order (entries already admitted are skipped)
        by_shape = {}                   # shape -> deque of waiting requests, in arrival order
        waiting = 0
        inflight = []
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                queue.append(r)
                by_shape.setdefault(r.shape, deque()).append(r)
                waiting += 1
                self.stats.max_waiting = max(self.stats.max_waiting, waiting)
            # retire finished groups
            still = []
            for g in inflight:
                if g.event.query():
                    done = time.perf_counter() - t0
                    for r in g.reqs:
                        r.t_done = done
                        if not self.keep_results:
                            r.C = None
                        self.stats.latencies.append(done - r.arrival)
                        self.stats.waits.append(r.t_admit - r.arrival)
                        self.stats.services.append(done - r.t_admit)
                        self.stats.flops += r.flops
                        self.stats.completed += 1
                    self.used -= g.nbytes
                    self.free_slots.append(self.streams.index(g.stream))
                else:
                    still.append(g)
            inflight = still
            # admit and group by (plan, shape) while memory and slots allow
            while waiting and self.free_slots:
                while queue[0].t_admit >= 0:
                    queue.popleft()
                head = queue[0]
                plan = self._plan(*head.shape)
                need = self._bytes(plan, *head.shape)
                if self.used + need > self.budget and inflight:
                    break
                graphed = self.use_graphs and self._seen.get((id(plan), head.shape), 0) >= 1
                if self.group_shapes and self._groupable(plan, head.shape) and not graphed:
                    # requests of any shape, in arrival order, whose plans group
                    group, plans, total = [], [], 0
                    for r in queue:
                        if len(group) >= max_group:
                            break
                        if r.t_admit >= 0:
                            continue
                        pr = self._plan(*r.shape)
                        nb = self._bytes(pr, *r.shape)
                        if not self._groupable(pr, r.shape) or (self.use_graphs and
                                                                self._seen.get((id(pr), r.shape), 0) >= 1):
                            continue
                        if group and self.used + total + nb > self.budget:
                            break
                        group.append(r)
                        plans.append(pr)
                        total += nb
                    for r, pr in zip(group, plans):
                        r.t_admit = now
                        by_shape[r.shape].remove(r)
                        if not by_shape[r.shape]:
                            del by_shape[r.shape]
                        key = (id(pr), r.shape)
                        self._seen[key] = self._seen.get(key, 0) + 1
                    waiting -= len(group)
                    slot = self.free_slots.popleft()
                    g = self._launch_grouped(group, plans, slot)
                else:
                    same = by_shape[head.shape]
                    group = []
                    while same and len(group) < max_group and (not group or self.used + need * (len(group) + 1)
                                                               <= self.budget):
                        group.append(same.popleft())
                    if not same:
                        del by_shape[head.shape]
                    for r in group:
                        r.t_admit = now
                    waiting -= len(group)
                    slot = self.free_slots.popleft()
                    g = self._launch(group, plan, slot)
                self.used += g.nbytes
                inflight.append(g)
                self.stats.max_inflight = max(self.stats.max_inflight, len(inflight))
            if not waiting and not inflight and pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.001)))
        self.stats.wall_s = time.perf_counter() - t0
        return self.stats.summary()


def request_shapes(count, lo=256, hi=8192, seed=1409, shape_pool=0):
    """m, k, n of each request, each log-uniform in [lo, hi]; with
    shape_pool > 0 the requests draw (uniformly) from that many such shapes,
    so shapes recur as they do when a service sees a fixed set of models."""
    g = np.random.default_rng(seed)
    if shape_pool:
        pool = np.exp(g.uniform(np.log(lo), np.log(hi), size=(shape_pool, 3))).astype(int)
        return pool[g.integers(0, shape_pool, size=count)]
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=(count, 3))).astype(int)


def poisson_requests(count, rate_per_s, lo=256, hi=8192, seed=1409, device="cuda", pool=None, shape_pool=0):
    """Requests with Poisson arrivals and m, k, n each log-uniform in
    [lo, hi]; operands uniform[-1, 1] on the device.  With `pool` (a 1-D
    float64 device tensor of at least hi*hi elements) the operands are views
    of it instead of fresh allocations (the operands stay device-resident and
    a long stream of requests fits in memory)."""
    import torch
    g = np.random.default_rng(seed + 1)
    t = np.cumsum(g.exponential(1.0 / rate_per_s, size=count))
    dims = request_shapes(count, lo, hi, seed, shape_pool)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    reqs = []
    for i in range(count):
        m, k, n = (int(x) for x in dims[i])
        if pool is not None:
            A = pool[:m * k].view(m, k)
            B = pool[m * k:m * k + k * n].view(k, n) if m * k + k * n <= pool.numel() else pool[:k * n].view(k, n)
        else:
            A = torch.rand((m, k), dtype=torch.float64, device=device, generator=gen) * 2 - 1
            B = torch.rand((k, n), dtype=torch.float64, device=device, generator=gen) * 2 - 1
        reqs.append(Request(i, A, B, float(t[i])))
    return reqs
