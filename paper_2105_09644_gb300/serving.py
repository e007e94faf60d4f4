"""Serving loop: continuous batching of TreeRay/OnTheSpot requests on one GPU.

Requests (a grid snapshot with its own sources and ray resolution) arrive
over time.  The loop

* admits waiting requests while their HBM footprint fits the budget (first
  come first served, a smaller request may pass a larger one that does not
  fit yet);
* builds an admitted request's tree once and keeps it resident until the
  request is done;
* launches ONE persistent walk kernel (tr_walk_sweep_batch) at a time over
  a slice of the remaining target cells of every active request: requests
  with the least remaining work get their slice first, large requests are cut
  into Morton ranges so that they do not hold up small ones; while it runs,
  new arrivals are admitted, uploaded and built on a second stream, and
  finished results copied back;
* retires a request when its last slice is done and records its latency
  (completion - arrival).

The scheduling part (`Scheduler`) is plain Python without device calls, so
it can be tested on the CPU; `Server` adds the device work through the C ABI.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                      # seconds on the server clock
    N: int
    dx: float
    n_H: np.ndarray                     # (N, N, N) float64
    src_xyz: np.ndarray                 # (S, 3) float64 cm
    src_Q: np.ndarray                   # (S,) float64 s^-1
    nside: int = 2
    theta_lim: float = 0.5
    theta_src: float = math.inf
    make: object = None                 # optional: fills n_H, src_xyz, src_Q when called (lazy request data)
    # filled by the server
    admitted: float | None = None
    footprint: int = 0                  # device bytes counted against the budget while resident
    done: float | None = None
    next_target: int = 0
    result: dict | None = None

    @property
    def n_targets(self) -> int:
        return self.N ** 3

    @property
    def remaining(self) -> int:
        return self.n_targets - self.next_target

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


def num_points(N: int, eta_r: int = 2) -> int:
    """N_R of a uniform N^3 grid with the default L_ray (the box diagonal, Eq. 5)."""
    return eta_r * int(math.floor(math.sqrt(2.0 * N * math.sqrt(3.0)))) + 1


def footprint_bytes(N: int, precision: int, n_sources: int = 1000, eta_r: int = 2) -> int:
    """Device bytes a request holds while resident, counted per allocation
    and each rounded up to 2 MiB (an upper bound: the device allocator
    rounds large allocations to 2 MiB and packs small ones together): the
    library's tree (node records and build sums; the FP32 forms keep the
    FP64 tree beside the FP32 one, and a word for its error bound), mapped
    emission, status words and counters, the job record, the twelve ray
    tables; and the request's inputs and outputs.  The node->ray table of
    each N_side is shared by all requests and is not counted here."""
    def rounded(b):
        return max(1, -(-int(b) // (2 << 20))) * (2 << 20)
    n_nodes = ((1 << (3 * (int(math.log2(N)) + 1))) - 1) // 7
    cells = N ** 3
    nr = num_points(N, eta_r)
    lib = [n_nodes * 64, n_nodes * 24] if precision == 0 else [n_nodes * 32, n_nodes * 12, n_nodes * 64,
                                                                n_nodes * 24, 4]
    lib += [cells * 8, 16, 64, 4, 512]                                     # emission, status, stats, counter, job
    lib += [nr * 8] * 5 + [nr * nr * 8] * 7                                # ray tables
    io = [cells * 8, n_sources * 32, cells * 8, cells * 8, cells]          # n_H, sources, F, e, ion
    return sum(rounded(b) for b in lib + io)


class Scheduler:
    """Admission by footprint and slicing of the active requests' targets."""

    def __init__(self, budget_bytes: int, tick_targets: int, precision: int = 1, min_slice: int = 4096):
        self.budget = budget_bytes
        self.tick_targets = tick_targets
        self.precision = precision
        self.min_slice = min_slice
        self.waiting: list[Request] = []
        self.active: list[Request] = []
        self.finished: list[Request] = []
        self.in_use = 0

    def submit(self, req: Request):
        self.waiting.append(req)

    def admit(self, now: float) -> list[Request]:
        admitted = []
        for req in list(self.waiting):
            fp = footprint_bytes(req.N, self.precision, len(req.src_Q) if req.src_Q is not None else 1000)
            req.footprint = fp
            if fp > self.budget:
                raise ValueError(f"request {req.rid} needs {fp} bytes, more than the whole budget {self.budget}")
            if self.in_use + fp <= self.budget:
                self.waiting.remove(req)
                self.active.append(req)
                self.in_use += fp
                req.admitted = now
                admitted.append(req)
        return admitted

    def plan(self) -> list[tuple[Request, int, int]]:
        """Slices (request, first Morton index, count) for one launch: least
        remaining work first, at most tick_targets in total."""
        left = self.tick_targets
        out = []
        for req in sorted(self.active, key=lambda r: (r.remaining, r.arrival)):
            if left <= 0:
                break
            take = min(req.remaining, max(left, self.min_slice))
            if take > 0:
                out.append((req, req.next_target, take))
                left -= take
        return out

    def complete(self, slices, now: float) -> list[Request]:
        done = []
        for req, first, count in slices:
            assert first == req.next_target
            req.next_target += count
            if req.remaining == 0:
                req.done = now
                self.active.remove(req)
                self.in_use -= req.footprint
                self.finished.append(req)
                done.append(req)
        return done

    def idle(self) -> bool:
        return not self.waiting and not self.active


class Server:
    """Scheduler plus the device work (tree builds and batched walks).

    The batched walk runs on a stream of its own, launched from a worker
    thread (the C call releases the interpreter lock and returns when its
    launch is done), so that while one batch is on the GPU the host keeps
    admitting arrivals, uploads their inputs and builds their trees on a
    side stream, and copies finished results back to pinned host memory.
    The next batch waits on the builds of the trees it walks (CUDA events),
    not on the host.

    keep_results=False returns each result to the host and keeps only a
    summary (the flux total), for long streams whose results would not fit
    in host memory together."""

    def __init__(self, budget_bytes: int, tick_targets: int = 1 << 20, precision: int = 1, device=None,
                 keep_results: bool = True):
        import concurrent.futures
        import torch
        from . import binding as B
        self.B = B
        self.torch = torch
        self.dev = device or torch.device("cuda")
        self.sched = Scheduler(budget_bytes, tick_targets, precision)
        self.precision = precision
        self.state: dict[int, dict] = {}
        self.t0 = time.perf_counter()
        self.launches = 0
        self.keep_results = keep_results
        self.side = None                                        # uploads, builds, result copies
        self.walk = None                                        # batched walks (both made on first use)
        self.worker = concurrent.futures.ThreadPoolExecutor(max_workers=1)
        self.inflight = None                                    # (future, slices) of the running batch
        self.copies = []                                        # results on their way to the host

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.sched.submit(req)

    def _streams(self):
        if self.side is None:
            self.side = self.torch.cuda.Stream(device=self.dev)
            self.walk = self.torch.cuda.Stream(device=self.dev)

    def _start(self, req: Request):
        """Upload the request and build its tree on the side stream (no wait)."""
        torch, B = self.torch, self.B
        self._streams()
        with torch.cuda.stream(self.side):
            d = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().to(self.dev, non_blocking=True)
                 for k, a in (("n_H", req.n_H), ("xyz", req.src_xyz), ("Q", req.src_Q))}
            shape = (req.N,) * 3
            d["F"] = torch.empty(shape, dtype=torch.float64, device=self.dev)
            d["e"] = torch.empty_like(d["F"])
            d["ion"] = torch.empty(shape, dtype=torch.uint8, device=self.dev)
            p = B.tr_params_default(nside=req.nside, theta_lim=req.theta_lim, theta_src=req.theta_src,
                                    precision=self.precision)
            d["tree"] = B.tr_build_tree(B.make_grid(d["n_H"], req.dx), B.make_sources(d["xyz"], d["Q"]), p,
                                        stream=self.side)
            d["ready"] = torch.cuda.Event()
            d["ready"].record(self.side)
        self.state[req.rid] = d
        if req.make is not None:                 # the host copy of lazy request data is no longer needed
            req.n_H = None

    def _launch(self, slices):
        self._streams()
        st = [self.state[r.rid] for r, _, _ in slices]
        for d in st:
            self.walk.wait_event(d["ready"])
        fut = self.worker.submit(self.B.tr_walk_sweep_batch, [d["tree"] for d in st], [f for _, f, _ in slices],
                                 [c for _, _, c in slices], [d["F"] for d in st], [d["e"] for d in st],
                                 [d["ion"] for d in st], self.walk)
        self.inflight = (fut, slices)

    def _retire(self):
        fut, slices = self.inflight
        fut.result()                             # raises what the batch raised
        self.inflight = None
        self.launches += 1
        for req in self.sched.complete(slices, self.now()):
            self._finish(req)

    def _finish(self, req: Request):
        """Copy a finished request's results to pinned host memory (side stream)."""
        torch = self.torch
        d = self.state.pop(req.rid)
        with torch.cuda.stream(self.side):
            host = {k: torch.empty(d[k].shape, dtype=d[k].dtype, pin_memory=True) for k in ("F", "e", "ion")}
            for k in host:
                host[k].copy_(d[k], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.side)
        self.copies.append((req, ev, host, d))

    def _drain(self, block: bool = False):
        left = []
        for req, ev, host, d in self.copies:
            if block:
                ev.synchronize()
            if not ev.query():
                left.append((req, ev, host, d))
                continue
            res = {k: v.numpy() for k, v in host.items()}
            req.result = res if self.keep_results else dict(F_sum=float(res["F"].sum()), ionised=int(res["ion"].sum()))
        self.copies = left

    def tick(self) -> int:
        """One scheduling round: admit and start builds, retire the running
        batch if it is done, launch the next; returns targets launched."""
        for req in self.sched.admit(self.now()):
            self._start(req)
        if self.inflight is not None and self.inflight[0].done():
            self._retire()
        launched = 0
        if self.inflight is None:
            slices = self.sched.plan()
            if slices:
                self._launch(slices)
                launched = sum(c for _, _, c in slices)
        self._drain()
        return launched

    def run(self, requests: list[Request], prefetch: int = 4) -> list[Request]:
        """Replay requests at their arrival times (seconds after start).
        Requests with lazy data are filled by a host thread in arrival order,
        at most `prefetch` ahead of the ones already on the device."""
        import threading
        pending = sorted(requests, key=lambda r: r.arrival)
        ready = [threading.Event() for _ in pending]
        slots = threading.Semaphore(prefetch)

        def fill():
            for k, r in enumerate(pending):
                if r.make is not None:
                    slots.acquire()
                    r.make(r)
                ready[k].set()

        filler = threading.Thread(target=fill, daemon=True)
        filler.start()
        self.t0 = time.perf_counter()
        i = 0
        try:
            while i < len(pending) or not self.sched.idle() or self.inflight is not None:
                now = self.now()
                while i < len(pending) and pending[i].arrival <= now and ready[i].is_set():
                    self.submit(pending[i])
                    i += 1
                started = [r for r in self.sched.waiting]
                if self.tick() == 0:
                    time.sleep(0.0005 if self.inflight is not None else
                               max(0.0, min(0.002, pending[i].arrival - self.now())) if i < len(pending) else 0.0005)
                for r in started:
                    if r.make is not None and r.admitted is not None and r.n_H is None:
                        slots.release()
        finally:
            if self.inflight is not None:
                self.inflight[0].result()
                self.inflight = None
            self._drain(block=True)
            filler.join()
        return self.sched.finished


def poisson_stream(n: int, rate_hz: float, seed: int, sizes=(32, 64, 128, 256), nsides=(2, 4),
                   max_sources: int = 1000, box_pc: float = 10.0, lazy: bool = False) -> list[Request]:
    """Seeded request stream: Poisson arrivals, grid size uniform over `sizes`,
    N_side uniform over `nsides`, theta_lim = 0.5, log-normal k^-4 density,
    1..max_sources sources (log-uniform count).
    lazy=True draws each request's density and sources only when the server
    asks for them (the same values either way)."""
    from workloads import PC_CM, lognormal_density, uniform_sources
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    box = box_pc * PC_CM

    def maker(k, N, S):
        def make(req):
            req.n_H = lognormal_density(N, seed * 1000 + k)
            req.src_xyz, req.src_Q = uniform_sources(S, box, seed * 1000 + k + 500, 46.0, 49.0)
        return make

    for k in range(n):
        t += rng.exponential(1.0 / rate_hz)
        N = int(rng.choice(sizes))
        nside = int(rng.choice(nsides))
        S = int(round(10 ** rng.uniform(0.0, math.log10(max_sources))))
        req = Request(k, t, N, box / N, None, None, None, nside=nside, theta_lim=0.5, make=maker(k, N, S))
        if not lazy:
            req.make(req)
            req.make = None
        out.append(req)
    return out


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))
    return xs[k]
