"""Continuous-batching request loop for factor/solve requests on one GPU.

Requests arrive over time (factor + solve of a new matrix, or a repeat solve
on a factor that is already resident).  A fixed number of slots run requests
concurrently, each slot a host thread with its own CUDA stream; the library
calls release the GIL, so the persistent kernels of different slots overlap
on the device.  By default each handle's persistent grid fills the GPU: a
launch that finds the SMs busy starts its CTAs as the running launch's CTAs
retire, so consecutive requests overlap at their boundaries and each runs at
full width (on the serving stream: 47.7 req/s maximum and p99 232 ms at half
of it, against 33.7 req/s and 355 ms with grids capped at one CTA per SM, the
other setting, `ctas_per_sm`).  A request is admitted when a slot
is free and the device bytes of all resident factors plus its own stay within
the memory budget; least-recently-used idle factors are evicted to make room.
A request whose own footprint exceeds the whole budget is rejected
(``spchol.ENOMEM``) instead of waiting.  A handle's footprint is charged with
the solve workspace of the most right-hand sides a request may bring
(``max_nrhs``), so a later repeat solve with more of them stays inside the
budget.  The handles' device memory comes from PyTorch's caching allocator
(``spchol.torch_allocator``) by default: evicting a factor or growing a solve
workspace returns memory to the cache and never calls cudaFree, which would
wait for every other slot's kernels.
Latency is measured from arrival to the moment the result is on the host.  A
request's matrix is client data: a producer thread materializes each request's
matrix ahead of its arrival (if it falls behind, the wait counts as latency).
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time

import numpy as np

from . import spchol


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds, relative to the start of the run
    key: str                  # identity of the sparsity pattern (the analysis is shared)
    vkey: str                 # identity of the values (the factor)
    make: object              # callable returning (CscLower, perm) for this request's matrix
    B: np.ndarray             # n x nrhs, Fortran order
    repeat: bool = False      # True: a repeat solve with a factor that was computed before
    payload: object = None    # (CscLower, perm) once materialized
    # filled by the server
    X: np.ndarray | None = None
    start: float = 0.0
    done: float = 0.0
    rc: int = 0
    factored: bool = False
    # where the latency went (seconds): symbolic analysis of a new pattern, wait
    # for the pattern's handle, numeric factorization, solve and copy back
    t_analyze: float = 0.0
    t_lock: float = 0.0
    t_factor: float = 0.0
    t_solve: float = 0.0


class _Resident:
    def __init__(self, handle, footprint):
        self.h = handle
        self.footprint = footprint
        self.vkey = None  # values currently factored in the handle
        self.lock = threading.Lock()
        self.last_use = time.perf_counter()
        self.busy = 0


class Server:
    def __init__(self, slots: int = 4, budget_bytes: int | None = None, ctas_per_sm: int = 0,
                 precision: int = spchol.FP64, max_width: int = 64, device: int = 0, max_nrhs: int = 16,
                 allocator="torch"):
        import torch

        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(0.8 * free)
        self.budget = budget_bytes
        self.slots = slots
        self.opt_kw = dict(precision=precision, max_width=max_width, ctas_per_sm=ctas_per_sm, allocator=allocator)
        self.max_nrhs = max_nrhs
        self.fp32 = precision in (spchol.FP32, spchol.TF32, spchol.TF32X3)
        self.rejected = 0
        self.resident: dict[str, _Resident] = collections.OrderedDict()
        self.used = 0
        self.mem_cv = threading.Condition()
        self.factorizations = 0
        self.peak_used = 0

    # -------------------------------------------------------------- memory
    def _evict_locked(self, need: int) -> bool:
        """Free idle resident factors (least recently used first) until `need` fits."""
        while self.used + need > self.budget:
            victims = [k for k, r in self.resident.items() if r.busy == 0]
            if not victims:
                return False
            k = min(victims, key=lambda kk: self.resident[kk].last_use)
            r = self.resident.pop(k)
            spchol.destroy(r.h)
            self.used -= r.footprint
        return True

    def _acquire(self, req: Request, A, perm):
        """Resident handle of the request's pattern, analyzing it if needed."""
        with self.mem_cv:
            r = self.resident.get(req.key)
            if r is not None:
                r.busy += 1
                r.last_use = time.perf_counter()
                return r, False
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(**self.opt_kw))
        # the factor plus the solve workspace (Y and B; X and R too with refinement)
        # for the most right-hand sides any request may bring
        nrhs = max(self.max_nrhs, req.B.shape[1], 1)
        fp = spchol.stats(h)["footprint_bytes"] + (4 if self.fp32 else 2) * A.n * nrhs * 8
        if fp > self.budget:  # could never fit, even with every other factor evicted
            spchol.destroy(h)
            with self.mem_cv:
                self.rejected += 1
            return None, False
        with self.mem_cv:
            while True:
                r = self.resident.get(req.key)
                if r is not None:  # another slot created it meanwhile
                    spchol.destroy(h)
                    r.busy += 1
                    return r, False
                if self._evict_locked(fp):
                    break
                self.mem_cv.wait(timeout=0.05)
            r = _Resident(h, fp)
            r.busy = 1
            self.resident[req.key] = r
            self.used += fp
            self.peak_used = max(self.peak_used, self.used)
            return r, True

    def _release(self, r: _Resident):
        with self.mem_cv:
            r.busy -= 1
            r.last_use = time.perf_counter()
            self.mem_cv.notify_all()

    # -------------------------------------------------------------- request execution
    def _run_one(self, req: Request, stream, t0: float):
        torch = self.torch
        req.start = time.perf_counter() - t0
        A, perm = req.payload if req.payload is not None else req.make()
        req.payload = None  # the matrix is not kept after its request
        ta = time.perf_counter()
        r, fresh = self._acquire(req, A, perm)
        tb = time.perf_counter()
        req.t_analyze = tb - ta
        if r is None:  # larger than the whole memory budget
            req.rc = spchol.ENOMEM
            req.done = time.perf_counter() - t0
            return
        try:
            with r.lock:  # one slot at a time per handle
                tc = time.perf_counter()
                req.t_lock = tc - tb
                with torch.cuda.stream(stream):
                    if r.vkey != req.vkey:
                        vals = torch.from_numpy(np.ascontiguousarray(A.values)).cuda(non_blocking=True)
                        rc = spchol.factorize(r.h, vals, stream=stream)
                        req.t_factor = time.perf_counter() - tc
                        r.vkey = req.vkey if rc == 0 else None
                        req.factored = True
                        with self.mem_cv:
                            self.factorizations += 1
                        if rc != 0:
                            req.rc = rc
                            return
                    td = time.perf_counter()
                    nrhs = req.B.shape[1]
                    Bt = torch.from_numpy(np.ascontiguousarray(req.B.T)).cuda(non_blocking=True)
                    try:
                        spchol.solve(r.h, Bt, A.n, nrhs, stream=stream)
                    except spchol.SpcholError as e:
                        if e.code != spchol.ENOCONV:
                            raise
                        req.rc = e.code
                    req.X = np.asfortranarray(Bt.cpu().numpy().T)
                    req.t_solve = time.perf_counter() - td
        finally:
            self._release(r)
            req.done = time.perf_counter() - t0

    def run(self, requests: list[Request]) -> list[Request]:
        """Release requests at their arrival times and serve them with `slots` workers."""
        torch = self.torch
        pending: queue.Queue = queue.Queue()
        t0 = time.perf_counter()
        errors = []

        def worker():
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream()
            while True:
                req = pending.get()
                if req is None:
                    return
                try:
                    self._run_one(req, stream, t0)
                except Exception as e:  # surface to the caller
                    errors.append(e)
                    req.rc = -1

        order = sorted(requests, key=lambda q: q.arrival)
        ready = [threading.Event() for _ in order]

        def producer():  # the clients: each request's matrix, prepared ahead of its arrival
            for i, req in enumerate(order):
                if req.payload is None:
                    req.payload = req.make()
                ready[i].set()

        prod = threading.Thread(target=producer, daemon=True)
        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.slots)]
        prod.start()
        for th in threads:
            th.start()
        for i, req in enumerate(order):
            delay = req.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ready[i].wait()  # a late payload delays the request; its latency still counts from arrival
            pending.put(req)
        prod.join()
        for _ in threads:
            pending.put(None)
        for th in threads:
            th.join()
        if errors:
            raise errors[0]
        return requests

    def close(self):
        with self.mem_cv:
            for r in self.resident.values():
                spchol.destroy(r.h)
            self.resident.clear()
            self.used = 0


class MultiServer:
    """One Server per GPU of the node behind a dispatcher.

    Requests are independent units, so a stream splits over the GPUs with no
    exchange between them: each device runs its own Server (its own slots,
    streams, resident factors and admission against its own memory budget),
    and the dispatcher decides the device of every request before it arrives.
    A sparsity pattern stays on the device that first took it, where its
    analysis and factors are resident, so repeat solves find their factor; a
    new pattern goes to the device with the least work assigned so far.  The
    work of a request is estimated from its size alone, before its matrix
    exists: n^1.5 for a factorization (the flops of a nested-dissection
    factor grow like n^1.5 in 2D and n^2 in 3D) plus n x nrhs for the solve.
    """

    def __init__(self, devices, slots: int = 4, budget_bytes: int | None = None, **kw):
        self.devices = list(devices)
        self.servers = [Server(slots=slots, budget_bytes=budget_bytes, device=d, **kw) for d in self.devices]

    @staticmethod
    def assign(requests: list[Request], ndev: int) -> list[int]:
        """Device index of each request (in the order given), by arrival time."""
        dev_of_key: dict[str, int] = {}
        load = [0.0] * ndev
        out = [0] * len(requests)
        for i in sorted(range(len(requests)), key=lambda k: (requests[k].arrival, k)):
            q = requests[i]
            n, nrhs = q.B.shape[0], (q.B.shape[1] if q.B.ndim > 1 else 1)
            d = dev_of_key.get(q.key)
            if d is None:
                d = min(range(ndev), key=lambda k: (load[k], k))
                dev_of_key[q.key] = d
            out[i] = d
            load[d] += (0.0 if q.repeat else float(n) ** 1.5) + float(n) * nrhs
        return out

    def run(self, requests: list[Request]) -> list[Request]:
        where = self.assign(requests, len(self.servers))
        shares = [[q for q, d in zip(requests, where) if d == k] for k in range(len(self.servers))]
        errors = []

        def drive(srv, reqs):
            try:
                if reqs:
                    srv.run(reqs)
            except Exception as e:  # surface to the caller
                errors.append(e)

        ths = [threading.Thread(target=drive, args=(srv, reqs), daemon=True)
               for srv, reqs in zip(self.servers, shares)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        if errors:
            raise errors[0]
        return requests

    @property
    def factorizations(self) -> int:
        return sum(s.factorizations for s in self.servers)

    def close(self):
        for s in self.servers:
            s.close()


def latency_summary(reqs: list[Request]) -> dict:
    lat = np.array([q.done - q.arrival for q in reqs]) * 1e3
    rep = np.array([q.done - q.arrival for q in reqs if q.repeat]) * 1e3
    span = max(q.done for q in reqs) - min(q.arrival for q in reqs)
    out = {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "solves_per_s": len(reqs) / span if span > 0 else None}
    if rep.size:
        out["repeat_p50_ms"] = float(np.percentile(rep, 50))
        out["repeat_p99_ms"] = float(np.percentile(rep, 99))
    # mean breakdown of the slowest 5 % (arrival to start = wait for a slot)
    tail = [q for q, l in zip(reqs, lat) if l >= np.percentile(lat, 95)]
    if tail:
        parts = {"queue": [q.start - q.arrival for q in tail], "analyze": [q.t_analyze for q in tail],
                 "handle_wait": [q.t_lock for q in tail], "factor": [q.t_factor for q in tail],
                 "solve": [q.t_solve for q in tail]}
        out["tail5_ms"] = {k: float(np.mean(v)) * 1e3 for k, v in parts.items()}
    return out


def make_stream(n_requests: int, rate: float, seed: int = 4321, repeat_frac: float = 0.3, patterns: int = 32,
                small: bool = False) -> list[Request]:
    """Poisson stream (rate requests/s; 0 = all at once) of mixed 2D (32^2..256^2) and
    3D (16^3..48^3) Laplacian / diffusion problems with 1..16 right-hand sides.
    A fresh request carries new values on one of `patterns` sparsity patterns
    (a shift of the Laplacian, a new conductivity field of the diffusion) and
    needs a factorization; `repeat_frac` of the requests repeat a solve with
    the values of an earlier request, whose factor may still be resident.
    `small` shrinks the size ranges (used by the tests)."""
    import gridgen

    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests)) if rate > 0 else np.zeros(n_requests)
    specs = []
    for i in range(patterns):
        dim3 = rng.random() < 0.5
        lap = rng.random() < 0.5
        if dim3:
            side = int(rng.integers(6, 13)) if small else int(rng.integers(16, 49))
        else:
            side = int(rng.integers(10, 33)) if small else int(rng.integers(32, 257))
        specs.append((dim3, lap, side))

    perms = {}  # the ordering depends on the grid only: one per pattern

    def maker(j, v):
        dim3, lap, side = specs[j]

        def make():
            if dim3:
                A = gridgen.laplacian_3d(side, shift=1e-3 * v) if lap else \
                    gridgen.diffusion_3d_27pt(side, sigma=2.0, seed=1000 * j + v)
            else:
                A = gridgen.laplacian_2d(side, shift=1e-3 * v) if lap else \
                    gridgen.diffusion_2d_5pt(side, sigma=2.0, seed=1000 * j + v)
            if j not in perms:
                perms[j] = gridgen.geometric_nd(A.dims)
            return A, perms[j]

        return make

    reqs, issued = [], []
    nvals = [0] * patterns
    for rid in range(n_requests):
        repeat = bool(issued) and rng.random() < repeat_frac
        if repeat:
            j, v = issued[int(rng.integers(0, len(issued)))]
        else:
            j = int(rng.integers(0, patterns))
            v = nvals[j]
            nvals[j] += 1
            issued.append((j, v))
        dim3, lap, side = specs[j]
        n = side ** 3 if dim3 else side ** 2
        nrhs = int(rng.integers(1, 17))
        B = np.asfortranarray(rng.uniform(-1, 1, (nrhs, n)).T)
        reqs.append(Request(rid, float(t[rid]), f"s{seed}p{j}", f"s{seed}p{j}v{v}", maker(j, v), B, repeat=repeat))
    return reqs
