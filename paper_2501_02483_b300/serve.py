"""Continuous-batching request loop over the C ABI.

Requests are factorize + logdet + solve of an arrowhead SPD matrix, or a
re-solve against a factor that is still resident.  The loop:

* admits requests as they arrive: new matrices go through the analysis pool
  (host threads; the C analysis releases the GIL) and then wait for the GPU;
* keeps ``gpu_workers`` GPU jobs in flight, each on its own CUDA stream: as
  soon as a worker is free it takes the analysed requests that fit the HBM
  budget (up to ``max_batch`` matrices and, if set, ``max_job_flops`` tile
  flops, so that later arrivals reach the next job sooner) and runs them as one batched persistent
  factorization (stiles_batch_*), their log-determinants in one launch and
  their first solves in one batched forward/backward sweep (FP64 refinement
  for BF16/FP16 factors).  Requests that arrive meanwhile join the next job,
  whose kernels overlap the running ones (a persistent launch frees its SMs as
  its own tasks run out);
* keeps finished factors resident in an LRU cache bounded by the HBM budget
  (resident plus in-flight bytes); re-solve requests against one resident
  batch are served together by one batched solve that covers only the
  targeted matrices; a re-solve whose factor was evicted is refactorized (and
  counted as a miss).

Plans are cached per pattern (the same structure with new values -- e.g. a
hyperparameter sweep -- reuses the symbolic analysis, Section III.A); a server
can be started with the plans of known patterns (``warm``).

Every GPU job records a CUDA event on its stream before its first call and
after its last; ``intervals()`` returns them on one device clock, so that the
overlap of jobs on the device can be read (``overlap()``).

All numerical work runs in libstiles.so; this module only schedules it.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import os
import threading
import time

from . import stiles as st

__all__ = ["Request", "Server"]

MAX_RHS = 16  # right-hand sides per matrix in one batched solve


class Request:
    """One request: ``kind`` is "new" or "resolve"; ``matrix`` holds n, n_arrow,
    colptr, rowidx, values (new requests) and ``key`` names its pattern; ``rhs``
    is n x nrhs; ``target`` (resolve) is the id of the request whose factor to
    reuse.  ``t_arrival`` is filled in by the server."""

    __slots__ = ("id", "kind", "key", "matrix", "rhs", "target", "t_arrival", "t_done", "logdet", "x", "relres",
                 "status", "refactorized", "batch_size")

    def __init__(self, rid, kind, key=None, matrix=None, rhs=None, target=None):
        self.id = rid
        self.kind = kind
        self.key = key
        self.matrix = matrix
        self.rhs = rhs
        self.target = target
        self.t_arrival = None
        self.t_done = None
        self.logdet = None
        self.x = None
        self.relres = None
        self.status = None
        self.refactorized = False
        self.batch_size = 0


class _Resident:
    """A batch kept on the device; its factors serve re-solves."""

    def __init__(self, batch, members, nbytes):
        self.batch = batch
        self.members = members  # request id -> index in the batch
        self.nbytes = nbytes
        self.busy = 0           # jobs using the batch (not evictable meanwhile)


class Server:
    def __init__(self, precision=st.PREC_BF16, tile=64, ordering=st.ORDER_NONE, hbm_budget=150e9, max_batch=256,
                 analyze_threads=None, refine_tol=1e-10, gpu_workers=2, max_job_flops=None):
        import torch

        self._torch = torch
        self.opts = dict(tile=tile, ordering=ordering, precision=precision, refine_tol=refine_tol)
        self.hbm_budget = float(hbm_budget)
        self.max_batch = max_batch
        self.max_job_flops = max_job_flops
        self.jobs = []             # (kind, requests, start event, end event) per GPU job
        self.kernels = []          # (start ms, end ms) of each factor job's persistent kernel
        if analyze_threads is None:  # the C analysis releases the GIL: one thread per core, up to 32
            analyze_threads = max(1, min(32, os.cpu_count() or 1))
        self.pool = cf.ThreadPoolExecutor(max_workers=analyze_threads)
        self.gpu_pool = cf.ThreadPoolExecutor(max_workers=gpu_workers)
        self.streams = [torch.cuda.Stream() for _ in range(gpu_workers)]
        self.free_streams = list(range(gpu_workers))
        self.plans = {}            # pattern key -> Plan
        self.plan_lock = threading.Lock()
        self.lock = threading.Lock()  # resident cache, byte counts, free streams, stats
        self.resident = collections.OrderedDict()  # resident key -> _Resident (LRU order)
        self.where = {}            # request id -> resident key holding its factor
        self.resident_bytes = 0.0
        self.inflight_bytes = 0.0
        self.stats = collections.Counter()
        self.times = collections.Counter()  # seconds per phase, summed over jobs
        self._next_key = 0

    # -- analysis (host threads) -------------------------------------------
    def warm(self, matrices):
        """Analyse known patterns ahead of the stream: {key: matrix}."""
        futs = [self.pool.submit(self._plan_for_key, k, m) for k, m in matrices.items()]
        for f in futs:
            f.result()

    def _plan_for_key(self, key, matrix):
        with self.plan_lock:
            p = self.plans.get(key)
        if p is not None:
            return p
        p = st.Plan.from_matrix(matrix, **self.opts)
        with self.plan_lock:
            self.plans.setdefault(key, p)
            return self.plans[key]

    def _plan_for(self, req):
        with self.plan_lock:
            p = self.plans.get(req.key)
        if p is not None:
            return p
        t0 = time.perf_counter()
        p = st.Plan.from_matrix(req.matrix, **self.opts)
        with self.plan_lock:
            self.times["analyze"] += time.perf_counter() - t0
            self.plans.setdefault(req.key, p)
            return self.plans[req.key]

    def _bytes(self, plan):
        inf = plan.info()
        # tiles (FP32 + 16-bit copy, or FP64) + values + flags + solve workspace + the diagonal
        # inverses and, for FP64 factors, the sweeps' folded terms (5 B^2 per diagonal sub-tile)
        B = inf["block"]
        nsb = -(-inf["n"] // B)
        per_diag = 40.0 if self.opts["precision"] in (st.PREC_F64, st.PREC_SLICED) else 4.0
        return (float(inf["factor_bytes"]) + 8.0 * inf["nnz"] + 4.0 * inf["nsub"] + 48.0 * MAX_RHS * inf["n"]
                + per_diag * nsb * B * B)

    # -- residency (callers hold self.lock) ----------------------------------
    def _evict_until(self, need):
        for key in list(self.resident.keys()):
            if self.resident_bytes + self.inflight_bytes + need <= self.hbm_budget:
                break
            res = self.resident[key]
            if res.busy:
                continue
            del self.resident[key]
            for rid in res.members:
                self.where.pop(rid, None)
            res.batch.close()
            self.resident_bytes -= res.nbytes
            self.stats["evicted_batches"] += 1

    # -- GPU jobs (worker threads) ---------------------------------------------
    def _event(self, stream):
        e = self._torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def _job_factor(self, reqs, plans, nbytes, si):
        stream = self.streams[si]
        ev0 = self._event(stream)
        t0 = time.perf_counter()
        batch = st.Batch(plans)
        t1 = time.perf_counter()
        statuses, _ = batch.factorize([r.matrix["values"] for r in reqs], stream=stream, raise_on_error=False)
        window = batch.kernel_window(self._base)
        t2 = time.perf_counter()
        lds = batch.logdets(stream=stream)
        # all first solves of the job in one batched forward + backward sweep
        # (requests with more than MAX_RHS right-hand sides are solved on their own)
        rhs = [r.rhs if statuses[i] == 0 and r.rhs.shape[1] <= MAX_RHS else None for i, r in enumerate(reqs)]
        xs, rel, _, bst = batch.solve(rhs, stream=stream, raise_on_error=False)
        t3 = time.perf_counter()
        members = {}
        solved = 0
        for i, r in enumerate(reqs):
            r.batch_size = len(reqs)
            r.status = int(statuses[i])
            if r.status == 0:
                r.logdet = float(lds[i])
                if rhs[i] is None:
                    self._solve_single(r, batch.factor(i), stream)
                elif bst in (0, 6):  # OK, or NOT_CONVERGED (judged per request)
                    r.x, r.relres = xs[i], float(rel[i])
                else:
                    r.status, r.relres = int(bst), float("inf")
                if r.status == 0 and r.relres <= self.opts["refine_tol"]:
                    solved += r.rhs.shape[1]
            members[r.id] = i
        ev1 = self._event(stream)
        now = time.perf_counter()
        with self.lock:
            self.jobs.append(("factor", [r.id for r in reqs], ev0, ev1))
            self.kernels.append(window)
            key = self._next_key
            self._next_key += 1
            self.resident[key] = _Resident(batch, members, nbytes)
            for rid in members:
                self.where[rid] = key
            self.inflight_bytes -= nbytes
            self.resident_bytes += nbytes
            self.stats["batches"] += 1
            self.stats["factorized"] += len(reqs)
            self.stats["solved_columns"] += solved
            self.times["batch_create"] += t1 - t0
            self.times["factorize"] += t2 - t1
            self.times["logdet_solve"] += t3 - t2
            self.free_streams.append(si)
        for r in reqs:
            r.t_done = now
        return reqs

    def _job_resolve(self, res, group, si):
        """group: list of (request, member index); one batched solve over the
        targeted members of one resident batch."""
        stream = self.streams[si]
        ev0 = self._event(stream)
        t0 = time.perf_counter()
        rhs = [None] * len(res.members)
        for r, i in group:
            if r.rhs.shape[1] <= MAX_RHS:
                rhs[i] = r.rhs
        xs, rel, _, bst = res.batch.solve(rhs, stream=stream, raise_on_error=False)
        for r, i in group:
            if rhs[i] is None:  # more right-hand sides than one batched call takes
                r.status = 0
                self._solve_single(r, res.batch.factor(i), stream)
        ev1 = self._event(stream)
        now = time.perf_counter()
        solved = 0
        for r, i in group:
            if rhs[i] is None:
                if r.status == 0 and r.relres <= self.opts["refine_tol"]:
                    solved += r.rhs.shape[1]
            elif bst in (0, 6):
                r.status, r.x, r.relres = 0, xs[i], float(rel[i])
                if r.relres <= self.opts["refine_tol"]:
                    solved += r.rhs.shape[1]
            else:
                r.status, r.relres = int(bst), float("inf")
            r.t_done = now
        with self.lock:
            self.jobs.append(("resolve", [r.id for r, _ in group], ev0, ev1))
            res.busy -= 1
            self.stats["solved_columns"] += solved
            self.stats["resolve_jobs"] += 1
            self.times["resolve"] += now - t0
            self.free_streams.append(si)
        return [r for r, _ in group]

    def _solve_single(self, req, factor, stream):
        try:
            req.x, req.relres = factor.solve(req.rhs, stream=stream, relres=True)
        except st.StilesError as e:
            req.status = e.status
            req.relres = float("inf")

    def _take_stream(self):
        with self.lock:
            return self.free_streams.pop() if self.free_streams else None

    # -- the loop --------------------------------------------------------------
    def run(self, requests, arrivals, stream=None, realtime=True):
        """Serve ``requests`` (Request objects) arriving at ``arrivals`` [s]
        after the start.  Returns the list of completed requests.  ``stream``
        is accepted for compatibility; every GPU job runs on a worker stream."""
        self.jobs, self.kernels = [], []
        self._base = self._event(self._torch.cuda.current_stream())
        t0 = time.perf_counter()
        pending_an = collections.deque()   # (request, future of its plan)
        ready = collections.deque()        # (request, plan or None) waiting for the GPU
        resolves = collections.deque()
        running = set()                    # futures of GPU jobs
        done = []
        order = sorted(range(len(requests)), key=lambda i: arrivals[i])
        nxt = 0
        by_id = {r.id: r for r in requests}
        while len(done) < len(requests):
            now = time.perf_counter() - t0
            # admit everything that has arrived
            while nxt < len(order) and (not realtime or arrivals[order[nxt]] <= now):
                r = requests[order[nxt]]
                r.t_arrival = t0 + arrivals[order[nxt]]
                if r.kind == "resolve":
                    resolves.append(r)
                else:
                    pending_an.append((r, self.pool.submit(self._plan_for, r)))
                nxt += 1
            while pending_an and pending_an[0][1].done():
                r, fut = pending_an.popleft()
                ready.append((r, fut.result()))
            # collect finished jobs
            progressed = False
            for fut in [f for f in running if f.done()]:
                running.discard(fut)
                done.extend(fut.result())
                progressed = True
            # re-solves: group the ones whose factor is resident and idle, per batch
            if resolves:
                groups, keep = {}, collections.deque()
                with self.lock:
                    while resolves:
                        r = resolves.popleft()
                        src = by_id[r.target]
                        key = self.where.get(r.target)
                        if key is None:
                            if src.t_done is None:      # the factor is still being built
                                keep.append(r)
                                continue
                            r.refactorized = True       # evicted: refactorize
                            self.stats["resolve_misses"] += 1
                            r.matrix, r.key = src.matrix, src.key
                            ready.append((r, None))
                            continue
                        res = self.resident[key]
                        i = res.members[r.target]
                        grp = groups.setdefault(key, [])
                        if res.busy or any(j == i for _, j in grp):
                            keep.append(r)              # one slot per member and call: retry later
                            continue
                        grp.append((r, i))
                    for key, grp in groups.items():
                        if not grp:
                            continue
                        if not self.free_streams:
                            keep.extend(r for r, _ in grp)
                            continue
                        res = self.resident[key]
                        self.resident.move_to_end(key)
                        res.busy += 1
                        for r, _ in grp:
                            r.logdet = by_id[r.target].logdet
                        si = self.free_streams.pop()
                        running.add(self.gpu_pool.submit(self._job_resolve, res, grp, si))
                        progressed = True
                resolves = keep
            # new factorizations: everything analysed so far, within the budget
            if ready and self.free_streams:
                take, plans, need, flops = [], [], 0.0, 0
                with self.lock:
                    room = self.hbm_budget - self.resident_bytes - self.inflight_bytes
                while ready and len(take) < self.max_batch:
                    r, p = ready[0]
                    if p is None:
                        p = self._plan_for(r)
                    b = self._bytes(p)
                    if take and need + b > max(room, 0.0) + self._evictable():
                        break
                    fl = p.info()["flops_total"]
                    if take and self.max_job_flops is not None and flops + fl > self.max_job_flops:
                        break
                    ready.popleft()
                    take.append(r)
                    plans.append(p)
                    need += b
                    flops += fl
                with self.lock:
                    self._evict_until(need)
                    fits = self.resident_bytes + self.inflight_bytes + need <= self.hbm_budget
                    si = None
                    if (fits or not running) and self.free_streams:  # an oversized job runs when alone
                        self.inflight_bytes += need
                        si = self.free_streams.pop()
                if si is not None:
                    running.add(self.gpu_pool.submit(self._job_factor, take, plans, need, si))
                    progressed = True
                else:
                    for r, p in reversed(list(zip(take, plans))):
                        ready.appendleft((r, p))
            if not progressed:
                if nxt < len(order) and realtime:
                    time.sleep(max(0.0, min(0.001, arrivals[order[nxt]] - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
        self.wall = time.perf_counter() - t0
        return done

    def intervals(self):
        """GPU jobs on one device clock: (kind, start ms, end ms, request ids), start
        order; ms from the start of the last run."""
        self._torch.cuda.synchronize()
        out = [(k, self._base.elapsed_time(e0), self._base.elapsed_time(e1), ids) for k, ids, e0, e1 in self.jobs]
        return sorted(out, key=lambda j: j[1])

    def overlap(self, kernels=False):
        """(ms during which at least two GPU jobs were in flight, ms during which at
        least one was, largest number in flight at once); kernels=True: the same for
        the factor jobs' persistent kernels (work running on the device at once)."""
        pts = []
        spans = self.kernels if kernels else [(a, b) for _, a, b, _ in self.intervals()]
        for a, b in spans:
            pts += [(a, 1), (b, -1)]
        pts.sort()
        depth, last, both, busy, peak = 0, 0.0, 0.0, 0.0, 0
        for t, d in pts:
            if depth >= 2:
                both += t - last
            if depth >= 1:
                busy += t - last
            depth += d
            peak = max(peak, depth)
            last = t
        return both, busy, peak

    def _evictable(self):
        with self.lock:
            return sum(res.nbytes for res in self.resident.values() if not res.busy)

    def close(self):
        self.gpu_pool.shutdown(wait=True)
        with self.lock:
            for res in self.resident.values():
                res.batch.close()
            self.resident.clear()
        self.pool.shutdown(wait=True)
