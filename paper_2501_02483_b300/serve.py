"""Continuous-batching request loop over the C ABI.

Requests are factorize + logdet + solve of an arrowhead SPD matrix, or a
re-solve against a factor that is still resident.  The loop:

* admits requests as they arrive: new matrices go through the analysis pool
  (host threads; the C analysis releases the GIL) and then wait for the GPU;
* every time the GPU side is free it takes *all* analysed requests that fit
  the HBM budget and factorizes them in one batched persistent launch
  (stiles_batch_*), then computes their log-determinants in one launch and
  their solves in one batched forward/backward sweep (FP64 refinement for
  BF16/FP16 factors); requests that arrive meanwhile join the next launch,
  so their work overlaps the running one;
* keeps finished factors resident in an LRU cache bounded by the HBM budget;
  re-solve requests for a resident factor skip the factorization, a re-solve
  whose factor was evicted is refactorized (and counted as a miss).

Plans are cached per pattern (the same structure with new values -- e.g. a
hyperparameter sweep -- reuses the symbolic analysis, Section III.A).

All numerical work runs in libstiles.so; this module only schedules it.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np

from . import stiles as st

__all__ = ["Request", "Server"]


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


class Server:
    def __init__(self, precision=st.PREC_BF16, tile=64, ordering=st.ORDER_NONE, hbm_budget=150e9, max_batch=64,
                 analyze_threads=8, refine_tol=1e-10):
        self.opts = dict(tile=tile, ordering=ordering, precision=precision, refine_tol=refine_tol)
        self.hbm_budget = float(hbm_budget)
        self.max_batch = max_batch
        self.pool = cf.ThreadPoolExecutor(max_workers=analyze_threads)
        self.plans = {}            # pattern key -> Plan
        self.plan_lock = threading.Lock()
        self.resident = collections.OrderedDict()  # request id of first member -> _Resident (LRU)
        self.where = {}            # request id -> resident key holding its factor
        self.resident_bytes = 0.0
        self.stats = collections.Counter()

    # -- analysis (host threads) -------------------------------------------
    def _plan_for(self, req):
        with self.plan_lock:
            p = self.plans.get(req.key)
        if p is not None:
            return p
        p = st.Plan.from_matrix(req.matrix, **self.opts)
        with self.plan_lock:
            self.plans.setdefault(req.key, p)
            return self.plans[req.key]

    @staticmethod
    def _bytes(plan):
        inf = plan.info()
        # tiles (FP32 + 16-bit copy, or FP64) + values + scatter map + flags, per matrix
        return float(inf["factor_bytes"]) + 24.0 * inf["nnz"] + 4.0 * inf["nsub"]

    # -- residency -----------------------------------------------------------
    def _evict_until(self, need):
        while self.resident and self.resident_bytes + need > self.hbm_budget:
            key, res = self.resident.popitem(last=False)
            for rid in res.members:
                self.where.pop(rid, None)
            res.batch.close()
            self.resident_bytes -= res.nbytes
            self.stats["evicted_batches"] += 1

    def _factor_of(self, rid):
        key = self.where.get(rid)
        if key is None:
            return None
        res = self.resident[key]
        self.resident.move_to_end(key)
        return res.batch.factor(res.members[rid])

    # -- GPU side ----------------------------------------------------------------
    def _run_batch(self, reqs, plans, stream):
        nbytes = sum(self._bytes(p) for p in plans)
        self._evict_until(nbytes)
        batch = st.Batch(plans)
        statuses, _ = batch.factorize([r.matrix["values"] for r in reqs], stream=stream, raise_on_error=False)
        lds = batch.logdets(stream=stream)
        # all first solves of the launch in one batched forward + backward sweep
        # (requests with more than 16 right-hand sides are solved on their own)
        rhs = [r.rhs if statuses[i] == 0 and r.rhs.shape[1] <= 16 else None for i, r in enumerate(reqs)]
        xs, rel, _, bst = batch.solve(rhs, stream=stream, raise_on_error=False)
        members = {}
        for i, r in enumerate(reqs):
            r.batch_size = len(reqs)
            r.status = int(statuses[i])
            if r.status == 0:
                r.logdet = float(lds[i])
                if rhs[i] is None:
                    self._solve(r, batch.factor(i), stream)
                elif bst in (0, 6):  # OK, or NOT_CONVERGED (judged per request below)
                    r.x, r.relres = xs[i], float(rel[i])
                    self.stats["solved_columns"] += r.rhs.shape[1] if r.relres <= self.opts["refine_tol"] else 0
                else:
                    r.status, r.relres = int(bst), float("inf")
            r.t_done = time.perf_counter()
            members[r.id] = i
        self.resident[reqs[0].id] = _Resident(batch, members, nbytes)
        for rid in members:
            self.where[rid] = reqs[0].id
        self.resident_bytes += nbytes
        self.stats["batches"] += 1
        self.stats["factorized"] += len(reqs)

    def _solve(self, req, factor, stream):
        try:
            req.x, req.relres = factor.solve(req.rhs, stream=stream, relres=True)
            self.stats["solved_columns"] += req.rhs.shape[1] if req.relres <= self.opts["refine_tol"] else 0
        except st.StilesError as e:
            req.status = e.status
            req.relres = float("inf")

    def run(self, requests, arrivals, stream=None, realtime=True):
        """Serve ``requests`` (Request objects) arriving at ``arrivals`` [s]
        after the start.  Returns the list of completed requests."""
        t0 = time.perf_counter()
        pending_an = collections.deque()   # (request, future of its plan)
        ready = collections.deque()        # (request, plan) analysed, waiting for the GPU
        resolves = collections.deque()
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
            progressed = False
            # re-solves against resident factors (or refactorize after eviction)
            while resolves:
                r = resolves.popleft()
                f = self._factor_of(r.target)
                src = by_id[r.target]
                if f is None:
                    if src.t_done is None:       # the factor is still being built: wait for it
                        resolves.appendleft(r)
                        break
                    r.refactorized = True
                    self.stats["resolve_misses"] += 1
                    r.matrix, r.key = src.matrix, src.key
                    ready.append((r, self._plan_for(r)))
                    continue
                r.logdet = src.logdet
                r.status = 0
                self._solve(r, f, stream)
                r.t_done = time.perf_counter()
                done.append(r)
                progressed = True
            # one batched launch over everything analysed so far (continuous batching)
            if ready:
                take, plans, budget = [], [], 0.0
                while ready and len(take) < self.max_batch:
                    r, p = ready[0]
                    need = self._bytes(p)
                    if take and budget + need > self.hbm_budget:
                        break
                    ready.popleft()
                    take.append(r)
                    plans.append(p)
                    budget += need
                self._run_batch(take, plans, stream)
                done.extend(take)
                progressed = True
            if not progressed:
                if nxt < len(order) and realtime:
                    time.sleep(max(0.0, min(0.002, arrivals[order[nxt]] - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0005)
        self.wall = time.perf_counter() - t0
        return done

    def close(self):
        for res in self.resident.values():
            res.batch.close()
        self.resident.clear()
        self.pool.shutdown(wait=True)
