"""Thin Python binding of libstiles.so (argument marshalling only).

Every computation runs inside the C ABI declared in ``include/stiles.h``;
this module only converts numpy arrays / torch tensors to pointers and
status codes to exceptions.  There is no fallback: if the shared library is
missing, every call raises.

Host arrays are numpy arrays; device arrays are torch CUDA tensors (torch is
used only for device memory and streams).  Streams are passed as the integer
``torch.cuda.Stream.cuda_stream`` handle (None = the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

__all__ = ["Plan", "Factor", "Batch", "autotune", "StilesError", "lib", "probe_fp64_peak", "kernel_launches", "ORDER_NONE", "ORDER_RCM", "ORDER_AUTO", "ORDER_ND",
           "PREC_F64", "PREC_BF16", "PREC_F16", "PREC_SLICED", "LIB_PATH"]

ORDER_NONE, ORDER_RCM, ORDER_AUTO, ORDER_ND = 0, 1, 2, 3
PREC_F64, PREC_BF16, PREC_F16, PREC_SLICED = 0, 1, 2, 3
STATUS = {0: "OK", 1: "INVALID", 2: "NOT_SPD", 3: "NOMEM", 4: "CUDA", 5: "TIMEOUT", 6: "NOT_CONVERGED",
          7: "UNSUPPORTED"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstiles.so")


class Opts(ctypes.Structure):
    _fields_ = [("tile", c_int32), ("ordering", c_int32), ("precision", c_int32), ("block", c_int32),
                ("tree_chunk", c_int32), ("tree_fanin", c_int32), ("max_refine", c_int32),
                ("ctas_per_sm", c_int32), ("refine_tol", c_double), ("spin_limit", c_int64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(k, c_int64) for k in ("n", "n_arrow", "nnz", "tile", "nt", "nnzt", "block", "nsub", "ntasks",
                                       "npairs", "nscratch", "flops_potrf", "flops_syrk", "flops_gemm",
                                       "flops_trsm", "flops_total", "factor_bytes")] + [
        ("ordering_used", c_int32), ("chain_split", c_int32)]


_LIB = None


def lib():
    """Load libstiles.so (once) and declare its prototypes."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built (python -m paper_2501_02483_b300.build)")
        L = ctypes.CDLL(LIB_PATH)
        P = c_void_p
        L.stiles_default_opts.argtypes = [POINTER(Opts)]
        L.stiles_default_opts.restype = None
        L.stiles_analyze.argtypes = [c_int64, P, P, c_int64, POINTER(Opts), POINTER(c_void_p)]
        L.stiles_plan_get_info.argtypes = [P, POINTER(PlanInfo)]
        L.stiles_plan_perm.argtypes = [P, P]
        L.stiles_plan_tilemap.argtypes = [P, P, P]
        L.stiles_factorize.argtypes = [P, P, P, POINTER(c_void_p), POINTER(c_int64)]
        L.stiles_factorize_solve.argtypes = [P, P, P, P, c_int32, c_int64, P, POINTER(c_void_p), POINTER(c_int64)]
        L.stiles_factorize_async.argtypes = [P, P, P, POINTER(c_void_p)]
        L.stiles_factor_wait.argtypes = [P, POINTER(c_int64)]
        L.stiles_logdet.argtypes = [P, POINTER(c_double)]
        L.stiles_solve.argtypes = [P, P, P, c_int64, c_int64, P, POINTER(c_double)]
        L.stiles_factor_tiles.argtypes = [P, P, P]
        L.stiles_plan_destroy.argtypes = [P]
        L.stiles_plan_destroy.restype = None
        L.stiles_factor_destroy.argtypes = [P]
        L.stiles_factor_destroy.restype = None
        L.stiles_strerror.argtypes = [c_int32]
        L.stiles_strerror.restype = c_char_p
        L.stiles_last_error.argtypes = []
        L.stiles_last_error.restype = c_char_p
        L.stiles_probe_fp64_peak.argtypes = [POINTER(c_double)]
        L.stiles_marginal_variances.argtypes = [P, P, P]
        L.stiles_selected_inverse_tiles.argtypes = [P, P, P]
        L.stiles_factor_timing.argtypes = [P, POINTER(c_double), POINTER(c_double)]
        L.stiles_factor_set_trace.argtypes = [P, c_int32]
        L.stiles_factor_get_trace.argtypes = [P, c_int32, P, POINTER(c_int64)]
        L.stiles_plan_tasks.argtypes = [P, c_int32, P, POINTER(c_int64)]
        L.stiles_factor_refine_iters.argtypes = [P]
        L.stiles_factor_cg_iters.argtypes = [P]
        L.stiles_factor_refine_iters.restype = c_int32
        L.stiles_batch_create.argtypes = [P, c_int32, POINTER(c_void_p)]
        L.stiles_batch_factorize.argtypes = [P, P, P, P, P]
        L.stiles_batch_factor.argtypes = [P, c_int32, POINTER(c_void_p)]
        L.stiles_batch_logdet.argtypes = [P, P, P]
        L.stiles_batch_solve.argtypes = [P, P, P, P, P, P, P]
        L.stiles_batch_timing.argtypes = [P, POINTER(c_double)]
        L.stiles_batch_kernel_window.argtypes = [P, P, POINTER(c_double), POINTER(c_double)]
        L.stiles_batch_kernel_window.restype = c_int32
        L.stiles_batch_destroy.argtypes = [P]
        L.stiles_batch_destroy.restype = None
        L.stiles_autotune.argtypes = [c_int64, P, P, c_int64, POINTER(Opts), P, c_int32, P, P, POINTER(c_int32), P]
        L.stiles_kernel_launches.argtypes = []
        L.stiles_kernel_launches.restype = c_int64
        for name in ("stiles_analyze", "stiles_plan_get_info", "stiles_plan_perm", "stiles_plan_tilemap",
                     "stiles_factorize", "stiles_factorize_solve", "stiles_factorize_async", "stiles_factor_wait", "stiles_logdet",
                     "stiles_solve", "stiles_factor_tiles", "stiles_probe_fp64_peak", "stiles_factor_timing",
                     "stiles_factor_set_trace", "stiles_factor_get_trace", "stiles_plan_tasks",
                     "stiles_batch_create", "stiles_batch_factorize", "stiles_batch_factor", "stiles_batch_logdet",
                     "stiles_autotune"):
            getattr(L, name).restype = c_int32
        _LIB = L
    return _LIB


class StilesError(RuntimeError):
    def __init__(self, status, detail, info=0):
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.info = info
        super().__init__(f"stiles {self.name}: {detail}")


def _check(status, info=0):
    if status != 0:
        L = lib()
        raise StilesError(status, L.stiles_last_error().decode() or L.stiles_strerror(status).decode(), info)


def _ptr(x):
    """Address of a numpy array or torch tensor (contiguous), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"expected numpy array or torch tensor, got {type(x)}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def default_opts():
    o = Opts()
    lib().stiles_default_opts(ctypes.byref(o))
    return o


class Plan:
    """Symbolic analysis of one pattern (stiles_analyze)."""

    def __init__(self, n, colptr, rowidx, n_arrow=0, tile=32, ordering=ORDER_AUTO, precision=PREC_F64, block=0,
                 tree_chunk=0, tree_fanin=0, spin_limit=0, refine_tol=0.0, max_refine=0, ctas_per_sm=0):
        L = lib()
        o = default_opts()
        o.tile, o.ordering, o.precision, o.block = tile, ordering, precision, block
        if tree_chunk:
            o.tree_chunk = tree_chunk
        if tree_fanin:
            o.tree_fanin = tree_fanin
        if spin_limit:
            o.spin_limit = spin_limit
        if refine_tol:
            o.refine_tol = refine_tol
        if max_refine:
            o.max_refine = max_refine
        o.ctas_per_sm = ctas_per_sm
        self._colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self._rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
        h = c_void_p()
        _check(L.stiles_analyze(int(n), _ptr(self._colptr), _ptr(self._rowidx), int(n_arrow), ctypes.byref(o),
                                ctypes.byref(h)))
        self._h = h
        self.n = int(n)

    @classmethod
    def from_matrix(cls, m, **kw):
        return cls(m["n"], m["colptr"], m["rowidx"], m["n_arrow"], **kw)

    @property
    def handle(self):
        return self._h

    def info(self):
        i = PlanInfo()
        _check(lib().stiles_plan_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in PlanInfo._fields_}

    def perm(self):
        out = np.empty(self.n, dtype=np.int64)
        _check(lib().stiles_plan_perm(self._h, _ptr(out)))
        return out

    def tilemap(self):
        inf = self.info()
        tc = np.empty(inf["nt"] + 1, dtype=np.int64)
        tr = np.empty(inf["nnzt"], dtype=np.int32)
        _check(lib().stiles_plan_tilemap(self._h, _ptr(tc), _ptr(tr)))
        return tc, tr

    def tasks(self, which=0):
        """Device task list (ticket order): int32 (ntasks, 16) for the factorization, (ntasks, 8)
        for a sweep (which 1, 2); the selected inverse's tasks (which 3: (ntasks, 8)), products
        (which 4: (n, 2)), loads of finished terms (which 5: (n, 3)) and X products (which 6: (n, 1));
        the sweeps' operand pairs (which 8 forward, 9 backward: (n, 2)) and partial lists (10, 11: (n, 1));
        the sweeps' release lists of a batched solve (12-14 forward, 15-17 backward: producer
        counts, reader offsets, readers; (n, 1) each)."""
        n = c_int64(0)
        _check(lib().stiles_plan_tasks(self._h, which, None, ctypes.byref(n)))
        width = {0: 16, 1: 8, 2: 8, 3: 8, 4: 2, 5: 3, 6: 1, 7: 16, 8: 2, 9: 2, 10: 1, 11: 1}.get(which, 1)
        out = np.empty((n.value, width), dtype=np.int32)
        _check(lib().stiles_plan_tasks(self._h, which, _ptr(out), ctypes.byref(n)))
        return out

    def close(self):
        if self._h:
            lib().stiles_plan_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Factor:
    """A numeric factorization of one plan (stiles_factorize & friends)."""

    def __init__(self, plan):
        self.plan = plan
        self._h = c_void_p()

    def factorize(self, values, stream=None):
        """values: host numpy or device torch float64 array of nnz entries."""
        info = c_int64(0)
        st = lib().stiles_factorize(self.plan.handle, _ptr(values), _stream(stream), ctypes.byref(self._h),
                                    ctypes.byref(info))
        _check(st, info.value)
        return self

    def factorize_solve(self, values, b, x=None, stream=None):
        """Factorize and solve A X = B in one pass (FP64 plans; the forward sweep runs inside
        the factorization launch).  values: as factorize; b: device torch (n,) or (n, nrhs)
        column-major, nrhs <= min(B, 16).  Returns x (device, b's shape)."""
        n = self.plan.n
        b2 = b.reshape(n, -1) if b.dim() == 1 else b.t().contiguous().t()
        nrhs = b2.shape[1]
        out = b2.t().contiguous().t().clone() if x is None else x
        info = c_int64(0)
        st = lib().stiles_factorize_solve(self.plan.handle, _ptr(values), _ptr(b2), _ptr(out), int(nrhs), int(n),
                                          _stream(stream), ctypes.byref(self._h), ctypes.byref(info))
        _check(st, info.value)
        return out.reshape(-1) if b.dim() == 1 else out

    def factorize_async(self, values, stream=None):
        _check(lib().stiles_factorize_async(self.plan.handle, _ptr(values), _stream(stream), ctypes.byref(self._h)))
        return self

    def wait(self):
        info = c_int64(0)
        st = lib().stiles_factor_wait(self._h, ctypes.byref(info))
        _check(st, info.value)
        return self

    def logdet(self):
        out = c_double(0.0)
        _check(lib().stiles_logdet(self._h, ctypes.byref(out)))
        return out.value

    def solve(self, b, x=None, stream=None, relres=False):
        """Solve A X = B; b is (n,) or (n, nrhs) Fortran-ordered, host numpy or device torch."""
        n = self.plan.n
        if isinstance(b, np.ndarray):
            b2 = np.asfortranarray(b.reshape(n, -1), dtype=np.float64)
            out = np.empty_like(b2, order="F") if x is None else x
            nrhs = b2.shape[1]
        else:
            b2 = b.reshape(n, -1) if b.dim() == 1 else b.t().contiguous().t()
            nrhs = b2.shape[1] if b2.dim() == 2 else 1
            out = b2.t().contiguous().t().clone() if x is None else x
        rr = c_double(0.0)
        _check(lib().stiles_solve(self._h, _ptr(b2), _ptr(out), int(nrhs), int(n), _stream(stream),
                                  ctypes.byref(rr) if relres else None))
        if isinstance(b, np.ndarray) and b.ndim == 1:
            out = out[:, 0]
        elif not isinstance(b, np.ndarray) and b.dim() == 1:
            out = out.reshape(-1)
        return (out, rr.value) if relres else out

    def timing(self):
        """(ms of the whole last factorize call on the device, ms of the persistent kernel)."""
        a, b = c_double(0.0), c_double(0.0)
        _check(lib().stiles_factor_timing(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def refine_iters(self):
        """Refinement steps of the last solve (0 for FP64 factors)."""
        return int(lib().stiles_factor_refine_iters(self._h))

    def cg_iters(self):
        """Of those, preconditioned conjugate-gradient iterations (refinement stalled)."""
        return int(lib().stiles_factor_cg_iters(self._h))

    def set_trace(self, enable=True):
        """Stamp every device task with the global timer (needs a factorization first)."""
        _check(lib().stiles_factor_set_trace(self._h, 1 if enable else 0))

    def trace(self, which=0):
        """Stamps of the last launch: int64 (ntasks, 4) = start, deps ready, done [ns], SM."""
        n = c_int64(0)
        _check(lib().stiles_factor_get_trace(self._h, which, None, ctypes.byref(n)))
        out = np.empty((n.value, 4), dtype=np.int64)
        _check(lib().stiles_factor_get_trace(self._h, which, _ptr(out), ctypes.byref(n)))
        return out

    def marginal_variances(self, out=None, stream=None):
        """diag(A^{-1}) in the original order (FP64 factors): host numpy unless ``out`` is given."""
        if out is None:
            out = np.empty(self.plan.n, dtype=np.float64)
        _check(lib().stiles_marginal_variances(self._h, _ptr(out), _stream(stream)))
        return out

    def selected_inverse_tiles(self, out=None, stream=None):
        """T x T tiles of Sigma = (P A P^T)^{-1} on L's tile map, tile-CSC order."""
        inf = self.plan.info()
        T = inf["tile"]
        if out is None:
            out = np.empty((inf["nnzt"], T, T), dtype=np.float64)
        _check(lib().stiles_selected_inverse_tiles(self._h, _ptr(out), _stream(stream)))
        return out

    def tiles(self, out=None, stream=None):
        """T x T column-major tiles of L in tile-CSC order (host numpy unless ``out`` is given)."""
        inf = self.plan.info()
        T = inf["tile"]
        if out is None:
            out = np.empty((inf["nnzt"], T, T), dtype=np.float64)
        _check(lib().stiles_factor_tiles(self._h, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if self._h:
            lib().stiles_factor_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _View(Factor):
    """A factor borrowed from a Batch (no destroy: the batch owns it)."""

    def __init__(self, plan, handle, batch):
        self.plan = plan
        self._h = handle
        self._batch = batch

    def close(self):
        self._h = c_void_p()


class Batch:
    """Many plans factorized in one persistent launch (stiles_batch_*)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = c_void_p()
        _check(lib().stiles_batch_create(arr, len(self.plans), ctypes.byref(h)))
        self._h = h

    def factorize(self, values, stream=None, raise_on_error=True):
        """values: list of host numpy / device torch arrays; returns (statuses, infos)."""
        self._keep = list(values)
        arr = (c_void_p * len(values))(*[_ptr(v) for v in values])
        statuses = np.zeros(len(values), dtype=np.int32)
        infos = np.zeros(len(values), dtype=np.int64)
        st = lib().stiles_batch_factorize(self._h, arr, _stream(stream), _ptr(statuses), _ptr(infos))
        if raise_on_error:
            _check(st)
        return statuses, infos

    def factor(self, i):
        h = c_void_p()
        _check(lib().stiles_batch_factor(self._h, i, ctypes.byref(h)))
        return _View(self.plans[i], h, self)

    def timing(self):
        """ms of the persistent factorization kernel of the last factorize."""
        ms = c_double(0.0)
        _check(lib().stiles_batch_timing(self._h, ctypes.byref(ms)))
        return ms.value

    def kernel_window(self, base_event):
        """(start, end) of the last factorize's persistent kernel in ms after ``base_event``
        (a timing torch.cuda.Event recorded earlier on this device)."""
        a, b = c_double(0.0), c_double(0.0)
        _check(lib().stiles_batch_kernel_window(self._h, c_void_p(base_event.cuda_event), ctypes.byref(a),
                                                ctypes.byref(b)))
        return a.value, b.value

    def logdets(self, stream=None):
        out = np.zeros(len(self.plans), dtype=np.float64)
        _check(lib().stiles_batch_logdet(self._h, _ptr(out), _stream(stream)))
        return out

    def solve(self, rhs, stream=None, relres=True, raise_on_error=True):
        """rhs: list (one per matrix) of n_i x k_i arrays (k_i <= 16; host numpy or device
        torch, column-major/Fortran order or 1-D), or None to skip a matrix.  Returns
        (xs, relres, iters, status); xs[i] matches rhs[i]'s kind (None where skipped)."""
        cnt = len(self.plans)
        if len(rhs) != cnt:
            raise ValueError("one right-hand side per matrix")
        bs, xs, ks = [], [], np.zeros(cnt, dtype=np.int32)
        for i, b in enumerate(rhs):
            if b is None:
                bs.append(None)
                xs.append(None)
                continue
            n = self.plans[i].n
            if isinstance(b, np.ndarray):
                bn = np.asfortranarray(b.reshape(n, -1), dtype=np.float64)
                xs.append(np.empty_like(bn, order="F"))
            else:  # torch tensor (device or host)
                bn = b.reshape(n, -1).t().contiguous().t()
                xs.append(bn.clone())
            ks[i] = bn.shape[1]
            bs.append(bn)
        barr = (c_void_p * cnt)(*[None if b is None else _ptr(b) for b in bs])
        xarr = (c_void_p * cnt)(*[None if x is None else _ptr(x) for x in xs])
        rel = np.zeros(cnt, dtype=np.float64)
        its = np.zeros(cnt, dtype=np.int32)
        st = lib().stiles_batch_solve(self._h, barr, xarr, _ptr(ks), _stream(stream),
                                      _ptr(rel) if relres else None, _ptr(its))
        if raise_on_error:
            _check(st)
        out = []
        for i, x in enumerate(xs):
            if x is not None and np.ndim(rhs[i]) == 1:
                x = x.reshape(-1)
            out.append(x)
        return out, rel, its, int(st)

    def close(self):
        if self._h:
            lib().stiles_batch_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(m, tiles, values=None, stream=None, **kw):
    """Fastest tile size among ``tiles`` for matrix ``m`` (stiles_autotune); returns (tile, ms list)."""
    o = default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    colptr = np.ascontiguousarray(m["colptr"], dtype=np.int64)
    rowidx = np.ascontiguousarray(m["rowidx"], dtype=np.int32)
    cand = np.ascontiguousarray(tiles, dtype=np.int32)
    ms = np.zeros(cand.size, dtype=np.float64)
    best = c_int32(0)
    vals = m["values"] if values is None else values
    _check(lib().stiles_autotune(int(m["n"]), _ptr(colptr), _ptr(rowidx), int(m["n_arrow"]), ctypes.byref(o),
                                 _ptr(cand), int(cand.size), _ptr(vals), _stream(stream), ctypes.byref(best),
                                 _ptr(ms)))
    return int(best.value), ms.tolist()


def kernel_launches():
    """CUDA kernels launched by libstiles.so so far in this process."""
    return int(lib().stiles_kernel_launches())


def probe_fp64_peak():
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    out = c_double(0.0)
    _check(lib().stiles_probe_fp64_peak(ctypes.byref(out)))
    return out.value
