"""SRCD for NMF with KL divergence on one GB300 GPU.

A thin Python binding over the C ABI of ``libnmfkl.so`` (``include/nmfkl.h``).
The binding only marshals arguments: every step of a sweep runs in the
library's CUDA kernels. PyTorch, when used, only provides device memory
(``tensor.data_ptr()``) and streams.

    import paper_1604_04026_gb300 as nk
    V = nk.synth.docs(30000, 100000, 50)
    model = nk.NMFKL(V.n, V.m, r=50)
    model.set_data(V)
    model.init()                      # Uniform[0,1) from the seed
    trace, done = model.fit(20)       # Algorithm 1, KL after each sweep
    W, F = model.get_W(), model.get_F()
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native, synth
from ._native import Counters, Params

__all__ = ["NMFKL", "NMFKLError", "Params", "Server", "default_params", "synth"]


class NMFKLError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.status_name = _native.STATUS_NAMES.get(status, str(status))
        super().__init__("%s: %s" % (self.status_name, message))


def default_params(r: int, **kw) -> Params:
    p = Params()
    _native.load().nmfkl_default_params(ctypes.byref(p), r)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown parameter %r" % k)
        setattr(p, k, v)
    return p


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, mem_kind, keepalive) for a numpy array or a torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float32: "torch.float32", np.int32: "torch.int32", np.int64: "torch.int64"}[dtype]
        if str(x.dtype) != want:
            raise TypeError("expected %s, got %s" % (want, x.dtype))
        return x.data_ptr(), (1 if x.is_cuda else 0), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


class NMFKL:
    """One factorization problem V (n x m) ~= W^T F with W (r x n), F (r x m)."""

    def __init__(self, n: int, m: int, r: int | None = None, params: Params | None = None,
                 device: int = 0, stream: int | None = None, **kw):
        self._lib = _native.load()
        if params is None:
            if r is None:
                raise ValueError("give r or params")
            params = default_params(r, **kw)
        self.params = params
        self.device = int(device)
        self.n, self.m, self.r = int(n), int(m), int(params.r)
        h = ctypes.c_void_p()
        st = self._lib.nmfkl_create(ctypes.byref(params), self.n, self.m, device,
                                    ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != 0:
            raise NMFKLError(st, "nmfkl_create failed")
        self._h = h

    # -- plumbing
    def _check(self, st: int, what: str):
        if st != 0:
            msg = self._lib.nmfkl_last_error(self._h)
            raise NMFKLError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.nmfkl_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    # -- data and state
    def set_data(self, V=None, *, nnz=None, colptr=None, rowidx=None, val=None, rowptr=None,
                 colidx=None, rval=None):
        """V: a synth.CountMatrix (host), or the six arrays (numpy or torch CUDA tensors)."""
        if V is not None:
            colptr, rowidx, val = V.colptr, V.rowidx, V.val
            rowptr, colidx, rval = V.rowptr, V.colidx, V.rval
            nnz = V.nnz
        p = [_ptr(colptr, np.int64), _ptr(rowidx, np.int32), _ptr(val, np.float32),
             _ptr(rowptr, np.int64), _ptr(colidx, np.int32), _ptr(rval, np.float32)]
        kinds = {k for _, k, _ in p if _ is not None}
        if len(kinds) > 1:
            raise ValueError("mix of host and device arrays")
        kind = kinds.pop() if kinds else 0
        if nnz is None:
            nnz = int(rowidx.shape[0])
        self._check(self._lib.nmfkl_set_data(self._h, int(nnz), *[x[0] for x in p], kind), "set_data")

    def init(self, W0=None, F0=None):
        """Starting W (r x n) and F (r x m); None draws Uniform[0,1) from the seed."""
        pw, kw, a = _ptr(W0, np.float32)
        pf, kf, b = _ptr(F0, np.float32)
        if W0 is not None and F0 is not None and kw != kf:
            raise ValueError("W0 and F0 must both be host or both device")
        kind = kw if W0 is not None else kf
        self._check(self._lib.nmfkl_init(self._h, pw, pf, kind), "init")

    def sweep_F(self, sweep: int):
        self._check(self._lib.nmfkl_sweep_F(self._h, int(sweep)), "sweep_F")

    def sweep_W(self, sweep: int):
        self._check(self._lib.nmfkl_sweep_W(self._h, int(sweep)), "sweep_W")

    def sweep(self, sweep: int):
        self.sweep_F(sweep)
        self.sweep_W(sweep)

    def sweep_range(self, side: int, sweep: int, u0: int, u1: int) -> float:
        """One half over the units u0 <= u < u1 (side 0: columns of F, 1: rows of
        W); returns the range's Eq. 1 data term for side 1 (0.0 for side 0)."""
        dt = ctypes.c_double()
        self._check(self._lib.nmfkl_sweep_range(self._h, int(side), int(sweep), int(u0), int(u1), ctypes.byref(dt)),
                    "sweep_range")
        return dt.value

    def linear_term(self) -> float:
        """sum_k (sum_i W_ki)(sum_j F_kj): Eq. 1's term over all entries of W^T F."""
        out = ctypes.c_double()
        self._check(self._lib.nmfkl_linear_term(self._h, ctypes.byref(out)), "linear_term")
        return out.value

    def factor_unit_major(self, side: int):
        """The device copy of F (side 0) or W (side 1), unit-major (units x ld
        floats), as a CUDA tensor sharing the context's memory."""
        import torch
        ptr, units, ld = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32()
        self._check(self._lib.nmfkl_factor_unit_major(self._h, int(side), ctypes.byref(ptr), ctypes.byref(units),
                                                      ctypes.byref(ld)), "factor_unit_major")

        class _View:
            __cuda_array_interface__ = {"shape": (units.value, ld.value), "typestr": "<f4",
                                        "data": (ptr.value, False), "version": 3, "strides": None}
        return torch.as_tensor(_View(), device="cuda:%d" % self.device)

    def set_wait_limit(self, cycles: int):
        """Limit (SM clock cycles) of the bounded waits between cluster CTAs;
        0 restores the default. A wait that gives up makes the half raise
        ETIMEOUT."""
        self._check(self._lib.nmfkl_set_wait_limit(self._h, int(cycles)), "set_wait_limit")

    def objective(self):
        """(Eq. 1 value, Eq. 2 regularizer) in FP64."""
        kl, reg = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.nmfkl_objective(self._h, ctypes.byref(kl), ctypes.byref(reg)), "objective")
        return kl.value, reg.value

    def fit(self, max_sweeps: int, rel_tol: float = 0.0, sweep0: int = 0, raise_notconv: bool = False):
        """Algorithm 1; returns (KL after each sweep, sweeps done)."""
        trace = np.zeros(max(max_sweeps, 1), dtype=np.float64)
        done = ctypes.c_int32()
        st = self._lib.nmfkl_fit(self._h, sweep0, max_sweeps, rel_tol, trace.ctypes.data, ctypes.byref(done))
        if st != 0 and not (st == 7 and not raise_notconv):
            self._check(st, "fit")
        return trace[:done.value], done.value

    def step(self, sweep: int) -> float:
        """F half, W half and the objective (the whole hot path); returns Eq. 1."""
        kl = ctypes.c_double()
        self._check(self._lib.nmfkl_step(self._h, int(sweep), ctypes.byref(kl)), "step")
        return kl.value

    def foldin(self, V=None, *, colptr=None, rowidx=None, val=None, nnz=None, doc_ids=None, F0=None,
               rel_tol: float = 1e-5, max_sweeps: int = 100, launch_mode: int = 0, out=None):
        """F (r x m_new) for new documents under the current W (held fixed).

        V: a synth.CountMatrix with n rows (host), or colptr/rowidx/val as numpy
        arrays or CUDA tensors. Returns (F, sweeps per document, objective per
        document); with CUDA inputs the three results are CUDA tensors."""
        if V is not None:
            colptr, rowidx, val, nnz = V.colptr, V.rowidx, V.val, V.nnz
        p = [_ptr(colptr, np.int64), _ptr(rowidx, np.int32), _ptr(val, np.float32), _ptr(doc_ids, np.int64),
             _ptr(F0, np.float32)]
        kinds = {k for x, k, _ in p if x is not None}
        if len(kinds) > 1:
            raise ValueError("mix of host and device arrays")
        kind = kinds.pop() if kinds else 0
        m_new = int(colptr.shape[0]) - 1
        if nnz is None:
            nnz = int(rowidx.shape[0])
        if kind == 1:
            import torch
            dev = colptr.device
            F = out if out is not None else torch.empty((self.r, m_new), dtype=torch.float32, device=dev)
            sweeps = torch.empty(max(m_new, 1), dtype=torch.int32, device=dev)
            obj = torch.empty(max(m_new, 1), dtype=torch.float64, device=dev)
            pf, ps, po = F.data_ptr(), sweeps.data_ptr(), obj.data_ptr()
        else:
            F = out if out is not None else np.empty((self.r, m_new), dtype=np.float32)
            sweeps = np.zeros(max(m_new, 1), dtype=np.int32)
            obj = np.zeros(max(m_new, 1), dtype=np.float64)
            pf, ps, po = F.ctypes.data, sweeps.ctypes.data, obj.ctypes.data
        st = self._lib.nmfkl_foldin(self._h, m_new, int(nnz), p[0][0], p[1][0], p[2][0], p[3][0], p[4][0], pf,
                                    float(rel_tol), int(max_sweeps), ps, po, int(launch_mode), kind)
        self._check(st, "foldin")
        return F, sweeps[:m_new], obj[:m_new]

    def plan(self) -> list:
        """Launch plan: one dict per (half, length bucket)."""
        cap = 128
        arr = (_native.BucketInfo * cap)()
        nb = self._lib.nmfkl_plan_info(self._h, arr, cap)
        return [{"kernel": arr[i].kernel.decode(), "side": arr[i].side, "count": arr[i].count,
                 "nnz": arr[i].nnz, "max_len": arr[i].max_len, "grid": arr[i].grid,
                 "block": arr[i].block, "smem": arr[i].smem, "ran_last": bool(arr[i].ran_last),
                 "list_plan": bool(arr[i].list_plan)}
                for i in range(min(nb, cap))]

    def plan_choice(self) -> dict:
        """The launch-plan choices: list_threshold and short_kernel[side][class]."""
        pc = _native.PlanChoice()
        self._check(self._lib.nmfkl_get_plan_choice(self._h, ctypes.byref(pc)), "get_plan_choice")
        return {"list_threshold": pc.list_threshold,
                "short_kernel": [[int(pc.short_kernel[s][k]) for k in range(4)] for s in range(2)]}

    def set_plan_choice(self, list_threshold=None, short_kernel=None):
        cur = self.plan_choice()
        pc = _native.PlanChoice()
        pc.list_threshold = cur["list_threshold"] if list_threshold is None else float(list_threshold)
        sk = cur["short_kernel"] if short_kernel is None else short_kernel
        for s in range(2):
            for k in range(4):
                pc.short_kernel[s][k] = int(sk[s][k])
        self._check(self._lib.nmfkl_set_plan_choice(self._h, ctypes.byref(pc)), "set_plan_choice")

    def autotune(self, sweep: int = 0, reps: int = 1, cache_path: str | None = None) -> dict:
        """Times both kernels of every short length class of the list plan from
        the current state (restored afterwards) and applies the faster ones;
        cached per configuration in cache_path (or NMFKL_TUNE_CACHE)."""
        pc = _native.PlanChoice()
        ms = (ctypes.c_double * 16)()
        fc = ctypes.c_int32()
        path = cache_path.encode() if cache_path else None
        self._check(self._lib.nmfkl_autotune(self._h, int(sweep), int(reps), path, ctypes.byref(pc), ms,
                                             ctypes.byref(fc)), "autotune")
        return {"short_kernel": [[int(pc.short_kernel[s][k]) for k in range(4)] for s in range(2)],
                "ms": [[[ms[(s * 4 + k) * 2 + a] for a in range(2)] for k in range(4)] for s in range(2)],
                "from_cache": bool(fc.value)}

    def _get(self, fn, rows, cols, out):
        if out is None:
            out = np.empty((rows, cols), dtype=np.float32)
        p, kind, keep = _ptr(out, np.float32)
        if kind == 0 and not isinstance(out, np.ndarray):
            raise TypeError("host output must be a numpy array")
        self._check(fn(self._h, p, kind), "get")
        return out

    def get_W(self, out=None):
        """W (r x n); out may be a numpy array or a CUDA tensor."""
        return self._get(self._lib.nmfkl_get_W, self.r, self.n, out)

    def get_F(self, out=None):
        """F (r x m); out may be a numpy array or a CUDA tensor."""
        return self._get(self._lib.nmfkl_get_F, self.r, self.m, out)

    def get_state(self, next_sweep: int) -> bytes:
        """Checkpoint (W, F, next sweep index) as a self-describing blob."""
        n = int(self._lib.nmfkl_state_bytes(self._h))
        buf = ctypes.create_string_buffer(n)
        self._check(self._lib.nmfkl_get_state(self._h, int(next_sweep), buf, n), "get_state")
        return buf.raw

    def set_state(self, blob: bytes) -> int:
        """Restores a checkpoint of this shape and seed; returns its next sweep index."""
        nxt = ctypes.c_int64(0)
        self._check(self._lib.nmfkl_set_state(self._h, blob, len(blob), ctypes.byref(nxt)), "set_state")
        return int(nxt.value)

    def counters(self, reset: bool = False) -> dict:
        c = Counters()
        self._check(self._lib.nmfkl_get_counters(self._h, ctypes.byref(c), int(reset)), "counters")
        return {k: int(getattr(c, k)) for k, _ in Counters._fields_}

    def set_timing(self, enable: bool = True):
        self._check(self._lib.nmfkl_set_timing(self._h, int(enable)), "set_timing")

    def set_metrics(self, path=None):
        """Appends one JSON line per step to `path` (None stops): objective,
        device time, throughput, work per coordinate, zeros of W and F."""
        self._check(self._lib.nmfkl_set_metrics(self._h, path.encode() if path else None), "set_metrics")

    def kernel_times(self, reset: bool = False) -> dict:
        cap = 64
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        nf = self._lib.nmfkl_kernel_times(self._h, names, launches, ms, cap, int(reset))
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(nf, cap))}

    def debug_perm(self, sweep: int, side: int, cols_dev, out_dev):
        """Device orders: out_dev[c, :] = ids of unit cols_dev[c] (CUDA tensors)."""
        self._check(self._lib.nmfkl_debug_perm(self._h, sweep, side, int(cols_dev.numel()),
                                               cols_dev.data_ptr(), out_dev.data_ptr()), "debug_perm")


class Ticket:
    """A submitted serving request and the host arrays its results land in."""

    def __init__(self, ticket, kind, keep, F, W, sweeps, obj):
        self.id, self.kind, self._keep = ticket, kind, keep
        self.F, self.W, self.sweeps, self.obj = F, W, sweeps, obj
        self.status = None
        self.message = ""
        self.queued_ms = self.run_ms = None
        self.batch_requests = None

    def _set(self, res):
        self.status = _native.STATUS_NAMES.get(res.status, str(res.status))
        self.message = res.message.decode(errors="replace")
        self.queued_ms, self.run_ms, self.batch_requests = res.queued_ms, res.run_ms, res.batch_requests
        self._keep = None


class Server:
    """Serving loop around one resident model W (r x n): fold-in requests and
    small factorizations, admitted as slots and memory free up (nmfkl_server_*)."""

    def __init__(self, W, params: Params | None = None, r: int | None = None, device: int = 0, slots: int = 4,
                 mem_budget: int = 16 << 30, max_pending: int = 4096, max_batch_docs: int = 20000,
                 max_batch_nnz: int = 1 << 26, **kw):
        self._lib = _native.load()
        W = np.ascontiguousarray(W, dtype=np.float32)
        if params is None:
            params = default_params(r or W.shape[0], **kw)
        self.params, self.r, self.n = params, int(params.r), int(W.shape[1])
        cfg = _native.ServerCfg()
        self._lib.nmfkl_server_default_cfg(ctypes.byref(cfg))
        cfg.device, cfg.slots, cfg.mem_budget, cfg.max_pending = device, slots, mem_budget, max_pending
        cfg.max_batch_docs, cfg.max_batch_nnz = max_batch_docs, max_batch_nnz
        h = ctypes.c_void_p()
        st = self._lib.nmfkl_server_create(ctypes.byref(cfg), ctypes.byref(params), self.n, W.ctypes.data,
                                           ctypes.byref(h))
        if st != 0:
            raise NMFKLError(st, "nmfkl_server_create failed")
        self._h = h

    def _submit(self, kind, V, r, seed, rel_tol, max_sweeps):
        colptr = np.ascontiguousarray(V.colptr, dtype=np.int64)
        rowidx = np.ascontiguousarray(V.rowidx, dtype=np.int32)
        val = np.ascontiguousarray(V.val, dtype=np.float32)
        F = np.zeros((r, V.m), dtype=np.float32)
        W = np.zeros((r, V.n), dtype=np.float32) if kind == 1 else None
        sweeps = np.zeros(max(V.m, 1) if kind == 0 else 1, dtype=np.int32)
        obj = np.zeros(max(V.m, 1) if kind == 0 else 1, dtype=np.float64)
        q = _native.Request(kind=kind, n=V.n, m=V.m, nnz=int(V.nnz), colptr=colptr.ctypes.data,
                            rowidx=rowidx.ctypes.data, val=val.ctypes.data, r=r, seed=seed, rel_tol=rel_tol,
                            max_sweeps=max_sweeps, F_out=F.ctypes.data, W_out=W.ctypes.data if W is not None else None,
                            sweeps_out=sweeps.ctypes.data, obj_out=obj.ctypes.data)
        t = ctypes.c_uint64()
        st = self._lib.nmfkl_server_submit(self._h, ctypes.byref(q), ctypes.byref(t))
        if st != 0:
            raise NMFKLError(st, "submit")
        return Ticket(t.value, kind, (F, W, sweeps, obj), F, W, sweeps[:V.m] if kind == 0 else sweeps,
                      obj[:V.m] if kind == 0 else obj)

    def submit_foldin(self, V, rel_tol: float = 1e-5, max_sweeps: int = 100) -> Ticket:
        """F for the documents (columns) of V (n x m, the model's n) under W."""
        return self._submit(0, V, self.r, 0, rel_tol, max_sweeps)

    def submit_fit(self, V, r: int, seed: int = 0, rel_tol: float = 1e-4, max_sweeps: int = 50) -> Ticket:
        """A full factorization of V with r factors from a Uniform[0,1) start."""
        return self._submit(1, V, int(r), int(seed), rel_tol, max_sweeps)

    def poll(self, t: Ticket) -> bool:
        res = _native.Result()
        st = self._lib.nmfkl_server_poll(self._h, t.id, ctypes.byref(res))
        if st == 6:
            return False
        if st != 0:
            raise NMFKLError(st, "poll")
        t._set(res)
        return True

    def wait(self, t: Ticket) -> Ticket:
        res = _native.Result()
        st = self._lib.nmfkl_server_wait(self._h, t.id, ctypes.byref(res))
        if st != 0:
            raise NMFKLError(st, "wait")
        t._set(res)
        return t

    def cancel(self, t: Ticket) -> bool:
        """Withdraws a request that still waits: True if it was withdrawn (it
        is then collected by poll/wait with status ECANCELED), False if it is
        already running or done."""
        st = self._lib.nmfkl_server_cancel(self._h, t.id)
        if st == 6:
            return False
        if st != 0:
            raise NMFKLError(st, "cancel")
        return True

    def stats(self) -> dict:
        x = _native.ServerStats()
        self._lib.nmfkl_server_stats(self._h, ctypes.byref(x))
        return {k: int(getattr(x, k)) for k, _ in _native.ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.nmfkl_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
