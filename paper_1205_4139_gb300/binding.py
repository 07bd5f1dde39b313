"""ctypes binding of libcsfast.so (C ABI in include/csfast.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (torch supplies device memory and
the current stream); complex tensors use torch's interleaved (re, im) layout,
which is the library's.  The library is loaded on first use and a missing
library raises ``RuntimeError``; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libcsfast.so")

CS_WHT, CS_DFT = 0, 1
CS_FP64, CS_FP32 = 0, 1
PATHS = {"fast": 0, "conv": 1, "hybrid": 2}
KINDS = {"wht": CS_WHT, "dft": CS_DFT}
PRECS = {"fp64": CS_FP64, "fp32": CS_FP32}

# Every function include/csfast.h declares.
EXPORTS = ["cs_plan_create", "cs_plan_create_ex", "cs_plan_memory", "cs_plan_switch", "cs_plan_destroy", "cs_plan_info", "cs_plan_status", "cs_plan_kernel", "cs_correlate",
           "cs_correlate_fast", "cs_omp", "cs_omp_batched", "cs_omp_batched_tune", "cs_sp", "cs_cosamp", "cs_omp_noalloc", "cs_plan_tune",
           "cs_server_create", "cs_server_submit", "cs_server_poll", "cs_server_stats", "cs_server_destroy",
           "cs_admit_next", "cs_fma_probe", "cs_status_string", "cs_last_error"]


class CsError(RuntimeError):
    pass


class Halt(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("path", ctypes.c_int32), ("t_switch", ctypes.c_int32),
                ("max_iter", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("prec", ctypes.c_int32), ("algo", ctypes.c_int32), ("K", ctypes.c_int32),
                ("N", ctypes.c_int64), ("M", ctypes.c_int64), ("omega_host", ctypes.POINTER(ctypes.c_int32)),
                ("y_host", ctypes.c_void_p), ("halt", Halt)]


class Result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("device_error", ctypes.c_int32), ("pad", ctypes.c_int32), ("resnorm", ctypes.c_double),
                ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double), ("t_done_us", ctypes.c_double),
                ("footprint_bytes", ctypes.c_int64)]


ALGOS = {"omp": 0, "cosamp": 1, "sp": 2}


_lib = None


def load(path: str = LIB_PATH):
    """Load the library and declare the signatures (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pi32 = ctypes.POINTER(ctypes.c_int32)
    pi64 = ctypes.POINTER(ctypes.c_int64)
    L.cs_plan_create.argtypes = [i64, pi32, i64, i32, i32, vp, ctypes.POINTER(vp)]
    L.cs_plan_create_ex.argtypes = [i64, pi32, i64, i32, i32, ctypes.c_uint32, vp, ctypes.POINTER(vp)]
    L.cs_plan_memory.argtypes = [vp, pi64]
    L.cs_plan_switch.argtypes = [vp, pi32]
    L.cs_plan_destroy.argtypes = [vp]
    L.cs_plan_info.argtypes = [vp, pi64, pi64, pi32, pi32, pi32]
    L.cs_plan_kernel.argtypes = [vp, vp, i32, vp]
    L.cs_plan_status.argtypes = [vp, pi32, vp]
    L.cs_correlate.argtypes = [vp, vp, i64, vp, vp, vp]
    L.cs_correlate_fast.argtypes = [vp, vp, vp, vp, i32, i64, vp, vp, vp]
    L.cs_omp.argtypes = [vp, vp, i64, i32, ctypes.POINTER(Halt), vp, vp, vp, vp, vp]
    L.cs_omp_noalloc.argtypes = [vp, vp, i64, i32, ctypes.POINTER(Halt), vp, vp, vp, vp, vp]
    L.cs_omp_batched.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp), pi32, ctypes.POINTER(Halt),
                                 ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp]
    L.cs_omp_batched_tune.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp), pi32, ctypes.c_double, pi32, pi32,
                                      pi32, ctypes.POINTER(ctypes.c_float), i32, pi32, vp]
    L.cs_omp_batched_tune.restype = ctypes.c_int
    L.cs_sp.argtypes = [vp, vp, i64, i32, ctypes.POINTER(Halt), vp, vp, vp, vp, vp]
    L.cs_cosamp.argtypes = [vp, vp, i64, i32, ctypes.POINTER(Halt), vp, vp, vp, vp, vp]
    L.cs_plan_tune.argtypes = [vp, vp, i64, i32, ctypes.c_double, pi32, pi32, ctypes.POINTER(ctypes.c_float), i32,
                               pi32, vp]
    L.cs_server_create.argtypes = [i32, i64, ctypes.POINTER(vp)]
    L.cs_server_submit.argtypes = [vp, ctypes.POINTER(Request), vp, pi32, pi64]
    L.cs_server_poll.argtypes = [vp, ctypes.POINTER(Result), i32, i32, pi32]
    L.cs_server_stats.argtypes = [vp, pi64, pi64, pi64, pi64]
    L.cs_server_destroy.argtypes = [vp]
    L.cs_admit_next.argtypes = [pi64, pi32, i32, i64, i64, i32]
    L.cs_admit_next.restype = ctypes.c_int32
    L.cs_fma_probe.argtypes = [i32, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.cs_fma_probe.restype = ctypes.c_int
    for f in ("cs_plan_create", "cs_plan_create_ex", "cs_plan_memory", "cs_plan_switch", "cs_plan_destroy", "cs_plan_info", "cs_plan_status", "cs_plan_kernel", "cs_correlate",
              "cs_correlate_fast", "cs_omp", "cs_omp_batched", "cs_sp", "cs_cosamp", "cs_omp_noalloc",
              "cs_plan_tune", "cs_server_create", "cs_server_submit", "cs_server_poll", "cs_server_stats", "cs_server_destroy"):
        getattr(L, f).restype = ctypes.c_int
    L.cs_status_string.argtypes = [ctypes.c_int]
    L.cs_status_string.restype = ctypes.c_char_p
    L.cs_last_error.argtypes = []
    L.cs_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        L = load()
        raise CsError(f"csfast status {st}: {L.cs_status_string(st).decode()} {L.cs_last_error().decode()}".strip())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def working_dtype(kind: str, prec: str):
    import torch
    if kind == "dft":
        return torch.complex64 if prec == "fp32" else torch.complex128
    return torch.float32 if prec == "fp32" else torch.float64


def ls_dtype(kind: str):
    import torch
    return torch.complex128 if kind == "dft" else torch.float64


class Plan:
    """A plan for Phi = S_Omega A (cs_plan_create)."""

    def __init__(self, N: int, omega, kind: str = "dft", prec: str = "fp32", stream=None, c_storage: str = "full",
                 tensor_cores: bool = False):
        """c_storage: 'full', 'half' (DFT, CS_PLAN_C_HALF) or 'int' (WHT, CS_PLAN_C_INT);
        tensor_cores: CS_PLAN_TENSOR_CORES (WHT FP32)."""
        L = load()
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.int32))
        self.N, self.M, self.kind, self.prec = int(N), int(om.size), kind, prec
        flags = {"full": 0, "half": 1, "int": 2}[c_storage] | (4 if tensor_cores else 0)
        h = ctypes.c_void_p()
        _check(L.cs_plan_create_ex(self.N, om.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.M, KINDS[kind],
                                   PRECS[prec], flags, _stream(stream), ctypes.byref(h)))
        self._h = h
        self.dtype = working_dtype(kind, prec)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        n, m = ctypes.c_int64(), ctypes.c_int64()
        k, p, ts = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().cs_plan_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(k), ctypes.byref(p),
                                   ctypes.byref(ts)))
        return {"N": n.value, "M": m.value, "kind": k.value, "prec": p.value, "t_switch_default": ts.value}

    def switch_point(self) -> int:
        """The switch point used when t_switch < 0 (cs_plan_switch)."""
        t = ctypes.c_int32()
        _check(load().cs_plan_switch(self._h, ctypes.byref(t)))
        return t.value

    def memory(self) -> int:
        """Device bytes of the plan's tables (cs_plan_memory)."""
        b = ctypes.c_int64()
        _check(load().cs_plan_memory(self._h, ctypes.byref(b)))
        return b.value

    def tune(self, y, K: int, rel_tol: float = 1e-6, stream=None) -> tuple[int, dict]:
        """cs_plan_tune: measure the hybrid switch point on (batch, M) y; returns
        (t_best, {t_switch: ms})."""
        self._want(y, self.M)
        cap = 64
        cand = (ctypes.c_int32 * cap)()
        ms = (ctypes.c_float * cap)()
        tb, n = ctypes.c_int32(), ctypes.c_int32()
        _check(load().cs_plan_tune(self._h, _ptr(y), y.shape[0], K, rel_tol, ctypes.byref(tb), cand, ms, cap,
                                   ctypes.byref(n), _stream(stream)))
        return tb.value, {int(cand[i]): float(ms[i]) for i in range(min(cap, n.value))}

    def device_error(self, stream=None) -> int:
        """Kernel-detected error bits since the last call (cs_plan_status)."""
        e = ctypes.c_int32()
        _check(load().cs_plan_status(self._h, ctypes.byref(e), _stream(stream)))
        return e.value

    def kernel_vector(self, prec: str = "fp64", stream=None):
        import torch
        c = torch.empty(self.N, dtype=working_dtype(self.kind, prec), device="cuda")
        _check(load().cs_plan_kernel(self._h, _ptr(c), PRECS[prec], _stream(stream)))
        return c

    def _want(self, t, n_last):
        if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or t.shape[-1] != n_last:
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor with last dim {n_last}")

    def correlate(self, r, want_h: bool = True, stream=None):
        """h = Phi^H r for a (batch, M) tensor; returns (h or None, argmax)."""
        import torch
        self._want(r, self.M)
        B = r.shape[0]
        h = torch.empty(B, self.N, dtype=self.dtype, device="cuda") if want_h else None
        am = torch.empty(B, dtype=torch.int32, device="cuda")
        _check(load().cs_correlate(self._h, _ptr(r), B, _ptr(h), _ptr(am), _stream(stream)))
        return h, am

    def correlate_fast(self, h0, supp, x, want_h: bool = True, stream=None):
        """h = h0 - sum x(k) c(j (-) supp(k)) for (batch, N) h0, (batch, s) supp/x."""
        import torch
        self._want(h0, self.N)
        B = h0.shape[0]
        s = supp.shape[1] if supp.dim() == 2 else 0
        if supp.dtype != torch.int32 or x.dtype != self.dtype or not supp.is_contiguous() or not x.is_contiguous():
            raise ValueError("supp must be int32 and x of the plan's dtype, both contiguous")
        h = torch.empty(B, self.N, dtype=self.dtype, device="cuda") if want_h else None
        am = torch.empty(B, dtype=torch.int32, device="cuda")
        _check(load().cs_correlate_fast(self._h, _ptr(h0), _ptr(supp) if s else None, _ptr(x) if s else None, s, B,
                                        _ptr(h), _ptr(am), _stream(stream)))
        return h, am

    def omp_into(self, y, K: int, x, supp, iters, resnorm, rel_tol: float = 1e-6, path: str = "hybrid",
                 t_switch: int = -1, stream=None):
        """cs_omp into outputs the caller provides."""
        hl = Halt(rel_tol, PATHS[path], t_switch, 0)
        _check(load().cs_omp(self._h, _ptr(y), y.shape[0], K, ctypes.byref(hl), _ptr(x), _ptr(supp), _ptr(iters),
                             _ptr(resnorm), _stream(stream)))

    def omp(self, y, K: int, rel_tol: float = 1e-6, path: str = "hybrid", t_switch: int = -1, stream=None):
        """OMP on a (batch, M) tensor; returns x (FP64), supp, iters, resnorm."""
        import torch
        self._want(y, self.M)
        B = y.shape[0]
        x = torch.empty(B, K, dtype=ls_dtype(self.kind), device="cuda")
        supp = torch.empty(B, K, dtype=torch.int32, device="cuda")
        iters = torch.empty(B, dtype=torch.int32, device="cuda")
        res = torch.empty(B, dtype=torch.float64, device="cuda")
        self.omp_into(y, K, x, supp, iters, res, rel_tol, path, t_switch, stream)
        return x, supp, iters, res

    def pursuit_into(self, algo: str, y, K: int, x, supp, iters, resnorm, rel_tol: float = 1e-6,
                     path: str = "fast", max_iter: int = 0, t_switch: int = -1, stream=None):
        """cs_sp (algo 'sp') or cs_cosamp (algo 'cosamp') into outputs the caller provides."""
        hl = Halt(rel_tol, PATHS[path], t_switch, max_iter)
        fn = load().cs_sp if algo == "sp" else load().cs_cosamp
        _check(fn(self._h, _ptr(y), y.shape[0], K, ctypes.byref(hl), _ptr(x), _ptr(supp), _ptr(iters),
                  _ptr(resnorm), _stream(stream)))

    def pursuit(self, algo: str, y, K: int, rel_tol: float = 1e-6, path: str = "fast", max_iter: int = 0,
                stream=None):
        """Subspace pursuit or CoSaMP on a (batch, M) tensor; returns x (FP64), supp, iters, resnorm."""
        import torch
        self._want(y, self.M)
        B = y.shape[0]
        x = torch.empty(B, K, dtype=ls_dtype(self.kind), device="cuda")
        supp = torch.empty(B, K, dtype=torch.int32, device="cuda")
        iters = torch.empty(B, dtype=torch.int32, device="cuda")
        res = torch.empty(B, dtype=torch.float64, device="cuda")
        self.pursuit_into(algo, y, K, x, supp, iters, res, rel_tol, path, max_iter, stream=stream)
        return x, supp, iters, res


class Batch:
    """Outputs of cs_omp_batched for a list of instances with their own plans,
    preallocated so that the call itself can be repeated (timed, captured):
    x[b] FP64 [K_b], supp[b] int32 [K_b], iters int32 [count], resnorm FP64
    [count]."""

    def __init__(self, plans, ys, Ks):
        import torch
        if not (len(plans) == len(ys) == len(Ks)):
            raise ValueError("plans, ys and Ks differ in length")
        for p, y in zip(plans, ys):
            if y.dtype != p.dtype or y.ndim != 1 or y.shape[0] != p.M or not y.is_cuda or not y.is_contiguous():
                raise ValueError("each y must be a contiguous CUDA vector of its plan's M and working type")
        n = len(plans)
        self.plans, self.ys, self.Ks = list(plans), list(ys), [int(k) for k in Ks]
        self.x = [torch.zeros(k, dtype=ls_dtype(p.kind), device="cuda") for p, k in zip(plans, self.Ks)]
        self.supp = [torch.full((k,), -1, dtype=torch.int32, device="cuda") for k in self.Ks]
        self.iters = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.resnorm = torch.zeros(n, dtype=torch.float64, device="cuda")
        vpa = ctypes.c_void_p * max(n, 1)
        self._plans = vpa(*[p._h.value for p in plans])
        self._y = vpa(*[y.data_ptr() for y in ys])
        self._x = vpa(*[t.data_ptr() if t.numel() else None for t in self.x])
        self._s = vpa(*[t.data_ptr() if t.numel() else None for t in self.supp])
        self._K = (ctypes.c_int32 * max(n, 1))(*self.Ks)

    def run(self, rel_tol: float = 1e-6, path: str = "hybrid", t_switch: int = -1, stream=None):
        """cs_omp_batched on the instances (asynchronous on the stream)."""
        hl = Halt(rel_tol, PATHS[path], t_switch, 0)
        _check(load().cs_omp_batched(self._plans, len(self.plans), self._y, self._K, ctypes.byref(hl), self._x,
                                     self._s, _ptr(self.iters), _ptr(self.resnorm), _stream(stream)))
        return self


GROUPS = {0: "wht fp32 shared", 1: "wht fp32 global", 2: "wht fp64 shared", 3: "wht fp64 global",
          4: "dft fp32 shared", 5: "dft fp32 global", 6: "dft fp64 shared", 7: "dft fp64 global"}


def batch_tune(batch: "Batch", rel_tol: float = 1e-6, stream=None) -> list[dict]:
    """cs_omp_batched_tune on a Batch's instances: the launch shape chosen for
    each launch group, stored in the library for later cs_omp_batched calls."""
    cap = 8
    g, c, t = (ctypes.c_int32 * cap)(), (ctypes.c_int32 * cap)(), (ctypes.c_int32 * cap)()
    ms, n = (ctypes.c_float * cap)(), ctypes.c_int32()
    _check(load().cs_omp_batched_tune(batch._plans, len(batch.plans), batch._y, batch._K, rel_tol, g, c, t, ms, cap,
                                      ctypes.byref(n), _stream(stream)))
    return [{"group": GROUPS[g[i]], "ctas_per_sm": int(c[i]), "t_switch": int(t[i]), "ms": float(ms[i])}
            for i in range(min(cap, n.value))]


def batch_untune(stream=None):
    """Forget the launch shapes batch_tune stored for the current device."""
    n = ctypes.c_int32()
    _check(load().cs_omp_batched_tune(None, 0, None, None, 1e-6, None, None, None, None, 0, ctypes.byref(n),
                                      _stream(stream)))


def omp_batched(plans, ys, Ks, rel_tol: float = 1e-6, path: str = "hybrid", t_switch: int = -1, stream=None):
    """OMP on instances that each have their own plan and K (cs_omp_batched);
    returns a Batch with x, supp (lists), iters and resnorm."""
    return Batch(plans, ys, Ks).run(rel_tol, path, t_switch, stream)


def admit_next(footprints, bypassed, in_use: int, budget: int, max_bypass: int = 8) -> int:
    """cs_admit_next: the runtime's admission rule (host only)."""
    n = len(footprints)
    fp = (ctypes.c_int64 * max(n, 1))(*footprints)
    by = (ctypes.c_int32 * max(n, 1))(*bypassed)
    return int(load().cs_admit_next(fp, by, n, in_use, budget, max_bypass))


class Server:
    """The request runtime (cs_server_*): jobs of mixed sizes, kinds and
    algorithms admitted under a device-memory budget onto `workers` streams."""

    def __init__(self, workers: int = 4, budget_bytes: int = 8 << 30):
        h = ctypes.c_void_p()
        _check(load().cs_server_create(workers, int(budget_bytes), ctypes.byref(h)))
        self._h = h
        self._jobs = {}

    def submit(self, kind: str, prec: str, N: int, omega, y, K: int, algo: str = "omp", rel_tol: float = 1e-6,
               path: str = "hybrid", t_switch: int = -1, max_iter: int = 0) -> int:
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.int32))
        dt = {"dft": {"fp32": np.complex64, "fp64": np.complex128}, "wht": {"fp32": np.float32, "fp64": np.float64}}
        yv = np.ascontiguousarray(np.asarray(y, dtype=dt[kind][prec]))
        x = np.zeros(max(K, 1), dtype=np.complex128 if kind == "dft" else np.float64)
        supp = np.zeros(max(K, 1), dtype=np.int32)
        req = Request(KINDS[kind], PRECS[prec], ALGOS[algo], K, int(N), int(om.size),
                      om.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), yv.ctypes.data,
                      Halt(rel_tol, PATHS[path], t_switch, max_iter))
        t = ctypes.c_int64()
        _check(load().cs_server_submit(self._h, ctypes.byref(req), x.ctypes.data,
                                       supp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(t)))
        self._jobs[t.value] = (x, supp, K)
        return t.value

    def poll(self, wait_ms: int = 0, max_results: int = 256) -> list:
        buf = (Result * max_results)()
        n = ctypes.c_int32()
        _check(load().cs_server_poll(self._h, buf, max_results, wait_ms, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            x, supp, K = self._jobs.pop(r.ticket)
            out.append({"ticket": r.ticket, "status": r.status, "iters": r.iters, "device_error": r.device_error,
                        "resnorm": r.resnorm, "x": x[:K], "supp": supp[:K], "t_submit_us": r.t_submit_us,
                        "t_admit_us": r.t_admit_us, "t_done_us": r.t_done_us, "footprint_bytes": r.footprint_bytes})
        return out

    def wait_all(self, timeout_s: float = 600.0) -> list:
        import time
        out, t0 = [], time.time()
        while self._jobs and time.time() - t0 < timeout_s:
            out += self.poll(wait_ms=100)
        if self._jobs:
            raise CsError(f"{len(self._jobs)} jobs not finished after {timeout_s} s")
        return out

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().cs_server_stats(self._h, *[ctypes.byref(a) for a in v]))
        return dict(zip(("pending", "running", "completed", "bytes_in_use"), (a.value for a in v)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fma_probe(iters: int = 1 << 14, stream=None) -> float:
    """cs_fma_probe: queue the FP32 FMA probe on the stream; returns its flops."""
    f = ctypes.c_double()
    _check(load().cs_fma_probe(int(iters), None, ctypes.byref(f), _stream(stream)))
    return f.value
