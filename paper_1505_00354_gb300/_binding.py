"""ctypes binding of the gbdlt C ABI (include/gbdlt.h).

Argument marshalling only: every step of every transform runs in the CUDA
library ``_lib/libgbdlt.so``.  There is no CPU fallback; if the library is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

FP64 = 0
FP32 = 1
METHOD_AUTO = 0
METHOD_FAST = 1
METHOD_DIRECT = 2
MAX_BANDS = 32

STATUS = {
    0: "ok",
    -1: "invalid argument",
    -2: "unsupported N",
    -3: "CUDA error",
    -4: "device allocation failed",
    -5: "node iteration did not converge",
    -6: "unimplemented",
}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgbdlt.so")
_lib = None
_lock = threading.Lock()


class GbdltError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"gbdlt {where}: {STATUS.get(status, 'unknown')} ({status})")


class Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64),
        ("prec", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("L", ctypes.c_int),
        ("M", ctypes.c_int),
        ("K", ctypes.c_int),
        ("band_ns", ctypes.c_int64 * MAX_BANDS),
        ("band_ka", ctypes.c_int64 * MAX_BANDS),
        ("band_kb", ctypes.c_int64 * MAX_BANDS),
        ("rec_steps", ctypes.c_int64),
        ("seg_len", ctypes.c_int),
        ("flops_dlt", ctypes.c_double),
        ("bytes_dlt", ctypes.c_double),
        ("bytes_idlt", ctypes.c_double),
        ("workspace_bytes", ctypes.c_size_t),
        ("method", ctypes.c_int),
        ("direct_steps", ctypes.c_int64),
        ("head", ctypes.c_int64),
        ("M_fp32", ctypes.c_int),
        ("M_ff", ctypes.c_int),
        ("L_ff", ctypes.c_int),
        ("grid_n", ctypes.c_int64),
    ]

    def to_dict(self) -> dict:
        K = self.K
        return {
            "N": self.N, "prec": self.prec, "eps": self.eps, "L": self.L, "M": self.M, "K": K,
            "bands": [(self.band_ns[i], self.band_ka[i], self.band_kb[i]) for i in range(K)],
            "rec_steps": self.rec_steps, "seg_len": self.seg_len, "flops_dlt": self.flops_dlt,
            "bytes_dlt": self.bytes_dlt, "bytes_idlt": self.bytes_idlt,
            "workspace_bytes": self.workspace_bytes, "method": self.method,
            "direct_steps": self.direct_steps, "head": self.head,
            "M_fp32": self.M_fp32, "M_ff": self.M_ff,
            "L_ff": self.L_ff, "grid_n": self.grid_n,
        }


ENTRY_POINTS = (
    "gbdlt_plan_params", "gbdlt_plan_params_ex", "gbdlt_plan_create", "gbdlt_plan_create_ex",
    "gbdlt_plan_destroy", "gbdlt_plan_set_stream",
    "gbdlt_plan_sync", "gbdlt_plan_get_params", "gbdlt_plan_set_node_iterations", "gbdlt_plan_set_fft_staging", "gbdlt_plan_set_fft_mix", "gbdlt_plan_set_wait_limit",
    "gbdlt_legpts", "gbdlt_legpts_noalloc", "gbdlt_leg2cheb",
    "gbdlt_leg2cheb_t", "gbdlt_chebeval", "gbdlt_chebeval_t", "gbdlt_dlt", "gbdlt_dlt_t",
    "gbdlt_idlt", "gbdlt_idlt_t", "gbdlt_plan_profile", "gbdlt_plan_profile_read",
    "gbdlt_batch_create", "gbdlt_batch_create_ex", "gbdlt_batch_exec", "gbdlt_batch_info",
    "gbdlt_batch_group_info", "gbdlt_batch_group_info_ex", "gbdlt_batch_destroy",
    "gbdlt_status_string", "gbdlt_launch_count", "gbdlt_device_alloc_count", "gbdlt_fp64_fma_rate",
)


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"gbdlt CUDA library not found at {LIB_PATH}; build it with "
                "`python -m paper_1505_00354_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.gbdlt_plan_params.argtypes = [i64, i32, dbl, ctypes.POINTER(Params)]
        L.gbdlt_plan_params_ex.argtypes = [i64, i32, dbl, i32, ctypes.POINTER(Params)]
        L.gbdlt_plan_create.argtypes = [i64, i32, dbl, vp, ctypes.POINTER(vp)]
        L.gbdlt_plan_create_ex.argtypes = [i64, i32, dbl, i32, vp, ctypes.POINTER(vp)]
        L.gbdlt_plan_destroy.argtypes = [vp]
        L.gbdlt_plan_set_stream.argtypes = [vp, vp]
        L.gbdlt_plan_sync.argtypes = [vp]
        L.gbdlt_plan_get_params.argtypes = [vp, ctypes.POINTER(Params)]
        L.gbdlt_plan_set_node_iterations.argtypes = [vp, i32]
        L.gbdlt_plan_set_fft_staging.argtypes = [vp, i32]
        L.gbdlt_plan_set_fft_mix.argtypes = [vp, i32]
        L.gbdlt_plan_set_wait_limit.argtypes = [vp, i64]
        L.gbdlt_legpts.argtypes = [vp, vp, vp, vp, vp]
        L.gbdlt_legpts_noalloc.argtypes = [i64, vp, vp, vp, vp, vp]
        for name in ("gbdlt_leg2cheb", "gbdlt_leg2cheb_t", "gbdlt_chebeval", "gbdlt_chebeval_t",
                     "gbdlt_dlt", "gbdlt_dlt_t", "gbdlt_idlt", "gbdlt_idlt_t"):
            getattr(L, name).argtypes = [vp, vp, vp, i64]
        L.gbdlt_batch_create.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                         i64, i32, dbl, ctypes.POINTER(vp)]
        L.gbdlt_batch_create_ex.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                            i64, i32, dbl, i32, ctypes.POINTER(vp)]
        L.gbdlt_batch_group_info.argtypes = [vp, i64, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        L.gbdlt_batch_group_info_ex.argtypes = [vp, i64, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i64)]
        L.gbdlt_batch_exec.argtypes = [vp, vp, vp, vp]
        L.gbdlt_batch_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.gbdlt_batch_destroy.argtypes = [vp]
        L.gbdlt_plan_profile.argtypes = [vp, i32]
        L.gbdlt_plan_profile_read.argtypes = [vp, ctypes.c_char_p, i64]
        L.gbdlt_status_string.argtypes = [i32]
        L.gbdlt_status_string.restype = ctypes.c_char_p
        L.gbdlt_launch_count.restype = ctypes.c_uint64
        L.gbdlt_device_alloc_count.restype = ctypes.c_uint64
        L.gbdlt_fp64_fma_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        for name in ENTRY_POINTS:
            if name not in ("gbdlt_status_string", "gbdlt_launch_count", "gbdlt_device_alloc_count"):
                getattr(L, name).restype = i32
        L.gbdlt_plan_profile_read.restype = i64
        _lib = L
        return L


def _check(status: int, where: str):
    if status != 0:
        raise GbdltError(status, where)


def plan_params(N: int, prec: int = FP64, eps: float = 0.0, method: int = METHOD_AUTO) -> dict:
    """Parameters the library derives for (N, prec, eps, method); host only, no GPU."""
    p = Params()
    _check(lib().gbdlt_plan_params_ex(N, prec, eps, method, ctypes.byref(p)), "plan_params")
    return p.to_dict()


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().gbdlt_launch_count())


def device_alloc_count() -> int:
    """Device allocations (cudaMalloc calls) the library has made since it was loaded."""
    return int(lib().gbdlt_device_alloc_count())


def fp64_fma_rate(stream=None) -> float:
    """FP64 flops per second reached by the library's FMA-chain probe on the
    current device (the roofline denominator of the FP64 kernels)."""
    s = torch.cuda.current_stream() if stream is None else stream
    r = ctypes.c_double()
    _check(lib().gbdlt_fp64_fma_rate(ctypes.c_void_p(s.cuda_stream), ctypes.byref(r)), "fp64_fma_rate")
    return float(r.value)


def _dtype(prec: int):
    return torch.float64 if prec == FP64 else torch.float32


class Plan:
    """A transform plan for one length N and precision on the current CUDA device.

    Methods mirror the C ABI: leg2cheb, leg2cheb_t, chebeval, chebeval_t, dlt,
    dlt_t, idlt, idlt_t take a CUDA tensor of shape [..., N] (float64 for FP64
    plans, float32 for FP32 plans) and return a new tensor (or write ``out``).
    """

    def __init__(self, N: int, prec: int = FP64, eps: float = 0.0, stream=None, device=None,
                 method: int = METHOD_AUTO):
        self._h = None
        self.N = int(N)
        self.prec = prec
        self.dtype = _dtype(prec)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream() if stream is None else stream
            self.stream = s
            h = ctypes.c_void_p()
            _check(lib().gbdlt_plan_create_ex(self.N, prec, eps, method, ctypes.c_void_p(s.cuda_stream),
                                              ctypes.byref(h)), "plan_create")
        self._h = h

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.gbdlt_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def params(self) -> dict:
        p = Params()
        _check(lib().gbdlt_plan_get_params(self._h, ctypes.byref(p)), "plan_get_params")
        return p.to_dict()

    def sync(self):
        _check(lib().gbdlt_plan_sync(self._h), "plan_sync")

    def set_node_iterations(self, max_iter: int):
        """Cap the Newton iterations of later legpts() calls (0..24; 24 is the default)."""
        _check(lib().gbdlt_plan_set_node_iterations(self._h, int(max_iter)), "set_node_iterations")

    def set_fft_staging(self, enable: bool):
        """FP32 FFT passes staged by the tensor memory accelerator (default) or not."""
        _check(lib().gbdlt_plan_set_fft_staging(self._h, 1 if enable else 0), "set_fft_staging")

    def set_fft_mix(self, mode):
        """FP64 plans, Taylor FFTs: 0 / False two streams; 1 / True (default) one mixed
        FP64 / float-float launch pair at N >= 2^20; 2 mixed at every length above 4096."""
        _check(lib().gbdlt_plan_set_fft_mix(self._h, int(mode)), "set_fft_mix")

    def set_wait_limit(self, sm_cycles: int):
        """SM cycles a staged FFT pass waits for a tile copy (failure-path hook; default 2^32)."""
        _check(lib().gbdlt_plan_set_wait_limit(self._h, int(sm_cycles)), "set_wait_limit")

    def set_stream(self, stream):
        self.stream = stream
        _check(lib().gbdlt_plan_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "set_stream")

    def profile(self, mode: int = 1):
        """1: start/re-anchor per-kernel timing, 0: stop, 2: clear totals."""
        _check(lib().gbdlt_plan_profile(self._h, mode), "plan_profile")

    def profile_report(self) -> dict:
        """{kernel: {launches, ms, flops, bytes}} accumulated while profiling was on."""
        n = lib().gbdlt_plan_profile_read(self._h, None, 0)
        if n < 0:
            raise GbdltError(int(n), "plan_profile_read")
        buf = ctypes.create_string_buffer(int(n) + 1)
        lib().gbdlt_plan_profile_read(self._h, buf, n + 1)
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms, fl, by = line.split()
            out[name] = {"launches": int(cnt), "ms": float(ms), "flops": float(fl), "bytes": float(by)}
        return out

    def legpts(self):
        """Recompute the nodes on the GPU; returns (x, theta, w, dtheta) float64 tensors."""
        outs = [torch.empty(self.N, dtype=torch.float64, device=self.device) for _ in range(4)]
        _check(lib().gbdlt_legpts(self._h, *[ctypes.c_void_p(t.data_ptr()) for t in outs]), "legpts")
        return tuple(outs)

    def _run(self, name: str, x: torch.Tensor, out: torch.Tensor | None):
        if not x.is_cuda or x.dtype != self.dtype or x.shape[-1] != self.N:
            raise ValueError(f"{name}: expected a CUDA {self.dtype} tensor [..., {self.N}], got "
                             f"{x.dtype} {tuple(x.shape)} on {x.device}")
        x = x.contiguous()
        if out is None:
            out = torch.empty_like(x)
        elif out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous():
            raise ValueError(f"{name}: out must be a contiguous tensor like the input")
        batch = x.numel() // self.N if self.N else 0
        _check(getattr(lib(), "gbdlt_" + name)(self._h, ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), batch), name)
        return out

    def leg2cheb(self, c, out=None):
        return self._run("leg2cheb", c, out)

    def leg2cheb_t(self, y, out=None):
        return self._run("leg2cheb_t", y, out)

    def chebeval(self, chat, out=None):
        return self._run("chebeval", chat, out)

    def chebeval_t(self, g, out=None):
        return self._run("chebeval_t", g, out)

    def dlt(self, c, out=None):
        return self._run("dlt", c, out)

    def dlt_t(self, g, out=None):
        return self._run("dlt_t", g, out)

    def idlt(self, f, out=None):
        return self._run("idlt", f, out)

    def idlt_t(self, g, out=None):
        return self._run("idlt_t", g, out)


class Batch:
    """Uneven batch of DLTs (dir 0) and IDLTs (dir 1) executed as one CUDA-graph
    replay (gbdlt_batch_*); ``method`` METHOD_AUTO lets the library time both
    methods per (N, direction) group and keep the faster.  ``run(x)`` takes and
    returns the concatenation of the B vectors in the given order."""

    def __init__(self, Ns, dirs, prec: int = FP64, eps: float = 0.0, method: int = METHOD_AUTO):
        import numpy as np
        Ns = np.ascontiguousarray(Ns, dtype=np.int64)
        dirs = np.ascontiguousarray(dirs, dtype=np.int32)
        if Ns.shape != dirs.shape:
            raise ValueError("Ns and dirs must have the same length")
        self._h = None
        self.Ns, self.dirs, self.prec, self.dtype = Ns, dirs, prec, _dtype(prec)
        self.offsets = np.concatenate([[0], np.cumsum(Ns)])
        h = ctypes.c_void_p()
        _check(lib().gbdlt_batch_create_ex(Ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           dirs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           Ns.size, prec, eps, method, ctypes.byref(h)), "batch_create")
        self._h = h

    def info(self) -> dict:
        t, g, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().gbdlt_batch_info(self._h, ctypes.byref(t), ctypes.byref(g), ctypes.byref(k)), "batch_info")
        return {"total_elements": t.value, "groups": g.value, "graph_kernels": k.value}

    def groups(self) -> list:
        """Per group: N (a grid group's grid G), dir, count, method, the
        autotuner's timings, whether it runs inside its direction's persistent
        direct launch, and its number of distinct lengths."""
        out = []
        for g in range(self.info()["groups"]):
            N, d, c, m = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
            tf, td, fu, nl = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_int64()
            _check(lib().gbdlt_batch_group_info_ex(self._h, g, ctypes.byref(N), ctypes.byref(d), ctypes.byref(c),
                                                   ctypes.byref(m), ctypes.byref(tf), ctypes.byref(td),
                                                   ctypes.byref(fu), ctypes.byref(nl)),
                   "batch_group_info")
            out.append({"N": N.value, "dir": d.value, "count": c.value, "method": m.value,
                        "ms_fast": tf.value, "ms_direct": td.value, "fused": bool(fu.value),
                        "lengths": nl.value})
        return out

    def run(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        n = int(self.offsets[-1])
        if not x.is_cuda or x.dtype != self.dtype or x.numel() != n:
            raise ValueError(f"batch: expected a CUDA {self.dtype} tensor of {n} elements")
        x = x.contiguous()
        out = torch.empty_like(x) if out is None else out
        _check(lib().gbdlt_batch_exec(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "batch_exec")
        return out

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.gbdlt_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# convenience functions with a plan cache keyed by (N, prec, device, stream)
# --------------------------------------------------------------------------
_plans: dict = {}


def get_plan(N: int, prec: int, device=None, method: int = METHOD_AUTO) -> Plan:
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    stream = torch.cuda.current_stream(dev)
    key = (int(N), prec, dev, stream.cuda_stream, method)
    p = _plans.get(key)
    if p is None:
        p = Plan(N, prec, stream=stream, device=dev, method=method)
        _plans[key] = p
    return p


def _prec_of(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return FP64
    if t.dtype == torch.float32:
        return FP32
    raise ValueError(f"unsupported dtype {t.dtype}")


def _op(name):
    def f(x: torch.Tensor, out=None):
        p = get_plan(x.shape[-1], _prec_of(x), x.device)
        return getattr(p, name)(x, out)
    f.__name__ = name
    f.__doc__ = f"{name} of a CUDA tensor [..., N] through a cached plan."
    return f


leg2cheb = _op("leg2cheb")
leg2cheb_t = _op("leg2cheb_t")
chebeval = _op("chebeval")
chebeval_t = _op("chebeval_t")
dlt = _op("dlt")
dlt_t = _op("dlt_t")
idlt = _op("idlt")
idlt_t = _op("idlt_t")


def legpts(N: int, device=None):
    """(x, theta, w, dtheta) of the N-point Gauss-Legendre rule, computed on the GPU."""
    return get_plan(N, FP64, device).legpts()
