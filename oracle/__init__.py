"""CPU oracle for the discrete Legendre transform (Hale & Townsend).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct FP64 / double-double
definitions of every quantity the GPU library computes (Eq. 1, Eq. 2, Eq. 3, the
matrix M of Sec. 3, the nodes and weights of the Gauss-Legendre rule).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library.

The arithmetic lives in ``oracle.c`` (compiled on first use with gcc into
``oracle/_build/liboracle.so``).  This module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        # no OpenMP runtime: the same code runs single-threaded
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, d = ctypes.c_int64, ctypes.c_double
        lib.orc_legendre_p.argtypes = [i64, _D, i64, _D]
        lib.orc_legendre_p_dd.argtypes = [i64, _D, _D, i64, _D]
        lib.orc_chebyshev_t.argtypes = [i64, _D, i64, _D]
        lib.orc_sincos_dd.argtypes = [d, d, _D, _D, _D, _D]
        lib.orc_legpts.argtypes = [i64, _I64, i64, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_legpts.restype = i64
        lib.orc_dlt_rows.argtypes = [i64, _D, i64, _D, _D, _D]
        lib.orc_dlt_t.argtypes = [i64, _D, _D, _D, _D]
        lib.orc_idlt.argtypes = [i64, _D, _D, _D, _D, _D, _D]
        lib.orc_idlt_rows.argtypes = [i64, _D, i64, _D, _D, _D, _D, _D]
        lib.orc_ndct_rows.argtypes = [i64, _D, i64, _D, _D, _D]
        lib.orc_ndct_t.argtypes = [i64, _D, _D, _D, _D]
        lib.orc_leg2cheb.argtypes = [i64, _D, _D]
        lib.orc_leg2cheb_t.argtypes = [i64, _D, _D]
        lib.orc_leg2cheb_matrix.argtypes = [i64, _D]
        lib.orc_dlt_t_rows.argtypes = [i64, _D, i64, _D, _D, _D]
        lib.orc_ndct_t_rows.argtypes = [i64, _D, i64, _D, _D, _D]
        lib.orc_leg2cheb_rows.argtypes = [i64, _D, _I64, i64, _D]
        lib.orc_leg2cheb_t_rows.argtypes = [i64, _D, _I64, i64, _D]
        lib.orc_legpts_f64.argtypes = [i64, _I64, i64, _D, _D, _D]
        lib.orc_legpts_f64.restype = i64
        lib.orc_dlt_rows_f64.argtypes = [i64, _D, i64, _D, _D]
        lib.orc_idlt_rows_f64.argtypes = [i64, _D, i64, _D, _D, _D]
        lib.orc_two_prod.argtypes = [d, d, _D, _D]
        lib.orc_two_sum.argtypes = [d, d, _D, _D]
        lib.orc_dd_div.argtypes = [d, d, d, d, _D, _D]
        lib.orc_dd_sqrt.argtypes = [d, d, _D, _D]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(_load().orc_num_threads())


# --------------------------------------------------------------------------
# polynomials
# --------------------------------------------------------------------------
def legendre_p(n: int, x) -> np.ndarray:
    """P_n(x) by the three-term recurrence in double-double."""
    x = _f64(x).ravel()
    out = np.empty_like(x)
    _load().orc_legendre_p(n, _dp(x), x.size, _dp(out))
    return out


def legendre_p_at(n: int, nodes) -> np.ndarray:
    """P_n at the double-double points held in ``nodes`` (x_hi + x_lo)."""
    xh, xl = _f64(nodes["x_hi"]).ravel(), _f64(nodes["x_lo"]).ravel()
    out = np.empty_like(xh)
    _load().orc_legendre_p_dd(n, _dp(xh), _dp(xl), xh.size, _dp(out))
    return out


def chebyshev_t(n: int, x) -> np.ndarray:
    """T_n(x) by T_{j+1} = 2x T_j - T_{j-1} in double-double."""
    x = _f64(x).ravel()
    out = np.empty_like(x)
    _load().orc_chebyshev_t(n, _dp(x), x.size, _dp(out))
    return out


def sincos_dd(hi: float, lo: float = 0.0):
    """(sin, cos) of a double-double angle, each as (hi, lo)."""
    v = [ctypes.c_double() for _ in range(4)]
    _load().orc_sincos_dd(hi, lo, *[ctypes.byref(t) for t in v])
    return (v[0].value, v[1].value), (v[2].value, v[3].value)


# --------------------------------------------------------------------------
# nodes and weights
# --------------------------------------------------------------------------
class Nodes(dict):
    """Gauss-Legendre nodes for a list of indices; arrays in double-double."""

    @property
    def x(self):
        return self["x_hi"] + self["x_lo"]

    @property
    def w(self):
        return self["w_hi"] + self["w_lo"]

    @property
    def theta(self):
        return self["theta_hi"] + self["theta_lo"]


def legpts(N: int, ks=None) -> Nodes:
    """Nodes k (theta ascending / x descending), weights and theta - theta^cheb1.

    ``ks`` selects node indices (default: all N).  Raises if any Newton iteration
    failed to settle.
    """
    ks = np.arange(N, dtype=np.int64) if ks is None else np.ascontiguousarray(ks, dtype=np.int64)
    m = ks.size
    out = {k: np.empty(m) for k in ("theta_hi", "theta_lo", "x_hi", "x_lo", "w_hi", "w_lo", "dtheta")}
    bad = _load().orc_legpts(N, ks.ctypes.data_as(_I64), m, *[_dp(out[k]) for k in
                             ("theta_hi", "theta_lo", "x_hi", "x_lo", "w_hi", "w_lo", "dtheta")])
    if bad:
        raise RuntimeError(f"oracle legpts: {bad} node(s) did not converge (N={N})")
    res = Nodes(out)
    res["k"] = ks
    res["N"] = N
    return res


# --------------------------------------------------------------------------
# transforms
# --------------------------------------------------------------------------
def dlt_rows(c, nodes: Nodes) -> np.ndarray:
    """Eq. 1 at the rows held in ``nodes``: f_k = sum_n c_n P_n(x_k)."""
    c = _f64(c)
    N = c.size
    xh, xl = _f64(nodes["x_hi"]), _f64(nodes["x_lo"])
    f = np.empty(xh.size)
    _load().orc_dlt_rows(N, _dp(c), xh.size, _dp(xh), _dp(xl), _dp(f))
    return f


def dlt(c, nodes: Nodes | None = None) -> np.ndarray:
    c = _f64(c)
    nodes = legpts(c.size) if nodes is None else nodes
    return dlt_rows(c, nodes)


def dlt_t(g, nodes: Nodes) -> np.ndarray:
    """(P^T g)_n = sum_k g_k P_n(x_k) over all N nodes."""
    g = _f64(g)
    N = g.size
    assert nodes["x_hi"].size == N
    out = np.empty(N)
    _load().orc_dlt_t(N, _dp(g), _dp(_f64(nodes["x_hi"])), _dp(_f64(nodes["x_lo"])), _dp(out))
    return out


def idlt(f, nodes: Nodes | None = None) -> np.ndarray:
    """Eq. 2: c_n = (n+1/2) sum_k w_k f_k P_n(x_k)."""
    f = _f64(f)
    N = f.size
    nodes = legpts(N) if nodes is None else nodes
    assert nodes["x_hi"].size == N
    out = np.empty(N)
    _load().orc_idlt(N, _dp(f), _dp(_f64(nodes["x_hi"])), _dp(_f64(nodes["x_lo"])),
                     _dp(_f64(nodes["w_hi"])), _dp(_f64(nodes["w_lo"])), _dp(out))
    return out


def idlt_rows(f_rows, nodes: Nodes, N: int) -> np.ndarray:
    """Contribution of the rows held in ``nodes`` to Eq. 2 (length-N vector);
    summed over all rows it is the IDLT."""
    f_rows = _f64(f_rows)
    out = np.empty(N)
    _load().orc_idlt_rows(N, _dp(f_rows), f_rows.size, _dp(_f64(nodes["x_hi"])),
                          _dp(_f64(nodes["x_lo"])), _dp(_f64(nodes["w_hi"])),
                          _dp(_f64(nodes["w_lo"])), _dp(out))
    return out


def ndct_rows(chat, nodes: Nodes) -> np.ndarray:
    """Eq. 3 at the rows held in ``nodes``: f_k = sum_n chat_n T_n(x_k)."""
    chat = _f64(chat)
    xh, xl = _f64(nodes["x_hi"]), _f64(nodes["x_lo"])
    f = np.empty(xh.size)
    _load().orc_ndct_rows(chat.size, _dp(chat), xh.size, _dp(xh), _dp(xl), _dp(f))
    return f


def ndct_t(g, nodes: Nodes) -> np.ndarray:
    """(T^T g)_n = sum_k g_k T_n(x_k) over all N nodes."""
    g = _f64(g)
    N = g.size
    out = np.empty(N)
    _load().orc_ndct_t(N, _dp(g), _dp(_f64(nodes["x_hi"])), _dp(_f64(nodes["x_lo"])), _dp(out))
    return out


def leg2cheb(c) -> np.ndarray:
    """chat = M c, the Legendre-to-Chebyshev matrix of Sec. 3."""
    c = _f64(c)
    out = np.empty_like(c)
    _load().orc_leg2cheb(c.size, _dp(c), _dp(out))
    return out


def leg2cheb_t(y) -> np.ndarray:
    """M^T y."""
    y = _f64(y)
    out = np.empty_like(y)
    _load().orc_leg2cheb_t(y.size, _dp(y), _dp(out))
    return out


def dlt_t_rows(g_rows, nodes: Nodes, N: int) -> np.ndarray:
    """(P^T g)_n for n < N when g vanishes off the rows held in ``nodes``
    (g_rows are its values there)."""
    g_rows = _f64(g_rows)
    out = np.empty(N)
    _load().orc_dlt_t_rows(N, _dp(g_rows), g_rows.size, _dp(_f64(nodes["x_hi"])), _dp(_f64(nodes["x_lo"])),
                           _dp(out))
    return out


def ndct_t_rows(g_rows, nodes: Nodes, N: int) -> np.ndarray:
    """(T^T g)_n for n < N when g vanishes off the rows held in ``nodes``."""
    g_rows = _f64(g_rows)
    out = np.empty(N)
    _load().orc_ndct_t_rows(N, _dp(g_rows), g_rows.size, _dp(_f64(nodes["x_hi"])), _dp(_f64(nodes["x_lo"])),
                            _dp(out))
    return out


def leg2cheb_rows(c, ks) -> np.ndarray:
    """(M c)_k at the listed k."""
    c = _f64(c)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    out = np.empty(ks.size)
    _load().orc_leg2cheb_rows(c.size, _dp(c), ks.ctypes.data_as(_I64), ks.size, _dp(out))
    return out


def leg2cheb_t_rows(y, ns) -> np.ndarray:
    """(M^T y)_n at the listed n."""
    y = _f64(y)
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    out = np.empty(ns.size)
    _load().orc_leg2cheb_t_rows(y.size, _dp(y), ns.ctypes.data_as(_I64), ns.size, _dp(out))
    return out


def leg2cheb_matrix(N: int) -> np.ndarray:
    m = np.empty((N, N))
    _load().orc_leg2cheb_matrix(N, _dp(m))
    return m


# --------------------------------------------------------------------------
# plain FP64 direct method (the timed CPU baseline; the dd functions above are
# the reference for accuracy)
# --------------------------------------------------------------------------
def legpts_f64(N: int, ks=None) -> dict:
    """Nodes (theta ascending), x and weights by Newton in double on the FP64
    recurrence; raises if a node did not settle."""
    ks = np.arange(N, dtype=np.int64) if ks is None else np.ascontiguousarray(ks, dtype=np.int64)
    out = {k: np.empty(ks.size) for k in ("theta", "x", "w")}
    bad = _load().orc_legpts_f64(N, ks.ctypes.data_as(_I64), ks.size, _dp(out["theta"]), _dp(out["x"]),
                                 _dp(out["w"]))
    if bad:
        raise RuntimeError(f"oracle legpts_f64: {bad} node(s) did not settle (N={N})")
    out["k"] = ks
    out["N"] = N
    return out


def dlt_rows_f64(c, x) -> np.ndarray:
    """Eq. 1 at the nodes x, every operation in double."""
    c, x = _f64(c), _f64(x)
    f = np.empty(x.size)
    _load().orc_dlt_rows_f64(c.size, _dp(c), x.size, _dp(x), _dp(f))
    return f


def idlt_rows_f64(f_rows, x, w, N: int) -> np.ndarray:
    """The rows' contribution to Eq. 2, every operation in double; summed over
    all N rows it is the plain FP64 IDLT."""
    f_rows, x, w = _f64(f_rows), _f64(x), _f64(w)
    out = np.empty(N)
    _load().orc_idlt_rows_f64(N, _dp(f_rows), f_rows.size, _dp(x), _dp(w), _dp(out))
    return out


# --------------------------------------------------------------------------
# dd primitives (for the tests that pin the arithmetic)
# --------------------------------------------------------------------------
def two_prod(a: float, b: float):
    hi, lo = ctypes.c_double(), ctypes.c_double()
    _load().orc_two_prod(a, b, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def two_sum(a: float, b: float):
    hi, lo = ctypes.c_double(), ctypes.c_double()
    _load().orc_two_sum(a, b, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def dd_div(a, b):
    qh, ql = ctypes.c_double(), ctypes.c_double()
    _load().orc_dd_div(a[0], a[1], b[0], b[1], ctypes.byref(qh), ctypes.byref(ql))
    return qh.value, ql.value


def dd_sqrt(a):
    rh, rl = ctypes.c_double(), ctypes.c_double()
    _load().orc_dd_sqrt(a[0], a[1], ctypes.byref(rh), ctypes.byref(rl))
    return rh.value, rl.value
