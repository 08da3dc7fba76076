"""FP64 CPU oracle for the BrainPy event-driven spiking-network hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never loads it, and it never loads the product
library: the two share no code.

``bp_oracle.c`` holds the per-element loops (Philox, JIT rows, event products,
the COBA network); this module compiles it with gcc on first use, loads it with
ctypes and wraps each routine in numpy.  ``bptt.py`` holds the differentiable
recurrent network and its hand-written adjoint, in numpy FP64.

Parity status of each routine (what pins it) is listed in the test files
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libbp_oracle.so")
_lock = threading.Lock()
_lib = None

W_HOMO, W_UNIFORM, W_NORMAL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile bp_oracle.c into a shared library with gcc -O2 (single thread)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Coba(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("n_e", ctypes.c_int64),
        ("dt", ctypes.c_double), ("tau_m", ctypes.c_double), ("tau_e", ctypes.c_double), ("tau_i", ctypes.c_double),
        ("V_rest", ctypes.c_double), ("V_th", ctypes.c_double), ("V_reset", ctypes.c_double),
        ("E_e", ctypes.c_double), ("E_i", ctypes.c_double), ("R", ctypes.c_double), ("I_ext", ctypes.c_double),
        ("w_e", ctypes.c_double), ("w_i", ctypes.c_double),
        ("ref_steps", ctypes.c_int32),
    ]


class _Conn(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p), ("data", ctypes.c_void_p),
        ("seed_e", ctypes.c_uint64), ("seed_i", ctypes.c_uint64), ("K", ctypes.c_int64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, u64, u32, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_double
        sig = {
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_splitmix64": (u64, [u64, u64]),
            "orc_projection_seed": (u64, [u64, ctypes.c_int]),
            "orc_jit_draw": (u32, [u64, u32, u32, u64]),
            "orc_jit_K": (i64, [f64]),
            "orc_jit_weight": (f64, [u64, u32, u64, ctypes.c_int, f64, f64]),
            "orc_jit_row": (i64, [u64, i64, ctypes.c_int, f64, f64, u32, i64, P, P, i64]),
            "orc_jitconn_event_mv": (None, [u64, i64, ctypes.c_int, f64, f64, i64, i64, P, P]),
            "orc_jitconn_mv": (None, [u64, i64, ctypes.c_int, f64, f64, i64, i64, P, P]),
            "orc_jitconn_mv_t": (None, [u64, i64, ctypes.c_int, f64, f64, i64, i64, P, P]),
            "orc_jit_row_lengths": (None, [u64, i64, i64, i64, P]),
            "orc_event_csrmv": (None, [i64, P, P, P, f64, P, P]),
            "orc_event_csr_count": (None, [i64, P, P, P, P]),
            "orc_csrmv_t": (None, [i64, P, P, P, f64, P, P]),
            "orc_event_csrmv_dw": (None, [i64, P, P, P, P, P]),
            "orc_coba_step": (i64, [P, P, P, P, P, P, P, P, P, P]),
            "orc_coba_run": (None, [P, P, i64, P, P, P, P, P, P, P, P, P, P]),
            "orc_rate_hz": (f64, [i64, i64, i64, f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC 2011): 4 counter words, 2 key words."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def splitmix64(state: int, j: int) -> int:
    """j-th output (0-based) of SplitMix64 started at `state`."""
    return int(_load().orc_splitmix64(state & (2**64 - 1), j))


def projection_seed(net_seed: int, projection: int) -> int:
    """Seed of projection 0 (excitatory rows) or 1 (inhibitory rows)."""
    return int(_load().orc_projection_seed(net_seed & (2**64 - 1), projection))


def jit_draw(seed: int, row: int, stream: int, k: int) -> int:
    return int(_load().orc_jit_draw(seed & (2**64 - 1), row, stream, k))


def jit_K(p: float) -> int:
    """Appendix C gap range K = ceil(2/p - 1), at least 1."""
    return int(_load().orc_jit_K(float(p)))


def jit_weight(seed, row, k, wkind, w0, w1) -> float:
    return float(_load().orc_jit_weight(seed & (2**64 - 1), row, k, wkind, w0, w1))


def jit_row(seed: int, K: int, row: int, n_post: int, wkind=W_HOMO, w0=1.0, w1=0.0):
    """Targets (int32) and weights (f64) of JIT row `row` (Appendix C)."""
    lib = _load()
    n = lib.orc_jit_row(seed & (2**64 - 1), K, wkind, w0, w1, row, n_post, None, None, 0)
    cols = np.zeros(max(n, 1), np.int32)
    w = np.zeros(max(n, 1), np.float64)
    lib.orc_jit_row(seed & (2**64 - 1), K, wkind, w0, w1, row, n_post, _p(cols), _p(w), n)
    return cols[:n], w[:n]


def jit_row_lengths(seed: int, K: int, n_pre: int, n_post: int):
    out = np.zeros(n_pre, np.int64)
    _load().orc_jit_row_lengths(seed & (2**64 - 1), K, n_pre, n_post, _p(out))
    return out


def jit_materialize(seed: int, K: int, n_pre: int, n_post: int, wkind=W_HOMO, w0=1.0, w1=0.0):
    """CSR (indptr int64, indices int32, weights f64) of the JIT matrix."""
    lens = jit_row_lengths(seed, K, n_pre, n_post)
    indptr = np.zeros(n_pre + 1, np.int64)
    np.cumsum(lens, out=indptr[1:])
    indices = np.zeros(int(indptr[-1]), np.int32)
    data = np.zeros(int(indptr[-1]), np.float64)
    for i in range(n_pre):
        c, w = jit_row(seed, K, i, n_post, wkind, w0, w1)
        indices[indptr[i]:indptr[i + 1]] = c
        data[indptr[i]:indptr[i + 1]] = w
    return indptr, indices, data


def jitconn_event_mv(seed, K, n_pre, n_post, events, wkind=W_HOMO, w0=1.0, w1=0.0, y=None):
    ev = _c(events, np.uint8)
    y = np.zeros(n_post, np.float64) if y is None else _c(y, np.float64).copy()
    _load().orc_jitconn_event_mv(seed & (2**64 - 1), K, wkind, w0, w1, n_pre, n_post, _p(ev), _p(y))
    return y


def jitconn_mv(seed, K, n_pre, n_post, x, wkind=W_HOMO, w0=1.0, w1=0.0):
    xx = _c(x, np.float64)
    y = np.zeros(n_post, np.float64)
    _load().orc_jitconn_mv(seed & (2**64 - 1), K, wkind, w0, w1, n_pre, n_post, _p(xx), _p(y))
    return y


def jitconn_mv_t(seed, K, n_pre, n_post, x, wkind=W_HOMO, w0=1.0, w1=0.0):
    xx = _c(x, np.float64)
    y = np.zeros(n_pre, np.float64)
    _load().orc_jitconn_mv_t(seed & (2**64 - 1), K, wkind, w0, w1, n_pre, n_post, _p(xx), _p(y))
    return y


# --------------------------------------------------------------------------- CSR
def event_csrmv(indptr, indices, data, events, n_post, w_homo=1.0):
    """Appendix B: y = W^T s over the spiking rows (FP64)."""
    ip, ix = _c(indptr, np.int64), _c(indices, np.int32)
    d = None if data is None else _c(data, np.float64)
    ev = _c(events, np.uint8)
    y = np.zeros(n_post, np.float64)
    _load().orc_event_csrmv(len(ip) - 1, _p(ip), _p(ix), _p(d), float(w_homo), _p(ev), _p(y))
    return y


def event_csr_count(indptr, indices, events, n_post):
    """Integer event counts c[post] (homogeneous-weight product without the weight)."""
    ip, ix = _c(indptr, np.int64), _c(indices, np.int32)
    ev = _c(events, np.uint8)
    c = np.zeros(n_post, np.int64)
    _load().orc_event_csr_count(len(ip) - 1, _p(ip), _p(ix), _p(ev), _p(c))
    return c


def csrmv_t(indptr, indices, data, x, w_homo=1.0):
    """Gather form y_pre = W x over all rows (FP64)."""
    ip, ix = _c(indptr, np.int64), _c(indices, np.int32)
    d = None if data is None else _c(data, np.float64)
    xx = _c(x, np.float64)
    y = np.zeros(len(ip) - 1, np.float64)
    _load().orc_csrmv_t(len(ip) - 1, _p(ip), _p(ix), _p(d), float(w_homo), _p(xx), _p(y))
    return y


def event_csrmv_dw(indptr, indices, events, delta):
    """dW[j] = s[row(j)] * delta[indices[j]] (FP64)."""
    ip, ix = _c(indptr, np.int64), _c(indices, np.int32)
    ev = _c(events, np.uint8)
    dd = _c(delta, np.float64)
    dw = np.zeros(len(ix), np.float64)
    _load().orc_event_csrmv_dw(len(ip) - 1, _p(ip), _p(ix), _p(ev), _p(dd), _p(dw))
    return dw


def spike_outer(x, delta):
    """Weight gradient of a spike-driven dense connection (Section 3.1: the
    reverse-mode rule of y_k = W^T x_k with binary x_k is dW = sum_k x_k dy_k^T):
    out[m][n] = sum_k [x[k][m] != 0] delta[k][n], in FP64 (x [K][M], delta
    [K][N])."""
    xb = (np.asarray(x) != 0).astype(np.float64)
    return xb.T @ np.asarray(delta, np.float64)


# --------------------------------------------------------------------------- COBA network
COBA_DEFAULTS = dict(dt=0.1, tau_m=20.0, tau_e=5.0, tau_i=10.0, V_rest=-60.0, V_th=-50.0, V_reset=-60.0,
                     E_e=0.0, E_i=-80.0, R=1.0, I_ext=20.0, w_e=0.6, w_i=6.7, tau_ref=5.0)


class CobaNet:
    """FP64 state of the COBA E/I network (Appendix F, Appendix N Listing S6).

    ``conn`` is either ("csr", indptr, indices, data_or_None) over all n rows, or
    ("jit", seed_e, seed_i, K).

    ``delay_e`` / ``delay_i``: synaptic delay of the E / I projection in steps
    (the delayed spike retrieval of Appendix D; 0 = the spikes of step t act at
    step t + 1).  Each projection keeps d + 1 pending event buffers: step t
    reads and clears buffer t mod (d + 1), then delivers its spikes into that
    same buffer, which is read again d + 1 steps later.

    ``align``: "post" (default) keeps one conductance per postsynaptic neuron
    and adds the delivered events to it (AlignPost, Section 4.3, Appendix E);
    "pre" keeps one synaptic trace per presynaptic neuron instead, s <- s a + z
    with the projection's decay a and the previous step's spikes z, and
    recomputes every step the conductance g = W^T s through the connection
    matrix (AlignPre, Appendix D).  For exponential synapses the two are the
    same dynamics (g_t = a g_{t-1} + W^T z_{t-1} follows from g = W^T s by
    linearity).  "pre" needs no delay.
    """

    def __init__(self, n, n_e, conn, V0, delay_e=0, delay_i=0, align="post", **params):
        p = dict(COBA_DEFAULTS)
        p.update(params)
        self.n, self.n_e = int(n), int(n_e)
        ref_steps = int(round(p.pop("tau_ref") / p["dt"]))
        self.P = _Coba(n=self.n, n_e=self.n_e, ref_steps=ref_steps, **p)
        self._keep = []
        if conn[0] == "csr":
            ip, ix = _c(conn[1], np.int64), _c(conn[2], np.int32)
            d = None if conn[3] is None else _c(conn[3], np.float64)
            self._keep = [ip, ix, d]
            self.C = _Conn(kind=0, indptr=ip.ctypes.data, indices=ix.ctypes.data,
                           data=None if d is None else d.ctypes.data, seed_e=0, seed_i=0, K=0)
        else:
            self.C = _Conn(kind=1, indptr=None, indices=None, data=None,
                           seed_e=conn[1] & (2**64 - 1), seed_i=conn[2] & (2**64 - 1), K=int(conn[3]))
        if delay_e < 0 or delay_i < 0:
            raise ValueError("delays must be >= 0")
        self.V = _c(V0, np.float64).copy()
        self.ge = np.zeros(self.n)
        self.gi = np.zeros(self.n)
        self.ref = np.zeros(self.n, np.int32)
        self.ring_e = [np.zeros(self.n) for _ in range(int(delay_e) + 1)]
        self.ring_i = [np.zeros(self.n) for _ in range(int(delay_i) + 1)]
        self.t = 0
        if align not in ("post", "pre"):
            raise ValueError("align must be 'post' or 'pre'")
        self.align = align
        if align == "pre":
            if delay_e or delay_i:
                raise ValueError("the AlignPre form here has no delay")
            if conn[0] == "csr":
                ip, ix, w = self._keep
            else:
                ipe, ixe, _ = jit_materialize(self.C.seed_e, self.C.K, self.n_e, self.n)
                ipi, ixi, _ = jit_materialize(self.C.seed_i, self.C.K, self.n - self.n_e, self.n)
                ip = np.concatenate([ipe, ipi[1:] + ipe[-1]])
                ix = np.concatenate([ixe, ixi])
                w = None
            self._pre_rows = np.repeat(np.arange(self.n), np.diff(ip))
            self._pre_cols = ix.astype(np.int64)
            self._pre_w = None if w is None else np.asarray(w, np.float64)
            self.s = np.zeros(self.n)                  # one trace per presynaptic neuron
            self._z = np.zeros(self.n)
            self._a = np.where(np.arange(self.n) < self.n_e, math.exp(-p["dt"] / p["tau_e"]),
                               math.exp(-p["dt"] / p["tau_i"]))

    @property
    def ye(self):
        """The E event buffer the next step reads."""
        return self.ring_e[self.t % len(self.ring_e)]

    @property
    def yi(self):
        return self.ring_i[self.t % len(self.ring_i)]

    def _align_pre_input(self):
        """Trace update and W^T s for this step; the step routine then sees
        g = 0 plus the recomputed conductance as its increment."""
        self.s = self.s * self._a + self._z
        contrib = self.s[self._pre_rows]
        if self._pre_w is not None:
            contrib = contrib * self._pre_w
        e_rows = self._pre_rows < self.n_e
        self.ye[:] = np.bincount(self._pre_cols[e_rows], weights=contrib[e_rows], minlength=self.n)
        self.yi[:] = np.bincount(self._pre_cols[~e_rows], weights=contrib[~e_rows], minlength=self.n)
        self.ge[:] = 0.0
        self.gi[:] = 0.0

    def step(self, return_vdec=False):
        """One step; returns the spike flags (and, if asked, the potential each
        threshold test saw, NaN for refractory neurons)."""
        spk = np.zeros(self.n, np.uint8)
        vdec = np.zeros(self.n) if return_vdec else None
        if self.align == "pre":
            self._align_pre_input()
        _load().orc_coba_step(ctypes.byref(self.P), ctypes.byref(self.C), _p(self.V), _p(self.ge), _p(self.gi),
                              _p(self.ref), _p(self.ye), _p(self.yi), _p(spk), _p(vdec))
        self.t += 1
        if self.align == "pre":
            self._z = spk.astype(np.float64)
        return (spk, vdec) if return_vdec else spk

    def run(self, T, raster=False, events=False):
        if len(self.ring_e) > 1 or len(self.ring_i) > 1 or self.align == "pre":
            return self._run_steps(T, raster, events)
        se = np.zeros(T, np.int64)
        si = np.zeros(T, np.int64)
        ev = np.zeros(T, np.int64) if events else None
        ras = np.zeros((T, self.n), np.uint8) if raster else None
        _load().orc_coba_run(ctypes.byref(self.P), ctypes.byref(self.C), T, _p(self.V), _p(self.ge), _p(self.gi),
                             _p(self.ref), _p(self.ye), _p(self.yi), _p(se), _p(si), _p(ev), _p(ras))
        self.t += T
        return dict(spikes_e=se, spikes_i=si, events=ev, raster=ras)

    def _run_steps(self, T, raster, events):
        se = np.zeros(T, np.int64)
        si = np.zeros(T, np.int64)
        ev = np.zeros(T, np.int64) if events else None
        ras = np.zeros((T, self.n), np.uint8) if raster else None
        lens = None
        if events:
            lens = row_lengths_of(self)
        for t in range(T):
            spk = self.step()
            se[t] = int(spk[:self.n_e].sum())
            si[t] = int(spk[self.n_e:].sum())
            if events:
                ev[t] = int(lens[spk.astype(bool)].sum())
            if raster:
                ras[t] = spk
        return dict(spikes_e=se, spikes_i=si, events=ev, raster=ras)


def row_lengths_of(net):
    """Out-degree of every row of an oracle network's connectivity."""
    if net.C.kind == 0:
        return np.diff(net._keep[0])
    K = net.C.K
    return np.concatenate([jit_row_lengths(net.C.seed_e, K, net.n_e, net.n),
                           jit_row_lengths(net.C.seed_i, K, net.n - net.n_e, net.n)])


def rate_hz(total_spikes, n, T, dt_ms):
    return float(_load().orc_rate_hz(int(total_spikes), int(n), int(T), float(dt_ms)))
