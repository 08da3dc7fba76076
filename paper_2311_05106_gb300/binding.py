"""Thin Python binding of libbp's C ABI (include/bp.h).

Argument marshalling only: every function takes torch CUDA tensors (device
memory allocated by PyTorch), passes their data pointers and sizes to the C
entry point of the same name on the current torch CUDA stream, and raises
``BpError`` on a non-zero status.  No computation of the method happens here.

The library is loaded from the package's ``_build`` directory; if it is
missing the first call raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

BP_OK = 0
BP_ERR_INVALID, BP_ERR_CUDA, BP_ERR_TIMEOUT, BP_ERR_OOM, BP_ERR_UNSUPPORTED, BP_ERR_DEVICE = 1, 2, 3, 4, 5, 6
BP_W_HOMO, BP_W_F32, BP_W_BF16 = 0, 1, 2
BP_JIT_HOMO, BP_JIT_UNIFORM, BP_JIT_NORMAL = 0, 1, 2
BP_OVERWRITE, BP_ACC_GLOBAL, BP_ACC_SHARED, BP_ACC_FIXED = 1, 2, 4, 8
BP_CONN_CSR, BP_CONN_JIT = 0, 1


class BpError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s returned status %d: %s" % (fn, status, msg))
        self.status = status


c_i64, c_i32, c_u32, c_u64, c_f32, c_f64 = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_float, ctypes.c_double)
VP = ctypes.c_void_p


class CobaParams(ctypes.Structure):
    _fields_ = [("dt", c_f64), ("tau_m", c_f64), ("tau_e", c_f64), ("tau_i", c_f64), ("tau_ref", c_f64),
                ("V_rest", c_f64), ("V_th", c_f64), ("V_reset", c_f64), ("E_e", c_f64), ("E_i", c_f64),
                ("R", c_f64), ("I_ext", c_f64), ("w_e", c_f64), ("w_i", c_f64)]


class JitDesc(ctypes.Structure):
    _fields_ = [("seed", c_u64), ("p", c_f64), ("K", c_i64), ("wkind", c_i32), ("w0", c_f32), ("w1", c_f32)]


class NetDesc(ctypes.Structure):
    _fields_ = [("n", c_i64), ("n_e", c_i64), ("coba", CobaParams), ("conn_kind", c_i32),
                ("indptr", VP), ("indices", VP), ("data", VP), ("wkind", c_i32),
                ("tile_ptr", VP), ("tile_cols", c_i32),
                ("seed", c_u64), ("p", c_f64),
                ("V", VP), ("ge", VP), ("gi", VP), ("ref", VP), ("ye", VP), ("yi", VP),
                ("spike_list", VP), ("n_spikes", VP), ("totals", VP), ("spk", VP),
                ("delay_e", c_i32), ("delay_i", c_i32), ("delay_buf", VP),
                ("align", c_i32), ("trace", VP)]


BP_ALIGN_POST = 0
BP_ALIGN_PRE = 1


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_nets", c_i32), ("n", VP), ("n_e", VP), ("seed", VP), ("p", VP), ("coba", CobaParams),
                ("V", VP), ("ge", VP), ("gi", VP), ("ref", VP), ("totals", VP),
                ("indptr", VP), ("indices", VP)]


class SnnDesc(ctypes.Structure):
    _fields_ = [("B", c_i32), ("T", c_i32), ("n_in", c_i32), ("n_rec", c_i32), ("n_out", c_i32),
                ("dt", c_f64), ("tau_m", c_f64), ("tau_s", c_f64), ("tau_o", c_f64),
                ("V_rest", c_f64), ("V_reset", c_f64), ("V_th", c_f64), ("R", c_f64), ("slope", c_f64),
                ("ckpt_every", c_i32),
                ("W_in", VP), ("indptr", VP), ("indices", VP), ("w_rec", VP), ("w_rec_kind", c_i32),
                ("W_out", VP), ("b_out", VP), ("nnz", c_i64),
                ("surrogate", c_i32), ("sg_alpha", c_f64), ("sg_width", c_f64),
                ("lambda_v", c_f64), ("v_hi", c_f64), ("v_lo", c_f64)]


BP_SG_SIGMOID = 0
BP_SG_RELU = 1


_SIGS = {
    "bp_version": (ctypes.c_char_p, []),
    "bp_last_error": (ctypes.c_char_p, []),
    "bp_sync_status": (c_i32, [VP]),
    "bp_tile_cols": (c_i32, []),
    "bp_tile_cols_for": (c_i32, [c_i64]),
    "bp_coba_params_default": (c_i32, [ctypes.POINTER(CobaParams)]),
    "bp_lif_step": (c_i32, [ctypes.POINTER(CobaParams), c_i64, c_i64, VP, VP, VP, VP, VP, VP, c_i32, VP, VP, VP, VP,
                            VP, VP]),
    "bp_spike_compact": (c_i32, [c_i64, VP, VP, VP, VP]),
    "bp_event_csrmv": (c_i32, [c_i64, c_i64, VP, VP, VP, c_i32, c_f32, VP, VP, c_i64, VP, c_i32, VP, c_i32, c_u32,
                               VP]),
    "bp_event_csrmv_dense_workspace_bytes": (ctypes.c_size_t, [c_i64]),
    "bp_event_csrmv_dense": (c_i32, [c_i64, c_i64, VP, VP, VP, c_i32, c_f32, VP, VP, VP, c_i32, VP, c_i32, c_u32,
                                     VP]),
    "bp_event_csrmv_dense_noalloc_max_pre": (c_i64, []),
    "bp_event_csrmv_dense_noalloc": (c_i32, [c_i64, c_i64, VP, VP, VP, c_i32, c_f32, VP, VP, c_i32, c_u32, VP]),
    "bp_csr_tile_index_size": (c_i64, [c_i64, c_i64, c_i32]),
    "bp_csr_tile_index": (c_i32, [c_i64, c_i64, VP, VP, c_i32, VP, VP]),
    "bp_csr_tile_weight_bound": (c_i32, [c_i64, c_i64, VP, VP, VP, c_i32, c_f32, c_i32, VP, VP, VP]),
    "bp_csr_check": (c_i32, [c_i64, c_i64, c_i64, VP, VP, VP, VP]),
    "bp_event_csrmv_t": (c_i32, [c_i64, c_i64, VP, VP, VP, c_i32, c_f32, VP, VP, VP, c_i32, c_u32, VP]),
    "bp_event_csrmv_bwd": (c_i32, [c_i64, c_i64, VP, VP, VP, c_i32, c_f32, VP, VP, c_i64, VP, VP, VP, VP, c_i32, VP]),
    "bp_jit_desc_init": (c_i32, [ctypes.POINTER(JitDesc), c_u64, c_f64, c_i32, c_f32, c_f32]),
    "bp_jitconn_event_mv": (c_i32, [ctypes.POINTER(JitDesc), c_i64, c_i64, VP, VP, c_i64, VP, c_i32, c_u32, VP]),
    "bp_jitconn_event_mv_bwd": (c_i32, [ctypes.POINTER(JitDesc), c_i64, c_i64, VP, VP, VP]),
    "bp_jitconn_mv": (c_i32, [ctypes.POINTER(JitDesc), c_i64, c_i64, VP, VP, c_u32, VP]),
    "bp_jit_materialize_csr": (c_i32, [ctypes.POINTER(JitDesc), c_i64, c_i64, VP, VP, VP, c_i32, VP]),
    "bp_projection_seed": (c_u64, [c_u64, c_i32]),
    "bp_network_create": (c_i32, [ctypes.POINTER(NetDesc), ctypes.POINTER(VP)]),
    "bp_network_reset_counters": (c_i32, [VP, VP]),
    "bp_network_step": (c_i32, [VP, VP]),
    "bp_network_step_count": (c_i64, [VP]),
    "bp_network_set_step_count": (c_i32, [VP, c_i64, VP]),
    "bp_simulate": (c_i32, [VP, c_i64, VP, VP]),
    "bp_simulate_prepare": (c_i32, [VP, c_i64, VP]),
    "bp_words_compact": (c_i32, [VP, c_i64, VP, VP, VP, VP]),
    "bp_words_scatter": (c_i32, [VP, VP, c_i64, VP, c_i64, VP]),
    "bp_network_stats": (c_i32, [VP, VP, VP]),
    "bp_network_destroy": (c_i32, [VP]),
    "bp_batch_layout": (c_i64, [c_i32, VP, VP]),
    "bp_batch_create": (c_i32, [ctypes.POINTER(BatchDesc), ctypes.POINTER(VP)]),
    "bp_batch_info": (c_i32, [VP, VP, VP, VP]),
    "bp_batch_tuning": (c_i32, [VP, VP, VP, VP, VP]),
    "bp_batch_set_tuning": (c_i32, [VP, c_i32, c_i32, c_i32]),
    "bp_batch_reset_counters": (c_i32, [VP, VP]),
    "bp_batch_simulate": (c_i32, [VP, c_i64, VP]),
    "bp_batch_autotune": (c_i32, [VP, c_i32, VP, VP]),
    "bp_batch_prepare": (c_i32, [VP, c_i64, VP]),
    "bp_batch_destroy": (c_i32, [VP]),
    "bp_roof_philox_threads": (c_i64, []),
    "bp_roof_philox": (c_i32, [c_i64, c_u64, VP, VP]),
    "bp_roof_l2_red_threads": (c_i64, []),
    "bp_roof_l2_red": (c_i32, [VP, c_i64, c_i64, VP]),
    "bp_roof_copy": (c_i32, [VP, VP, c_i64, c_i32, VP]),
    "bp_snn_desc_default": (c_i32, [ctypes.POINTER(SnnDesc)]),
    "bp_snn_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(SnnDesc)]),
    "bp_snn_forward": (c_i32, [ctypes.POINTER(SnnDesc), VP, VP, VP, VP]),
    "bp_snn_loss": (c_i32, [c_i32, c_i32, VP, VP, VP, VP, VP]),
    "bp_snn_reg_loss": (c_i32, [ctypes.POINTER(SnnDesc), VP, VP, VP]),
    "bp_lif_step_bwd": (c_i32, [ctypes.POINTER(SnnDesc), c_i64, VP, VP, VP, VP, VP, VP, VP, VP]),
    "bp_snn_backward": (c_i32, [ctypes.POINTER(SnnDesc), VP, VP, VP, VP, VP, VP, VP, VP]),
    "bp_spike_outer_workspace": (ctypes.c_size_t, [c_i64, c_i32, c_i32]),
    "bp_spike_outer": (c_i32, [VP, VP, c_i64, c_i32, c_i32, VP, c_u32, VP, ctypes.c_size_t, VP]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libbp (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError("libbp.so is not built (%s); run __graft_entry__.build() or "
                                   "python -m paper_2311_05106_gb300._build" % path)
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _check(name, status):
    if status != BP_OK:
        raise BpError(name, status, lib().bp_last_error().decode())


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor, got a %s tensor" % t.device)
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return VP(t.data_ptr())


# the current stream's raw handle without building a torch Stream object
# (0.1 us against ~3 us per call; the public route where torch lacks it)
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_cur_device = getattr(torch._C, "_cuda_getDevice", None)


def _stream(stream=None):
    if stream is None:
        if _raw_stream is not None and _cur_device is not None:
            return VP(_raw_stream(_cur_device()))
        stream = torch.cuda.current_stream()
    return VP(stream.cuda_stream)


def _wkind(data):
    if data is None:
        return BP_W_HOMO
    if data.dtype == torch.float32:
        return BP_W_F32
    if data.dtype == torch.bfloat16:
        return BP_W_BF16
    raise ValueError("weights must be float32 or bfloat16, got %s" % data.dtype)


def _csr_sizes(indices, data, n_pre, n_post, tile_ptr, tile_cols, spike_list=None, max_spikes=0):
    """Lengths the kernels rely on but cannot see through a raw pointer: one
    weight per stored entry, a tile index of the size bp_csr_tile_index
    writes, a spike list of at least max_spikes entries."""
    if data is not None and indices is not None and data.numel() < indices.numel():
        raise ValueError("data holds %d weights for %d stored entries" % (data.numel(), indices.numel()))
    if tile_ptr is not None and tile_cols > 0:
        need = int(lib().bp_csr_tile_index_size(n_pre, n_post, int(tile_cols)))
        if tile_ptr.dtype != torch.int32 or tile_ptr.numel() < need:
            raise ValueError("tile_ptr must be int32 with at least %d entries" % need)
    if spike_list is not None and spike_list.numel() < min(max_spikes, n_pre):
        raise ValueError("spike_list holds %d entries, max_spikes is %d" % (spike_list.numel(), max_spikes))


# ------------------------------------------------------------------ library
def bp_version() -> str:
    return lib().bp_version().decode()


def bp_last_error() -> str:
    return lib().bp_last_error().decode()


def bp_sync_status(stream=None) -> int:
    return int(lib().bp_sync_status(_stream(stream)))


def bp_tile_cols() -> int:
    return int(lib().bp_tile_cols())


def bp_tile_cols_for(n_post) -> int:
    """Equal tiles of at most bp_tile_cols() columns over n_post columns."""
    return int(lib().bp_tile_cols_for(int(n_post)))


def bp_coba_params_default(**overrides) -> CobaParams:
    p = CobaParams()
    _check("bp_coba_params_default", lib().bp_coba_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, float(v))
    return p


# ------------------------------------------------------------------ a1-a4
def bp_lif_step(p, n_e, V, ge, gi, ref, ye, yi, spike_list, n_spikes, I_vec=None, spk=None, spike_totals=None,
                stream=None):
    counts = 1 if ye.dtype == torch.int32 else 0
    if ref.dtype != torch.uint8:
        raise TypeError("ref holds one-byte refractory counters (torch.uint8), got %s" % ref.dtype)
    _check("bp_lif_step", lib().bp_lif_step(ctypes.byref(p), V.numel(), n_e, _p(V), _p(ge), _p(gi), _p(ref), _p(ye),
                                            _p(yi), counts, _p(I_vec), _p(spk), _p(spike_list), _p(n_spikes),
                                            _p(spike_totals), _stream(stream)))


def bp_spike_compact(events, spike_list, n_spikes, stream=None):
    _check("bp_spike_compact", lib().bp_spike_compact(events.numel(), _p(events), _p(spike_list), _p(n_spikes),
                                                      _stream(stream)))


# ------------------------------------------------------------------ a5
def bp_event_csrmv(indptr, indices, data, w_homo, spike_list, n_spikes, y, n_post=None, tile_ptr=None, tile_cols=0,
                   flags=0, max_spikes=None, stream=None):
    n_pre = indptr.numel() - 1
    n_post = y.numel() if n_post is None else n_post
    counts = 1 if y.dtype == torch.int32 else 0
    ms = n_pre if max_spikes is None else max_spikes
    _csr_sizes(indices, data, n_pre, n_post, tile_ptr, tile_cols, spike_list, ms)
    _check("bp_event_csrmv", lib().bp_event_csrmv(n_pre, n_post, _p(indptr), _p(indices), _p(data), _wkind(data),
                                                  float(w_homo), _p(spike_list), _p(n_spikes), ms, _p(y), counts,
                                                  _p(tile_ptr), int(tile_cols), int(flags), _stream(stream)))


def bp_event_csrmv_dense_workspace_bytes(n_pre) -> int:
    return int(lib().bp_event_csrmv_dense_workspace_bytes(n_pre))


def _dense_events(events, n_pre):
    """The dense event vector the compaction reads: one byte per presynaptic row."""
    if events is None or events.numel() < n_pre:
        raise ValueError("events holds %d flags for %d presynaptic rows"
                         % (0 if events is None else events.numel(), n_pre))
    if events.dtype != torch.uint8:
        raise ValueError("events must be uint8")


def bp_event_csrmv_dense(indptr, indices, data, w_homo, events, workspace, y, tile_ptr=None, tile_cols=0, flags=0,
                         stream=None):
    n_pre = indptr.numel() - 1
    counts = 1 if y.dtype == torch.int32 else 0
    _csr_sizes(indices, data, n_pre, y.numel(), tile_ptr, tile_cols)
    _dense_events(events, n_pre)
    need = bp_event_csrmv_dense_workspace_bytes(n_pre)
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        raise ValueError("workspace holds %d bytes, bp_event_csrmv_dense_workspace_bytes(%d) = %d"
                         % (0 if workspace is None else workspace.numel() * workspace.element_size(), n_pre, need))
    _check("bp_event_csrmv_dense", lib().bp_event_csrmv_dense(n_pre, y.numel(), _p(indptr), _p(indices), _p(data),
                                                              _wkind(data), float(w_homo), _p(events), _p(workspace),
                                                              _p(y), counts, _p(tile_ptr), int(tile_cols), int(flags),
                                                              _stream(stream)))


def bp_event_csrmv_dense_noalloc_max_pre() -> int:
    return int(lib().bp_event_csrmv_dense_noalloc_max_pre())


def bp_event_csrmv_dense_noalloc(indptr, indices, data, w_homo, events, y, flags=0, stream=None):
    """bp_event_csrmv_dense without a workspace argument: the library's fixed
    scratch holds the spike list (for callers that cannot allocate)."""
    n_pre = indptr.numel() - 1
    counts = 1 if y.dtype == torch.int32 else 0
    _csr_sizes(indices, data, n_pre, y.numel(), None, 0)
    _dense_events(events, n_pre)
    _check("bp_event_csrmv_dense_noalloc",
           lib().bp_event_csrmv_dense_noalloc(n_pre, y.numel(), _p(indptr), _p(indices), _p(data), _wkind(data),
                                              float(w_homo), _p(events), _p(y), counts, int(flags), _stream(stream)))


def bp_csr_tile_index_size(n_pre, n_post, tile_cols) -> int:
    return int(lib().bp_csr_tile_index_size(n_pre, n_post, tile_cols))


def bp_csr_tile_index(indptr, indices, n_post, tile_cols, tile_ptr, stream=None):
    _csr_sizes(indices, None, indptr.numel() - 1, n_post, tile_ptr, tile_cols)
    _check("bp_csr_tile_index", lib().bp_csr_tile_index(indptr.numel() - 1, n_post, _p(indptr), _p(indices),
                                                        int(tile_cols), _p(tile_ptr), _stream(stream)))


def bp_csr_tile_weight_bound(indptr, indices, data, w_homo, n_post, tile_cols, tile_ptr, work=None, stream=None):
    """Records in tile_ptr's last two entries the bounds of the fixed-point
    tile sums (BP_ACC_FIXED): the largest absolute sum of one row's entries in
    one column (FP32 bits) and the most rows with an entry in one column.
    work: int32 [n_post] device scratch (allocated here when None)."""
    _csr_sizes(indices, data, indptr.numel() - 1, n_post, tile_ptr, tile_cols)
    if work is None:
        work = torch.empty(max(int(n_post), 1), dtype=torch.int32, device=indptr.device)
    if work.dtype != torch.int32 or work.numel() < int(n_post):
        raise ValueError("work must hold n_post = %d int32 values" % int(n_post))
    _check("bp_csr_tile_weight_bound", lib().bp_csr_tile_weight_bound(
        indptr.numel() - 1, int(n_post), _p(indptr), _p(indices), _p(data), _wkind(data), float(w_homo),
        int(tile_cols), _p(tile_ptr), _p(work), _stream(stream)))


def bp_csr_check(indptr, indices, n_post, out, stream=None):
    """out int64 [4]: bad row extents, out-of-range indices, unsorted rows,
    rows with repeated columns."""
    _check("bp_csr_check", lib().bp_csr_check(indptr.numel() - 1, int(n_post), indices.numel(), _p(indptr),
                                              _p(indices), _p(out), _stream(stream)))


def bp_event_csrmv_t(indptr, indices, data, w_homo, x_post, y_pre, flags=0, stream=None, tile_ptr=None, tile_cols=0):
    _csr_sizes(indices, data, indptr.numel() - 1, x_post.numel(), tile_ptr, tile_cols)
    _check("bp_event_csrmv_t", lib().bp_event_csrmv_t(indptr.numel() - 1, x_post.numel(), _p(indptr), _p(indices),
                                                      _p(data), _wkind(data), float(w_homo), _p(x_post), _p(y_pre),
                                                      _p(tile_ptr), int(tile_cols), int(flags), _stream(stream)))


def bp_event_csrmv_bwd(indptr, indices, data, w_homo, spike_list, n_spikes, dy, dw=None, dx_pre=None,
                       max_spikes=None, stream=None, tile_ptr=None, tile_cols=0):
    n_pre = indptr.numel() - 1
    ms = n_pre if max_spikes is None else max_spikes
    _csr_sizes(indices, data, n_pre, dy.numel(), tile_ptr, tile_cols, spike_list, ms)
    _check("bp_event_csrmv_bwd", lib().bp_event_csrmv_bwd(n_pre, dy.numel(), _p(indptr), _p(indices), _p(data),
                                                          _wkind(data), float(w_homo), _p(spike_list), _p(n_spikes),
                                                          ms, _p(dy), _p(dw), _p(dx_pre), _p(tile_ptr),
                                                          int(tile_cols), _stream(stream)))


# ------------------------------------------------------------------ a6
def bp_jit_desc_init(seed, p, wkind=BP_JIT_HOMO, w0=1.0, w1=0.0) -> JitDesc:
    d = JitDesc()
    _check("bp_jit_desc_init", lib().bp_jit_desc_init(ctypes.byref(d), int(seed) & (2**64 - 1), float(p), int(wkind),
                                                      float(w0), float(w1)))
    return d


def bp_jitconn_event_mv(desc, n_pre, spike_list, n_spikes, y, flags=0, max_spikes=None, stream=None):
    counts = 1 if y.dtype == torch.int32 else 0
    ms = n_pre if max_spikes is None else max_spikes
    _csr_sizes(None, None, n_pre, y.numel(), None, 0, spike_list, ms)
    _check("bp_jitconn_event_mv", lib().bp_jitconn_event_mv(ctypes.byref(desc), n_pre, y.numel(), _p(spike_list),
                                                            _p(n_spikes), ms, _p(y), counts, int(flags),
                                                            _stream(stream)))


def bp_jitconn_event_mv_bwd(desc, dy, dx_pre, stream=None):
    _check("bp_jitconn_event_mv_bwd", lib().bp_jitconn_event_mv_bwd(ctypes.byref(desc), dx_pre.numel(), dy.numel(),
                                                                    _p(dy), _p(dx_pre), _stream(stream)))


def bp_jitconn_mv(desc, x_pre, y_post, flags=0, stream=None):
    _check("bp_jitconn_mv", lib().bp_jitconn_mv(ctypes.byref(desc), x_pre.numel(), y_post.numel(), _p(x_pre),
                                                _p(y_post), int(flags), _stream(stream)))


def bp_jit_materialize_csr(desc, n_pre, n_post, indptr, indices=None, data=None, stream=None):
    dk = _wkind(data)
    _check("bp_jit_materialize_csr", lib().bp_jit_materialize_csr(ctypes.byref(desc), n_pre, n_post, _p(indptr),
                                                                  _p(indices), _p(data), dk, _stream(stream)))


def bp_projection_seed(seed, projection) -> int:
    return int(lib().bp_projection_seed(int(seed) & (2**64 - 1), int(projection)))


def jit_materialize(desc, n_pre, n_post, data_dtype=None, device="cuda"):
    """Allocates and fills a CSR copy of a JIT matrix (two library calls; the
    row count is read back to size the index array)."""
    indptr = torch.empty(n_pre + 1, dtype=torch.int64, device=device)
    bp_jit_materialize_csr(desc, n_pre, n_post, indptr)
    nnz = int(indptr[-1].item())
    indices = torch.empty(max(nnz, 1), dtype=torch.int32, device=device)
    data = None if data_dtype is None else torch.empty(max(nnz, 1), dtype=data_dtype, device=device)
    bp_jit_materialize_csr(desc, n_pre, n_post, indptr, indices, data)
    return indptr, indices[:nnz], (None if data is None else data[:nnz])


# ------------------------------------------------------------------ a7/a8
def bp_network_create(desc: NetDesc):
    h = VP()
    _check("bp_network_create", lib().bp_network_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def bp_network_reset_counters(net, stream=None):
    _check("bp_network_reset_counters", lib().bp_network_reset_counters(net, _stream(stream)))


def bp_network_step_count(net) -> int:
    return int(lib().bp_network_step_count(net))


def bp_network_set_step_count(net, step, stream=None):
    _check("bp_network_set_step_count", lib().bp_network_set_step_count(net, int(step), _stream(stream)))


def bp_network_step(net, stream=None):
    _check("bp_network_step", lib().bp_network_step(net, _stream(stream)))


def bp_simulate(net, T, record=None, stream=None):
    _check("bp_simulate", lib().bp_simulate(net, int(T), _p(record), _stream(stream)))


def bp_simulate_prepare(net, T, stream=None):
    _check("bp_simulate_prepare", lib().bp_simulate_prepare(net, int(T), _stream(stream)))


def bp_words_compact(x, idx, val, count, stream=None):
    """Nonzero 32-bit words of x as (idx, val) pairs; count (int32 [1]) gets
    their number."""
    n = x.numel() * x.element_size() // 4
    if x.element_size() * x.numel() != 4 * n or idx.numel() < n or val.numel() < n or count.numel() < 1:
        raise ValueError("x must hold whole 32-bit words; idx and val need room for n = %d pairs" % n)
    _check("bp_words_compact", lib().bp_words_compact(_p(x), n, _p(idx), _p(val), _p(count), _stream(stream)))


def bp_words_scatter(idx, val, count, x, stream=None):
    """x[idx[k]] = val[k] (as 32-bit words) for k < count."""
    n = x.numel() * x.element_size() // 4
    if int(count) > min(idx.numel(), val.numel()):
        raise ValueError("count exceeds the pairs given")
    _check("bp_words_scatter", lib().bp_words_scatter(_p(idx), _p(val), int(count), _p(x), n, _stream(stream)))


def bp_network_stats(net, out, stream=None):
    _check("bp_network_stats", lib().bp_network_stats(net, _p(out), _stream(stream)))


def bp_network_destroy(net):
    _check("bp_network_destroy", lib().bp_network_destroy(net))


# ------------------------------------------------------------------ a9
def bp_batch_layout(n):
    """Offsets (numpy int64 [n_nets + 1]) of the concatenated batch layout."""
    import numpy as np
    nn = np.ascontiguousarray(n, dtype=np.int64)
    off = np.zeros(len(nn) + 1, np.int64)
    total = lib().bp_batch_layout(len(nn), nn.ctypes.data_as(VP), off.ctypes.data_as(VP))
    if total < 0:
        raise ValueError("bad network sizes")
    return off


def bp_batch_create(desc: BatchDesc):
    h = VP()
    _check("bp_batch_create", lib().bp_batch_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def bp_batch_info(b):
    bins, threads, total = c_i32(), c_i32(), c_i64()
    _check("bp_batch_info", lib().bp_batch_info(b, ctypes.byref(bins), ctypes.byref(threads), ctypes.byref(total)))
    return bins.value, threads.value, total.value


def bp_batch_tuning(b):
    """(threads, lanes_per_row, ctas_per_sm, stored_rows) of the batch."""
    th, g, ps, st = c_i32(), c_i32(), c_i32(), c_i32()
    _check("bp_batch_tuning", lib().bp_batch_tuning(b, ctypes.byref(th), ctypes.byref(g), ctypes.byref(ps),
                                                    ctypes.byref(st)))
    return th.value, g.value, ps.value, st.value


def bp_batch_set_tuning(b, threads, lanes_per_row, ctas_per_sm):
    _check("bp_batch_set_tuning", lib().bp_batch_set_tuning(b, int(threads), int(lanes_per_row), int(ctas_per_sm)))


def bp_batch_reset_counters(b, stream=None):
    _check("bp_batch_reset_counters", lib().bp_batch_reset_counters(b, _stream(stream)))


def bp_batch_simulate(b, T, stream=None):
    _check("bp_batch_simulate", lib().bp_batch_simulate(b, int(T), _stream(stream)))


def bp_batch_prepare(b, T, stream=None):
    _check("bp_batch_prepare", lib().bp_batch_prepare(b, int(T), _stream(stream)))


def bp_batch_autotune(b, probe_steps=20, stream=None):
    th = c_i32()
    _check("bp_batch_autotune", lib().bp_batch_autotune(b, int(probe_steps), ctypes.byref(th), _stream(stream)))
    return th.value


def bp_batch_destroy(b):
    _check("bp_batch_destroy", lib().bp_batch_destroy(b))


# ------------------------------------------------------------------ a10
def bp_snn_desc_default() -> SnnDesc:
    d = SnnDesc()
    _check("bp_snn_desc_default", lib().bp_snn_desc_default(ctypes.byref(d)))
    return d


def bp_snn_workspace_bytes(desc) -> int:
    return int(lib().bp_snn_workspace_bytes(ctypes.byref(desc)))


def bp_snn_forward(desc, u, m, workspace, stream=None):
    _check("bp_snn_forward", lib().bp_snn_forward(ctypes.byref(desc), _p(u), _p(m), _p(workspace), _stream(stream)))


def bp_snn_loss(m, labels, loss, g_m, stream=None):
    B, n_out = m.shape
    _check("bp_snn_loss", lib().bp_snn_loss(B, n_out, _p(m), _p(labels), _p(loss), _p(g_m), _stream(stream)))


def bp_snn_reg_loss(desc, workspace, loss, stream=None):
    _check("bp_snn_reg_loss", lib().bp_snn_reg_loss(ctypes.byref(desc), _p(workspace), _p(loss), _stream(stream)))


def bp_snn_backward(desc, u, g_m, workspace, dW_in, dw_rec, dW_out, db_out, stream=None):
    _check("bp_snn_backward", lib().bp_snn_backward(ctypes.byref(desc), _p(u), _p(g_m), _p(workspace), _p(dW_in),
                                                    _p(dw_rec), _p(dW_out), _p(db_out), _stream(stream)))


def bp_lif_step_bwd(desc, Vp, z, Vbar, zbar, Ibar_next, Ibar, Vbar_prev, stream=None):
    _check("bp_lif_step_bwd", lib().bp_lif_step_bwd(ctypes.byref(desc), Vp.numel(), _p(Vp), _p(z), _p(Vbar), _p(zbar),
                                                    _p(Ibar_next), _p(Ibar), _p(Vbar_prev), _stream(stream)))


def bp_spike_outer_workspace(K, M, N) -> int:
    return int(lib().bp_spike_outer_workspace(int(K), int(M), int(N)))


def spike_outer_workspace(K, M, N, device="cuda"):
    """A 1024-byte aligned uint8 workspace tensor for bp_spike_outer (a view
    into a slightly larger allocation)."""
    nbytes = bp_spike_outer_workspace(K, M, N)
    raw = torch.empty(nbytes + 1024, dtype=torch.uint8, device=device)
    off = (-raw.data_ptr()) % 1024
    return raw[off:off + nbytes]


def bp_spike_outer(x, delta, out, overwrite=False, work=None, stream=None):
    """out[m][n] (+)= sum_k [x[k][m] != 0] delta[k][n]; x uint8 [K][M], delta
    float32 [K][N], out float32 [M][N] (all contiguous, on the device)."""
    K, M = x.shape
    K2, N = delta.shape
    if K2 != K or tuple(out.shape) != (M, N):
        raise ValueError("shapes: x [K][M], delta [K][N], out [M][N]")
    if x.dtype != torch.uint8 or delta.dtype != torch.float32 or out.dtype != torch.float32:
        raise ValueError("x uint8, delta and out float32")
    if not (x.is_contiguous() and delta.is_contiguous() and out.is_contiguous()):
        raise ValueError("x, delta and out must be contiguous")
    if work is None:
        work = spike_outer_workspace(K, M, N, device=out.device)
    nbytes = work.numel() * work.element_size()
    _check("bp_spike_outer", lib().bp_spike_outer(_p(x), _p(delta), int(K), int(M), int(N), _p(out),
                                                  BP_OVERWRITE if overwrite else 0, _p(work), nbytes,
                                                  _stream(stream)))


# ------------------------------------------------------------------ measurement kernels
def bp_roof_philox_threads() -> int:
    return int(lib().bp_roof_philox_threads())


def bp_roof_philox(blocks_per_thread, sink, seed=1, stream=None):
    """Philox-only draws: 4 words per block per thread; sink uint32 [threads]."""
    if sink.dtype != torch.int32 or sink.numel() < bp_roof_philox_threads():
        raise ValueError("sink must be int32 with bp_roof_philox_threads() entries")
    _check("bp_roof_philox", lib().bp_roof_philox(int(blocks_per_thread), int(seed) & (2**64 - 1), _p(sink),
                                                  _stream(stream)))


def bp_roof_l2_red_threads() -> int:
    return int(lib().bp_roof_l2_red_threads())


def bp_roof_l2_red(y, per_thread, stream=None):
    """threads x per_thread scattered +1 reductions into y int32."""
    if y.dtype != torch.int32:
        raise ValueError("y must be int32")
    _check("bp_roof_l2_red", lib().bp_roof_l2_red(_p(y), y.numel(), int(per_thread), _stream(stream)))


def bp_roof_copy(src, dst, reps, stream=None):
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() < nbytes:
        raise ValueError("dst is shorter than src")
    _check("bp_roof_copy", lib().bp_roof_copy(_p(src), _p(dst), nbytes, int(reps), _stream(stream)))
