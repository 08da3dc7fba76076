"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/bp.h declares; the Python binding covers each of them.  No
compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        with open(h) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[a-zA-Z_][\w\s\*]*?\b(bp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_05106_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["bp_lif_step", "bp_event_csrmv", "bp_event_csrmv_t", "bp_event_csrmv_bwd", "bp_jitconn_event_mv",
                 "bp_jitconn_event_mv_bwd", "bp_network_step", "bp_simulate"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(bp_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu_and_binding_covers_header(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n)
    from paper_2311_05106_gb300 import binding
    assert set(declared_functions()) <= set(binding.exported_symbols())
    lib.bp_version.restype = ctypes.c_char_p
    assert lib.bp_version().decode().startswith("bp ")


def test_host_only_helpers(libpath):
    """Entry points that touch no device memory run on a machine without a GPU."""
    from paper_2311_05106_gb300 import binding as B
    p = B.bp_coba_params_default()
    assert (p.dt, p.tau_m, p.V_th, p.V_reset, p.w_e, p.w_i) == (0.1, 20.0, -50.0, -60.0, 0.6, 6.7)
    d = B.bp_jit_desc_init(7, 0.02)
    assert d.K == 99
    assert B.bp_jit_desc_init(7, 80.0 / 4e6).K == 99999
    with pytest.raises(B.BpError):
        B.bp_jit_desc_init(7, 0.0)
    assert B.bp_csr_tile_index_size(10, 100000, 57344) == 10 * 3 + 2  # + the two bound slots
    # equal tiles: the fewest tiles of at most bp_tile_cols() columns, each a
    # multiple of 32 columns, none of them nearly empty
    cap = B.bp_tile_cols()
    for n_post in (1, 31, 32, 1000, cap - 1, cap, cap + 1, 2 * cap, 2 * cap + 7, 1_000_000, 4_000_000, 2**31 - 1):
        W = B.bp_tile_cols_for(n_post)
        S = -(-n_post // cap)
        assert W % 32 == 0 and 0 < W <= cap
        assert -(-n_post // W) == S
        assert n_post - (S - 1) * W >= W - 32 * S  # the last tile is within 32 S columns of the others
    assert B.bp_tile_cols_for(1_000_000) == 52640 and B.bp_tile_cols_for(0) == 32
    import oracle as orc
    for s in (0, 2024, 2**63 + 5):
        for j in (0, 1):
            assert B.bp_projection_seed(s, j) == orc.projection_seed(s, j)


def test_snn_desc_defaults_and_host_checks(libpath):
    """bp_snn_desc round-trips through the binding's struct layout (defaults of
    the surrogate and regulariser fields read back), and invalid surrogate or
    regulariser settings are rejected on the host before any device work."""
    from paper_2311_05106_gb300 import binding as B
    d = B.bp_snn_desc_default()
    assert (d.dt, d.tau_m, d.tau_s, d.tau_o, d.V_th, d.slope, d.ckpt_every) == (1.0, 20.0, 100.0, 20.0, 1.0, 4.0, 100)
    assert (d.surrogate, d.sg_alpha, d.sg_width, d.lambda_v, d.v_hi, d.v_lo) == (B.BP_SG_SIGMOID, 0.3, 1.0, 0.0, 0.4, -2.0)
    d.B, d.T, d.n_in, d.n_rec, d.n_out, d.nnz = 2, 10, 8, 16, 3, 0
    base = B.bp_snn_workspace_bytes(d)
    assert base > 0 and base % 256 == 0
    L = B.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks fail first
    d.W_in = d.indptr = d.indices = d.w_rec = d.W_out = d.b_out = fake.value

    def variant(**kw):
        bad = B.SnnDesc.from_buffer_copy(d)
        for k, v in kw.items():
            setattr(bad, k, v)
        return ctypes.byref(bad)

    assert L.bp_snn_forward(variant(surrogate=7), fake, fake, fake, None) != 0
    assert b"surrogate" in L.bp_last_error()
    assert L.bp_snn_forward(variant(lambda_v=-1.0), fake, fake, fake, None) != 0
    assert b"lambda_v" in L.bp_last_error()
    assert L.bp_snn_reg_loss(variant(surrogate=B.BP_SG_RELU, sg_width=0.0), fake, fake, None) != 0
    assert b"sg_width" in L.bp_last_error()
    assert L.bp_lif_step_bwd(variant(lambda_v=0.1, v_lo=1.0, v_hi=0.5), 4, fake, fake, fake, fake, fake, fake, fake,
                             None) != 0
    assert b"v_lo" in L.bp_last_error()


def test_refractory_counter_range_host_check(libpath):
    """The refractory counters are one byte per neuron: a period of 255 steps
    is accepted and one of 256 is rejected on the host, with a message, by
    every entry point that takes COBA parameters (n = 0 makes no device call)."""
    from paper_2311_05106_gb300 import binding as B
    L = B.lib()
    p = B.bp_coba_params_default()
    p.tau_ref = 25.5                     # 255 steps at dt = 0.1 ms
    args = (0, 0, None, None, None, None, None, None, 1, None, None, None, None, None, None)
    assert L.bp_lif_step(ctypes.byref(p), *args) == 0
    p.tau_ref = 25.6                     # 256 steps
    assert L.bp_lif_step(ctypes.byref(p), *args) != 0
    assert b"refractory" in L.bp_last_error()
    d = B.NetDesc()
    d.n, d.n_e, d.coba = 10, 8, p
    h = ctypes.c_void_p()
    assert L.bp_network_create(ctypes.byref(d), ctypes.byref(h)) != 0
    assert b"refractory" in L.bp_last_error()


def test_operator_and_constructor_host_checks(libpath):
    """Invalid arguments to the event products, the JIT product, the spike
    compaction and the network / batch constructors are rejected on the host,
    with a message naming the problem, before any device work (this machine
    has no GPU; the pointers below are never dereferenced)."""
    from paper_2311_05106_gb300 import binding as B
    L = B.lib()
    fake = ctypes.c_void_p(256)

    def rejected(status, word):
        assert status != 0
        assert word in L.bp_last_error(), L.bp_last_error()

    H, F32 = B.BP_W_HOMO, B.BP_W_F32
    rejected(L.bp_event_csrmv(-1, 10, fake, fake, None, H, 1.0, fake, fake, 0, fake, 1, None, 0, 0, None),
             b"negative")
    rejected(L.bp_event_csrmv(10, 10, fake, fake, fake, F32, 1.0, fake, fake, 5, fake, 1, None, 0, 0, None),
             b"homogeneous")
    rejected(L.bp_event_csrmv(10, 10, fake, fake, None, H, 1.0, fake, fake, 11, fake, 1, None, 0, 0, None),
             b"max_spikes")
    rejected(L.bp_event_csrmv(10, 10, fake, fake, fake, 7, 1.0, fake, fake, 5, fake, 0, None, 0, 0, None),
             b"weight kind")
    rejected(L.bp_event_csrmv(10, 10, fake, fake, None, F32, 1.0, fake, fake, 5, fake, 0, None, 0, 0, None),
             b"weights are NULL")
    rejected(L.bp_event_csrmv(10, 10, fake, fake, None, H, 1.0, fake, fake, 5, fake, 1, fake, 100, 0, None),
             b"tile_cols")
    rejected(L.bp_event_csrmv(10, 10, fake, fake, fake, F32, 1.0, fake, fake, 5, fake, 0, None, 0,
                              B.BP_ACC_FIXED, None), b"BP_ACC_FIXED")
    rejected(L.bp_csr_tile_weight_bound(10, 10, fake, fake, None, F32, 1.0, 32, fake, fake, None), b"weights are NULL")
    rejected(L.bp_csr_tile_weight_bound(10, 10, fake, fake, fake, F32, 1.0, 33, fake, fake, None), b"tile_cols")
    rejected(L.bp_csr_tile_weight_bound(10, 10, fake, fake, fake, F32, 1.0, 32, fake, None, None), b"work is NULL")
    rejected(L.bp_words_compact(fake, -1, fake, fake, fake, None), b"n must be")
    rejected(L.bp_words_compact(fake, 10, fake, fake, None, None), b"count is NULL")
    rejected(L.bp_words_compact(None, 10, fake, fake, fake, None), b"required pointer")
    rejected(L.bp_words_scatter(fake, fake, -1, fake, 10, None), b"negative size")
    rejected(L.bp_words_scatter(None, fake, 5, fake, 10, None), b"required pointer")
    rejected(L.bp_event_csrmv_t(10, 10, None, fake, None, H, 1.0, fake, fake, None, 0, 0, None), b"indptr")
    rejected(L.bp_event_csrmv_t(10, 10, fake, fake, None, H, 1.0, None, fake, None, 0, 0, None), b"x_post")
    d = B.JitDesc()                      # K = 0: not initialised
    rejected(L.bp_jitconn_event_mv(ctypes.byref(d), 10, 10, fake, fake, 5, fake, 0, 0, None), b"K =")
    d = B.bp_jit_desc_init(1, 0.1, B.BP_JIT_NORMAL, 0.5, 0.1)
    rejected(L.bp_jitconn_event_mv(ctypes.byref(d), 10, 10, fake, fake, 5, fake, 1, 0, None), b"homogeneous")
    rejected(L.bp_spike_compact(-1, fake, fake, fake, None), b"out of range")
    rejected(L.bp_spike_compact(10, None, fake, fake, None), b"NULL")
    nd = B.NetDesc()
    h = ctypes.c_void_p()
    rejected(L.bp_network_create(ctypes.byref(nd), ctypes.byref(h)), b"out of range")
    bd = B.BatchDesc()
    rejected(L.bp_batch_create(ctypes.byref(bd), ctypes.byref(h)), b"missing")
    assert not h.value


def test_python_objects_reject_host_memory_and_bad_shapes():
    """The network objects hand raw pointers to the library, which reads them
    as device memory: host tensors, a CPU device, a short row-pointer array or
    mismatched per-network arrays are rejected in Python before any
    allocation or library call."""
    torch = pytest.importorskip("torch")
    import numpy as np
    from paper_2311_05106_gb300.network import BatchedNetworks, CobaNetwork
    with pytest.raises(ValueError, match="CUDA device"):
        CobaNetwork(100, device="cpu")
    with pytest.raises(ValueError, match="CUDA device"):
        BatchedNetworks(np.array([100]), np.array([1], np.uint64), device="cpu")
    ip = torch.zeros(101, dtype=torch.int64)
    ix = torch.zeros(0, dtype=torch.int32)
    with pytest.raises(ValueError, match="indptr"):
        CobaNetwork(100, conn="csr", csr=(ip, ix, None))        # host tensors
    with pytest.raises(ValueError, match="seeds"):
        BatchedNetworks(np.array([100, 200]), np.array([1], np.uint64))
    with pytest.raises(ValueError, match="V0"):
        CobaNetwork(100, V0=np.zeros(99, np.float32))


def test_bptt_descriptor_rejects_host_or_misshapen_parameters():
    """snn.make_desc hands the parameter pointers to the library as device
    memory: host tensors, wrong dtypes and wrong shapes are rejected first."""
    torch = pytest.importorskip("torch")
    from paper_2311_05106_gb300.snn import make_desc
    n_in, n_rec, n_out = 3, 4, 2
    W_in = torch.zeros(n_in, n_rec)
    ip = torch.zeros(n_rec + 1, dtype=torch.int64)
    ix = torch.zeros(0, dtype=torch.int32)
    with pytest.raises(ValueError, match="W_in must be a contiguous CUDA tensor"):
        make_desc(1, 5, n_in, n_rec, n_out, W_in, ip, ix, torch.zeros(0), torch.zeros(n_rec, n_out), torch.zeros(n_out))


def test_binding_checks_lengths_behind_raw_pointers():
    """Lengths the kernels cannot see through a pointer are checked by the
    binding first: weights shorter than the stored entries, a tile index
    shorter than bp_csr_tile_index writes, a spike list shorter than
    max_spikes (the tensors here are host tensors: the length checks come
    before any pointer is taken)."""
    torch = pytest.importorskip("torch")
    from paper_2311_05106_gb300 import binding as B
    n_pre, n_post = 10, 200000
    ip = torch.zeros(n_pre + 1, dtype=torch.int64)
    ix = torch.zeros(8, dtype=torch.int32)
    sl, ns = torch.zeros(n_pre, dtype=torch.int32), torch.zeros(1, dtype=torch.int32)
    y = torch.zeros(n_post, dtype=torch.float32)
    with pytest.raises(ValueError, match="weights for 8 stored entries"):
        B.bp_event_csrmv(ip, ix, torch.zeros(7), 0.0, sl, ns, y)
    tc = B.bp_tile_cols()
    short = torch.zeros(B.bp_csr_tile_index_size(n_pre, n_post, tc) - 1, dtype=torch.int32)
    with pytest.raises(ValueError, match="tile_ptr"):
        B.bp_event_csrmv(ip, ix, None, 1.0, sl, ns, y, tile_ptr=short, tile_cols=tc)
    with pytest.raises(ValueError, match="tile_ptr"):
        B.bp_csr_tile_index(ip, ix, n_post, tc, short)
    with pytest.raises(ValueError, match="spike_list"):
        B.bp_event_csrmv(ip, ix, None, 1.0, sl[:5], ns, y)


def test_dense_event_wrappers_check_lengths():
    """Both dense-event products check, before any library call, that the
    weights cover the stored entries, that the event vector holds one flag
    per presynaptic row, and (workspace form) that the workspace has the
    size bp_event_csrmv_dense_workspace_bytes reports (host tensors: the
    checks come before any pointer is taken)."""
    torch = pytest.importorskip("torch")
    from paper_2311_05106_gb300 import binding as B
    n_pre, n_post = 10, 64
    ip = torch.zeros(n_pre + 1, dtype=torch.int64)
    ix = torch.zeros(8, dtype=torch.int32)
    ev = torch.zeros(n_pre, dtype=torch.uint8)
    y = torch.zeros(n_post, dtype=torch.float32)
    ws = torch.zeros(B.bp_event_csrmv_dense_workspace_bytes(n_pre), dtype=torch.uint8)
    with pytest.raises(ValueError, match="weights for 8 stored entries"):
        B.bp_event_csrmv_dense_noalloc(ip, ix, torch.zeros(7), 0.0, ev, y)
    with pytest.raises(ValueError, match="weights for 8 stored entries"):
        B.bp_event_csrmv_dense(ip, ix, torch.zeros(7), 0.0, ev, ws, y)
    with pytest.raises(ValueError, match="events holds 9 flags"):
        B.bp_event_csrmv_dense_noalloc(ip, ix, None, 1.0, ev[:9], y)
    with pytest.raises(ValueError, match="events holds 9 flags"):
        B.bp_event_csrmv_dense(ip, ix, None, 1.0, ev[:9], ws, y)
    with pytest.raises(ValueError, match="workspace holds"):
        B.bp_event_csrmv_dense(ip, ix, None, 1.0, ev, ws[:-1], y)
