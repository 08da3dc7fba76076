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
        text = open(h).read()
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
    assert B.bp_csr_tile_index_size(10, 100000, 57344) == 10 * 3
    import oracle as orc
    for s in (0, 2024, 2**63 + 5):
        for j in (0, 1):
            assert B.bp_projection_seed(s, j) == orc.projection_seed(s, j)
