"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/slimgraph.h declares.  No GPU needed: nothing here launches work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "slimgraph.h")


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__

    return __graft_entry__._builder().build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sg_compress", "sg_divergence", "sg_graph_from_device", "sg_graph_from_host", "sg_graph_free",
                 "sg_ctx_create", "sg_last_error", "sg_pagerank", "sg_cc_count", "sg_kl_divergence"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sg_[a-z_0-9]+)\b", out))
    assert set(declared_functions()) <= exported


def test_build_targets_sm103a_only():
    import __graft_entry__

    b = __graft_entry__._builder()
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "--use_fast_math" not in b.FLAGS


@pytest.mark.gpu
def test_device_code_matches_the_gpu(libpath):
    import torch

    import paper_1912_08950_gb300 as sg

    v = ctypes.c_int()
    sg._check(sg.lib().sg_kernel_arch(0, ctypes.byref(v)))
    major, minor = torch.cuda.get_device_capability(0)
    assert v.value == 10 * major + minor == 103


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "slimgraph.h"\nint main(void){ sg_status s = SG_OK; (void)s; return 0; }\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-c", str(src), "-o", str(tmp_path / "t.o")])


def test_no_gpu_gives_clean_error(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1912_08950_gb300 as sg

    h = ctypes.c_void_p()
    st = sg.lib().sg_ctx_create(0, None, ctypes.byref(h))
    assert st != sg.SG_OK and not h.value
    assert sg.lib().sg_last_error()


def test_null_arguments_rejected(libpath):
    import paper_1912_08950_gb300 as sg

    L = sg.lib()
    assert L.sg_compress(None, None, 0, 0.5, 1, 0, None) == sg.SG_ERR_INVALID_ARG
    assert L.sg_ctx_create(0, None, None) == sg.SG_ERR_INVALID_ARG
    assert b"NULL" in L.sg_last_error()
