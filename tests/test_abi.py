"""The C-ABI library builds, loads without a GPU, and exports every function
that include/vine.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vine.h")).read()
    return sorted(set(re.findall(r"^\s*(?:vine_status|const char\*)\s+(vine_\w+)\s*\(", src, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("vine_batch_create", "vine_grow_step", "vine_simulate", "vine_get_state", "vine_grad",
              "vine_set_actuators", "vine_batch_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2509_15180_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header_and_defaults():
    from paper_2509_15180_gb300 import build
    build.build()
    from paper_2509_15180_gb300 import vine
    assert set(_declared()) <= set(vine.EXPORTED)
    p = vine.vine_params_default()
    assert (p.w_a, p.w_b, p.w_c, p.tol, p.discs_per_link) == (160.0, 15.0, 1.0, 1e-6, 2)


def _build_c_demo(tmp_path):
    """Compile and link the C caller of tests/c against include/vine.h and
    libvine.so (C99, warnings as errors): the header is plain C."""
    import subprocess
    from paper_2509_15180_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "abi_demo")
    libdir = os.path.dirname(lib)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "abi_demo.c"), "-o", exe, "-L", libdir, "-lvine",
                           "-Wl,-rpath," + libdir])
    return exe


def test_c_caller_compiles_and_links(tmp_path):
    assert os.path.exists(_build_c_demo(tmp_path))
