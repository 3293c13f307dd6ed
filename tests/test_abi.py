"""The C ABI: libbie.so loads on a machine without a GPU and exports every function that
include/bie.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2608_16208_b300", "libbie.so")
HEADER = os.path.join(ROOT, "include", "bie.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(bie_[a-z0-9_]+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("bie_surface_sample", "bie_kernel_modes", "bie_assemble", "bie_solve", "bie_field_eval",
                     "bie_blockdiag_create", "bie_net_train", "bie_batch_run", "bie_kernel_modes_noalloc"):
        assert required in names
    assert len(names) >= 38


def test_library_exports_every_declared_function():
    if not os.path.exists(LIB):
        subprocess.run([sys.executable, os.path.join(ROOT, "paper_2608_16208_b300", "build.py")], check=True)
    lib = ctypes.CDLL(LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_parameter_count_matches_oracle():
    import oracle.precond as P
    m = re.search(r"#define\s+BIE_NET_PARAMS\s+(\d+)", open(HEADER).read())
    assert int(m.group(1)) == P.N_PARAMS
