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
                     "bie_blockdiag_create", "bie_net_train", "bie_batch_run", "bie_kernel_modes_noalloc",
                     "bie_rho_inv_modes", "bie_kernel_modes_banded"):
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


def test_invalid_arguments_are_refused_before_any_device_call():
    """Documented error behaviour of the boundary: a null handle or pointer gives BIE_EINVAL (1) and a
    message naming the call, without touching the device (this runs on a machine without a GPU)."""
    lib = ctypes.CDLL(LIB)
    lib.bie_last_error.restype = ctypes.c_char_p
    vp, d, i32, i64, u = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint
    null = vp(None)
    calls = {
        "bie_surface_sample": (null, null, i32(4), i32(32), null, null),
        "bie_kernel_modes": (null, null, u(1), d(1.0), null, null, i64(1), null),
        "bie_assemble": (null, null, i32(0), d(1.0), d(1.0), null),
        "bie_assemble_near": (null, null, u(1), d(1.0), d(1.0), d(0.0), d(0.0), d(0.0), null),
        "bie_assemble_near_band": (null, null, u(1), d(1.0), d(1.0), d(0.0), d(0.0), d(0.0), null),
        "bie_solve": (null, i64(4), null, null, i32(1), null, null, null),
        "bie_field_eval": (null, null, i32(0), d(1.0), d(1.0), null, null, i64(1), i32(0), null),
        "bie_blockdiag_create": (null, i64(64), null, i32(32), null),
        "bie_batch_create": (null, i32(1), null, null, u(1), null, i64(1), null),
        "bie_matrix_create": (null, i64(4), null, u(0), null),
        "bie_matrix_matvec": (null, i32(0), null, i32(1), null),
        "bie_solve_matrix": (null, null, null, i32(1), null, null, null),
        "bie_rho_inv_modes": (null, null, null, null, null, i64(1), i32(64), d(1e-14), null, null),
        "bie_kernel_modes_banded": (null, null, d(1.0), null, null, i64(1), d(1e-14), null),
    }
    for name, args in calls.items():
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(*args) == 1, name
        assert lib.bie_last_error().decode().startswith(name), (name, lib.bie_last_error())
