"""The C-ABI library loads and exports every entry point include/motifs.h declares;
host-side input validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "motifs.h")).read()
    return sorted(set(re.findall(r"^(?:mt_status|const char\*)\s+(mt_[a-z_0-9]+)\(", src, re.M)))


@pytest.fixture(scope="module")
def mtlib():
    from paper_1804_09741_gb300 import build as b
    if not b.up_to_date():
        if shutil.which(b.NVCC) is None and not os.path.exists(b.NVCC):
            pytest.skip("nvcc not available to build the library")
        b.build()
    import paper_1804_09741_gb300 as mt
    return mt.load_library()


def test_every_declared_symbol_is_exported(mtlib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(mtlib, name), name


def test_binding_covers_the_header():
    import paper_1804_09741_gb300 as mt
    assert set(_declared()) == set(mt.SIGNATURES)


def test_status_strings(mtlib):
    for st in range(8):
        assert mtlib.mt_status_str(st)


def _load(mtlib, n, rp, col):
    rp = np.ascontiguousarray(rp, np.int32)
    col = np.ascontiguousarray(col if len(col) else [0], np.int32)
    h = ctypes.c_void_p()
    return mtlib.mt_graph_load_csr(n, int(rp[-1]), rp.ctypes.data, col.ctypes.data, None,
                                   ctypes.byref(h))


@pytest.mark.parametrize("case", ["selfloop", "range", "negative", "monotone", "rowend", "n0"])
def test_host_validation_rejects_malformed_csr(mtlib, case):
    n, rp, col = 3, [0, 1, 2, 3], [1, 2, 0]
    if case == "selfloop":
        col = [0, 2, 0]
    elif case == "range":
        col = [1, 3, 0]
    elif case == "negative":
        col = [1, -1, 0]
    elif case == "monotone":
        rp = [0, 2, 1, 3]
    elif case == "rowend":
        rp = np.array([0, 1, 2, 2], np.int32)
        col = [1, 2]
        rp = np.ascontiguousarray(rp)
        h = ctypes.c_void_p()
        c = np.array(col, np.int32)
        st = mtlib.mt_graph_load_csr(n, 3, rp.ctypes.data, c.ctypes.data, None, ctypes.byref(h))
        assert st == 1
        return
    elif case == "n0":
        h = ctypes.c_void_p()
        rp0 = np.zeros(1, np.int32)
        st = mtlib.mt_graph_load_csr(0, 0, rp0.ctypes.data, rp0.ctypes.data, None,
                                     ctypes.byref(h))
        assert st == 1
        return
    assert _load(mtlib, n, rp, col) == 1  # MT_EINVAL


@pytest.mark.parametrize("n", [65536, 70000])
def test_too_many_vertices_unsupported(mtlib, n):
    """Vertex ids are 16 bits on the device: 65,535 vertices at most."""
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(1, np.int32)
    h = ctypes.c_void_p()
    assert mtlib.mt_graph_load_csr(n, 0, rp.ctypes.data, col.ctypes.data, None,
                                   ctypes.byref(h)) == 2


def test_null_handles_rejected(mtlib):
    assert mtlib.mt_count(None, None, None, None) == 1
    assert mtlib.mt_table_build(7, None, ctypes.byref(ctypes.c_void_p())) == 2
    assert mtlib.mt_table_build(2, None, ctypes.byref(ctypes.c_void_p())) == 2
    assert mtlib.mt_randomize(None, 1, 1, None, ctypes.byref(ctypes.c_void_p())) == 1
    assert mtlib.mt_batch_create(None, None, 1, 1, ctypes.byref(ctypes.c_void_p())) == 1


def test_header_compiles_as_plain_c_and_links(mtlib, tmp_path):
    """include/motifs.h is a C header: a C99 program using it compiles with
    warnings as errors, links against the library and runs its host-only calls
    (no GPU)."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    import subprocess
    from paper_1804_09741_gb300 import build as b
    libdir = b.BUILD
    exe = str(tmp_path / "host_calls")
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi", "host_calls.c"),
                           "-L", libdir, "-lmotifs", "-Wl,-rpath," + libdir, "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert "c abi host calls ok" in out.stdout
