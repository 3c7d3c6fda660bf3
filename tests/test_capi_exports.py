"""The C-ABI library loads and exports every function include/mce.h
declares (no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mce.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mce_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1801_00202_gb300 as m
    m.build()
    return m.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mce_load_edges", "mce_load_bitset", "mce_enumerate", "mce_submit", "mce_poll",
                 "mce_enumerate_device", "mce_search", "mce_order", "mce_renumber"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    import paper_1801_00202_gb300 as m
    assert set(declared_functions()) <= set(m._SIGS)


def test_host_only_calls(lib):
    import paper_1801_00202_gb300 as m
    assert m.mce_strerror(m.MCE_EINVAL) == "invalid argument or graph"
    assert m.mce_strerror(m.MCE_OK) == "ok"
    # argument checks happen before any CUDA call
    assert m.mce_order(m.MCE_NMAX + 1, 200, 0, 0) == m.MCE_EINVAL
    assert m.mce_renumber(10, 0, 0, 0, 1, 0) == m.MCE_EINVAL
    assert m.mce_enumerate_device(10, 1, None, None, None, 0, None) == m.MCE_EINVAL


def test_loading_the_library_asks_for_32_hardware_queues():
    # a process that loads libmce before creating a CUDA context gets 32
    # stream queues for the served form unless it set its own value
    import subprocess
    import sys
    import paper_1801_00202_gb300 as m
    m.build()
    code = ("import ctypes; ctypes.CDLL(%r); libc = ctypes.CDLL(None); libc.getenv.restype = ctypes.c_char_p; "
            "v = libc.getenv(b'CUDA_DEVICE_MAX_CONNECTIONS'); print(v.decode() if v else None)" % m._LIB_PATH)
    env = {k: v for k, v in os.environ.items() if k != "CUDA_DEVICE_MAX_CONNECTIONS"}
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "32", r.stderr[-500:]
    env["CUDA_DEVICE_MAX_CONNECTIONS"] = "4"
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.stdout.strip() == "4"


def test_fault_sites_arm_and_disarm(lib):
    import paper_1801_00202_gb300 as m
    assert m.mce_fault_inject(0, 0, 1) == m.MCE_EINVAL
    assert m.mce_fault_inject(4, 0, 1) == m.MCE_EINVAL
    for site in (m.MCE_FAULT_ALLOC, m.MCE_FAULT_COPY, m.MCE_FAULT_ADMIT):
        assert m.mce_fault_inject(site, 3, 2) == m.MCE_OK
        assert m.mce_fault_inject(site, 0, 0) == m.MCE_OK
    assert m.mce_strerror(m.MCE_ECANCELED) == "cancelled"
    assert m.mce_strerror(m.MCE_EBUSY) == "already running"
