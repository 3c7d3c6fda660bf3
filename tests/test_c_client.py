"""include/mce.h is a complete C interface: a plain C program
(tests/c_client/mce_client.c) compiles against it and links against
libmce.so alone (no Python, no PyTorch).  On a GPU the program loads
graphs, enumerates each alone, through the served form and as one batch,
and checks that all three agree; loading the library gave it 32 hardware
stream queues without any setting of its own."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile(tmp_path):
    import paper_1801_00202_gb300 as m
    m.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "mce_client")
    lib = m._LIB_PATH
    cmd = [cc, "-O2", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client", "mce_client.c"), lib, "-Wl,-rpath," + os.path.dirname(lib),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_and_links_against_the_header_and_library(tmp_path):
    _compile(tmp_path)


@pytest.mark.gpu
def test_c_program_forms_agree(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _compile(tmp_path)
    env = {k: v for k, v in os.environ.items() if k != "CUDA_DEVICE_MAX_CONNECTIONS"}
    r = subprocess.run([exe, "48"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    assert sum(1 for x in lines if x.endswith(" agree")) == 48
    served = [x for x in lines if x.startswith("served ")]
    assert served and served[0].split()[-1] == "32"
