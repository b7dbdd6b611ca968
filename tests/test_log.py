"""QCS_LOG on the host (no GPU): the library's log level comes from the environment,
read once per process; level 1 prints every error message to stderr with the prefix
"[qcs] ", level 0 (the default) prints nothing.  The error here is the failed context
creation of a machine without a GPU."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = ("import ctypes, sys; sys.path.insert(0, %r); from paper_2506_22408_gb300 import qcs; "
         "lib = qcs.load(); h = ctypes.c_void_p(); print(lib.qcs_create(ctypes.byref(h), 0))" % ROOT)


@pytest.mark.skipif(torch.cuda.is_available(), reason="needs a machine without a GPU (context creation fails)")
@pytest.mark.parametrize("level,expect", [("0", False), ("1", True), (None, False)])
def test_log_level_from_environment(level, expect):
    env = dict(os.environ)
    env.pop("QCS_LOG", None)
    env.pop("QCS_LIBRARY", None)
    if level is not None:
        env["QCS_LOG"] = level
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().splitlines()[-1] == "2"  # QCS_ERR_CUDA
    assert ("[qcs] qcs_create(device 0):" in r.stderr) == expect, r.stderr
