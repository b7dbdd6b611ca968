"""The bounds-checked debug build (-DQCS_BOUNDS, libqcs_bounds.so) on small parity cases.

Every pair kernel of that build checks its shared-memory layout against the launch's
dynamic shared memory, the tile it takes from the work queue, the parity +1 count, each
snapshot index and the record it copies; a failed check raises QCS_ERR_BOUNDS in the
status word and skips the access.  The cases cover the tensor-core and ALU FP64 paths,
the two-warp group path (n > 16), the split precision, the adjoint and the local energy.
They run in a child process that loads the debug build through QCS_LIBRARY=bounds,
with QCS_LOG=3 so that the log lines of the calls and launches are checked as well."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

from paper_2506_22408_gb300 import _build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_build_runs_the_parity_cases_clean():
    _build.build(variant="bounds")
    env = dict(os.environ, QCS_LIBRARY="bounds", QCS_LOG="3")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"].endswith("libqcs_bounds.so")
    for name in ("tc", "alu", "alu_small", "group_n20"):
        assert out[name]["status"] == 0, (name, out[name])
        assert out[name]["pair_err_over_scale"] <= 1e-10, (name, out[name])
    assert out["split"]["status"] == 0 and out["split"]["pair_err_over_scale"] <= 2e-5
    assert out["grad"]["status"] == 0 and out["grad"]["rel_err"] <= 1e-9
    assert out["energy"]["status"] == 0 and out["energy"]["rel_err"] <= 1e-8
    # QCS_LOG=3: a line per entry-point call (level 2) and per launch (level 3)
    log = r.stderr
    assert "[qcs] qcs_overlap" in log and "path=fp64-tensor-core" in log and "path=fp64-alu" in log
    assert "[qcs] launched tc_pair_kernel" in log and "[qcs] launched split_pair_kernel" in log
