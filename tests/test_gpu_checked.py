"""The bounds-checked build (TQS_CHECKED): the kernels run with every state,
tile and output index range-checked.  The same workload (tests/checked_workload.py)
runs in child processes against the normal and the checked library; the
checked run must record no out-of-range access and give bitwise the same
outputs."""
import json
import os
import subprocess
import sys

import pytest

from paper_2305_14398_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_with(lib):
    env = dict(os.environ, TQS_LIB=lib, PYTHONPATH=ROOT + os.pathsep + HERE)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py")], env=env,
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_no_violations_same_outputs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    checked = build.build(checked=True)
    normal = build.build()
    a = run_with(normal)
    b = run_with(checked)
    assert a["violations"] == 0
    assert b["violations"] == 0
    assert a["digest"] == b["digest"]
