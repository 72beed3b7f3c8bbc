"""The index-checked build (-DWB_CHECKED): a probe shows the checks fire, and
every scenario of checked_scenarios.py forms no out-of-range zone index.
Runs in a child process that loads the checked library (WOMBAT_CHECKED=1)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_finds_no_bad_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, WOMBAT_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_scenarios.py")], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert res.pop("selftest") is True
    assert len(res) >= 12
    assert all(v == 0 for v in res.values()), res
