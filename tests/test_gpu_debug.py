"""The debug build's safety net (libpr_debug.so, -DPR_DEBUG).

compute-sanitizer is not available on every machine this library runs on, so
the debug build checks every index its kernels load from a graph array and,
after every round, the mass balance and the residual identity of Eq. 4 on the
device.  This test runs tests/debug_checks.py in its own process with
PR_LIBRARY=debug: clean solves of every algorithm, precision and delivery mode
on small graphs must pass every check and match the oracle, and a check forced
to fail at each site (a test hook that halves a bound or fails an invariant
outright, so no invalid access happens) must turn the solve into PR_ECHECK.
The bounded waits of graph creation's radix sort are made to give up at once:
the creation must return PR_ECUDA and the next one must work.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_checks_hold_and_fire():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, PR_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_checks.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["solves"] > 150
    assert res["clean"]["fails"] == 0 and res["clean"]["checks"] > 500
    assert sorted(int(k) for k in res["forced"]) == [1, 2, 3, 4, 16, 17]
    assert res["sort_wait"]  # graph creation's bounded waits fail cleanly
