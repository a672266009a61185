"""The index-checking build (every kernel compiled with -DMCG_CHECK: the
layout helpers test each index against its array, count a bad one and
redirect it inside the array).  One small case through every kernel family
(tests/_kernel_tour.py) must meet no out-of-range index, and give the regular
build's results (to the last bits where the arithmetic is deterministic;
the smearing backward sums with atomics)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOUR = os.path.join(ROOT, "tests", "_kernel_tour.py")


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, TOUR], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def _close(a, b, path=""):
    if isinstance(a, dict):
        for k in a:
            _close(a[k], b[k], path + "/" + k)
    elif isinstance(a, list):
        assert len(a) == len(b), path
        for i, (x, y) in enumerate(zip(a, b)):
            _close(x, y, f"{path}[{i}]")
    elif isinstance(a, float):
        tol = 1e-9 if path.endswith("smear_bwd") else 1e-12
        assert abs(a - b) <= tol * max(1.0, abs(a)), (path, a, b)
    else:
        assert a == b, (path, a, b)


def test_check_build_meets_no_bad_index_and_matches_the_regular_build():
    from paper_0807_0264_gb300 import build

    lib_check = build.build(check=True)
    regular = _run({})
    checked = _run({"MCG_LIBRARY": lib_check})
    assert regular["violations"] == -1
    assert checked["violations"] == 0
    _close(regular["results"], checked["results"])
    assert np.isfinite(regular["results"]["4x4x4x6"]["R_mixed_df"])
