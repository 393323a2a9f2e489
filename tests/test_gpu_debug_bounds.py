"""The bounds-checked debug build (include/lisa_debug.h): tiny likelihood and gradient cases (64
bins and 3 states, diagonal and dense covariance, both precisions; prior draws with close knots
for the compensated and fallback passes) run through liblisa_psd_debug.so in a child process.
Every checked tile, bin, knot, record, moment-slot and list index stays in range, the results
meet the parity bounds of the release tests, and the self-test shows that the checks fire."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def report():
    from paper_2507_06300_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, LISA_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_bounds_run.py")], env=env,
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    print(json.dumps(rep, indent=1))
    return rep


def test_checks_are_compiled_in(report):
    assert report["enabled"] is True


def test_no_index_leaves_its_range(report):
    b = report["after_cases"]
    assert b["count"] == 0, b


@pytest.mark.parametrize("case", ["tiny64", "prior_close_knots"])
def test_debug_build_meets_the_parity_bounds(report, case):
    c = report["cases"][case]
    assert c["states_ok"] >= 1
    assert c["status_equal"]
    assert c["fp64_rel"] <= 1e-12
    assert c["fp32_frac_of_bound"] <= 1.0, c
    for k in ("grad64", "grad32"):
        assert c[k + "_frac_of_bound"] <= 1.0, (k, c[k + "_worst"])


def test_debug_build_dense_covariance(report):
    c = report["cases"]["full64"]
    assert c["states_ok"] >= 1
    assert c["fp64_rel"] <= 1e-12
    assert c["fp32_frac_of_bound"] <= 1.0


def test_selftest_violations_are_recorded(report):
    b = report["after_selftest"]
    assert b["count"] == 32
    assert 5 <= b["first_index"] <= 36
    assert b["first_file"].endswith("lisa_data.cu") and b["first_line"] > 0
