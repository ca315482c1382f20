"""The range-checked library (PDFGPU_CHECKED=1: every table index computed
on the device is tested before use and a bad one sets PDF_S_BOUNDS) runs
every form of the hot path, on all four extrapolation options and on 12
randomly shaped grids, without a single out-of-range index, and gives bit
for bit the outputs of the release library.  Both run in child processes: the library is chosen at import."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(checked):
    env = dict(os.environ, PDFGPU_CHECKED="1" if checked else "0", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads([line for line in r.stdout.splitlines() if line.startswith("{")][-1])


def test_checked_library_finds_no_bad_index_and_changes_nothing():
    chk, rel = _run(True), _run(False)
    assert chk["library"].endswith(os.path.join("_build_checked", "libpdfgpu.so"))
    assert rel["library"].endswith(os.path.join("_build", "libpdfgpu.so"))
    for extrap in ("linear", "freeze", "error", "continuation"):
        assert not chk[extrap]["status"] & 4, extrap                 # PDF_S_BOUNDS never set
        assert chk[extrap]["digest"] == rel[extrap]["digest"], extrap
        assert chk[extrap]["status"] == rel[extrap]["status"], extrap
    for seed in range(12):                                          # randomly shaped grids
        k = f"random{seed}"
        assert not chk[k]["status"] & 4, k
        assert chk[k]["digest"] == rel[k]["digest"] and chk[k]["status"] == rel[k]["status"], k
