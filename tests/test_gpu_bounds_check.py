"""The bounds-checked build of the library (-DKH_BOUNDS_CHECK), standing in
for a device memory checker: its instrumented kernels check every work
item's cells against the allocation and count and skip a violation instead of
touching memory out of bounds. Stepping a set of small problems with it must
count no violation and give results bit-identical to the release build's
(the checks only skip work on a violation)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(tmp_path, lib, tag):
    out = str(tmp_path / f"{tag}.npz")
    env = dict(os.environ, KH_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(out)


def test_bounds_checked_build_counts_nothing_and_matches_release(tmp_path):
    from paper_2408_01361_gb300 import build
    rel = build.build()
    chk = build.build(bounds=True)
    a = _run(tmp_path, chk, "bounds")
    b = _run(tmp_path, rel, "release")
    names = sorted(k[: -len("_nbounds")] for k in a.files if k.endswith("_nbounds"))
    assert len(names) == 7
    for n in names:
        assert int(a[n + "_nbounds"]) == 0, (n, int(a[n + "_nbounds"]))
        assert int(b[n + "_nbounds"]) == 0
        for s in ("_U", "_P"):
            assert np.array_equal(a[n + s], b[n + s]), (n, s)
