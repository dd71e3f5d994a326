"""The bounds-checked build (library compiled with MTPT_CHECKED: every
kernel verifies its index invariants at run time and records violations in a
device word) runs a battery of workloads -- both forms in 2-d and 3-d,
repeated host loads, a batch, boxes far from the origin, the adjoint, the
no-allocation step -- in a child process.  No check may fire, and every
result must equal the normal build's bit for bit (the checks change no
arithmetic).  This stands in for a memory checker, which this pool does not
offer."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2204_03756_gb300 import mtpt

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

pytestmark = pytest.mark.gpu


def test_checked_build_fires_no_check_and_matches_the_normal_build(tmp_path):
    from paper_2204_03756_gb300 import build
    build.build()
    assert os.path.exists(build.LIB_CHECKED_PATH)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, MTPT_LIBRARY="checked",
               PYTHONPATH=os.pathsep.join([HERE, ROOT, os.environ.get("PYTHONPATH", "")]))
    proc = subprocess.run([sys.executable, os.path.join(HERE, "checked_battery.py"), str(out)],
                          env=env, capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stdout[-2000:] + proc.stderr[-4000:]
    got = dict(np.load(out))
    assert int(got.pop("check_word")[0]) == 0
    sys.path.insert(0, HERE)
    import checked_battery
    want = checked_battery.run()
    assert set(got) == set(want)
    for k in sorted(want):
        assert np.array_equal(got[k], want[k]), k

