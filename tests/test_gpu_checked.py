"""The checked build (device-side bounds checks, the stand-in for a memory checker):
a fixed workload over every kernel family runs in a child process against the
library compiled with -DMVP_CHECK_BOUNDS. No check may fire (every sync would raise
MVP_ERR_DEVICE), and the results must be those of the release library."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import checked_workload  # noqa: E402


def test_checked_build_is_silent_and_agrees(tmp_path):
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, MVP_CHECK_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py"), path], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    chk = dict(np.load(path))
    ref = checked_workload.run()
    assert int(chk["checked"][0]) == 1 and int(ref["checked"][0]) == 0
    assert set(chk) == set(ref)
    for k in sorted(ref):
        if k == "checked":
            continue
        a, b = ref[k], chk[k]
        assert a.shape == b.shape, k
        if "/g_" in k:  # gradients: float reductions in arrival order
            scale = max(float(np.abs(a).max()), 1e-30)
            assert float(np.abs(a - b).max()) <= 1e-5 * scale, k
        elif a.dtype.kind == "f":
            assert float(np.abs(a - b).max()) <= 1e-6, k
        else:
            np.testing.assert_array_equal(a, b, err_msg=k)
    assert int(chk["serve_status"][0]) == 0
    assert all(int(chk[k][0]) == 0 for k in chk if k.endswith("static_status"))
