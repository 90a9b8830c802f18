"""The WO_CHECK variant of the library (kernels test the indices of their
global accesses, skip and record any outside their buffers): small valid
calls of every kernel family must leave every status at WO_OK and give
results bit-identical to the normal library's (the checks change no
arithmetic).  The variant runs in a child process (WO_LIB=check)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from paper_2412_09775_gb300.build import build
build(check=True)
from paper_2412_09775_gb300 import binding as B
assert B.wo_check_build()
import check_cases
out, codes = check_cases.run(B, torch, torch.device("cuda:0"))
np.savez({path!r}, codes=np.array([c[1:] for c in codes]), names=np.array([c[0] for c in codes]), **out)
"""


def test_check_build_is_clean_and_identical(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding as B
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import check_cases
    assert not B.wo_check_build()
    path = str(tmp_path / "check.npz")
    env = dict(os.environ, WO_LIB="check")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=path)],
                       env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(path)
    assert np.all(got["codes"] == 0), list(zip(got["names"], got["codes"]))
    want, codes = check_cases.run(B, torch, torch.device("cuda:0"))
    assert all(c[1] == 0 for c in codes), codes
    for k, v in want.items():
        assert np.array_equal(got[k], v), k
