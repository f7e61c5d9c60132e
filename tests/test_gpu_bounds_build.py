"""The bounds-checked build (libsnap_bc.so, -DSNAP_BOUNDS_CHECK) on valid inputs, on the GPU: its
checked kernels (the 1-D tile kernels of the forward and adjoint, the heat-2 chains) give the
bits of the normal build and record no failure in the error word.  The checked library is
loaded in a child process (SNAP_BOUNDS_CHECK=1), since a process loads one of the two."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch

from paper_2607_00095_b300 import Problem, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = r"""
import sys, numpy as np, torch, ctypes as C
sys.path.insert(0, sys.argv[2])
from paper_2607_00095_b300 import Problem, synthetic, _abi
from tests import gpu_helpers as H
out = {}
uh, pr = synthetic.gen_1d(31, 40, 128, 30, "B")
p = Problem("B", 128, 30)
u, lam, st = p.project(H.to_dev(uh.reshape(40, -1)), H.to_dev(pr))
gb = synthetic.gen_gbar(32, (40, 30 * 128))
gh, gp = p.backward(H.to_dev(gb), u, lam, H.to_dev(pr), stats=st)
hu, hg = synthetic.gen_heat(33, 6, 40, 12)
q = Problem("F", 40, 12)
hu_, hl_, hs_ = q.project(H.to_dev(hu.reshape(6, -1)), H.to_dev(hg))
torch.cuda.synchronize()
for k, v in dict(u=u, lam=lam, gh=gh, gp=gp, hu=hu_, hl=hl_).items():
    out[k] = v.cpu().numpy()
w = C.c_ulonglong(1)
out["rc"] = np.array([_abi.lib().snap_bounds_error(C.byref(w), 1)])
out["word"] = np.array([w.value], dtype=np.uint64)
np.savez(sys.argv[1], **out)
"""


def _run(bounds):
    f = os.path.join(tempfile.mkdtemp(), "out.npz")
    env = dict(os.environ)
    env["SNAP_BOUNDS_CHECK"] = "1" if bounds else "0"
    subprocess.run([sys.executable, "-c", _RUN, f, ROOT], env=env, check=True, timeout=600)
    return dict(np.load(f))


def test_bounds_checked_build_matches_normal_build_and_records_nothing():
    if not os.path.exists(os.path.join(ROOT, "paper_2607_00095_b300", "libsnap_bc.so")):
        pytest.fail("libsnap_bc.so not built")
    bc = _run(True)
    nb = _run(False)
    assert int(bc["rc"][0]) == 0 and int(bc["word"][0]) == 0      # checked build: no failure
    assert int(nb["rc"][0]) == 2                                     # normal build: unsupported
    for k in ("u", "lam", "gh", "gp", "hu", "hl"):
        np.testing.assert_array_equal(bc[k], nb[k])
