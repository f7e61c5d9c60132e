"""Back-to-back calls on one stream: the 1-D prepare kernel starts as a programmatic dependent
of whatever kernel precedes it and waits for that kernel before its first access, and the tile
kernel that follows it reads u_hat before its own wait.  A projection whose u_hat is the
previous projection's output (written by kernels still in flight when the call is enqueued),
mixed with an adjoint, a family E and a 2-D call, must give the bits of the same calls with a
device synchronisation between every two of them, eagerly and inside one CUDA graph."""
import numpy as np
import pytest
import torch

from paper_2607_00095_b300 import Problem, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _inputs():
    B, nx, nt = 24, 64, 40
    uh, pr = synthetic.gen_1d(91, B, nx, nt, "B")
    gbar = synthetic.gen_gbar(92, (B, nt * nx))
    wh, pw = synthetic.gen_2d(93, 4, 16, 3)
    fh, fp = synthetic.gen_burgers_flux(94, 8, 33, 17)
    return dict(p1=Problem("B", nx, nt), pe=Problem("E", 33, 17, n_flux=5), p2=Problem("C", 16, 3),
                uh=H.to_dev(uh.reshape(B, -1)), pr=H.to_dev(pr), gbar=H.to_dev(gbar),
                wh=H.to_dev(wh.reshape(4, -1)), pw=H.to_dev(pw),
                fh=H.to_dev(fh.reshape(8, -1)), fp=H.to_dev(fp))


def _sequence(d, sync):
    """project; project again from the first output; adjoint of the second; family E; 2-D;
    a third 1-D projection from the second output.  Returns every result tensor."""
    def s():
        if sync:
            torch.cuda.synchronize()
    out = []
    u1, l1, s1 = d["p1"].project(d["uh"], d["pr"])
    s()
    u2, l2, s2 = d["p1"].project(u1, d["pr"])
    s()
    gh, gp = d["p1"].backward(d["gbar"], u2, l2, d["pr"], stats=s2)
    s()
    ue, le, se = d["pe"].project(d["fh"], d["fp"])
    s()
    uw, lw, sw = d["p2"].project(d["wh"], d["pw"])
    s()
    u3, l3, s3 = d["p1"].project(u2, d["pr"])
    s()
    out += [u1, l1, s1, u2, l2, s2, gh, gp, ue, le, se, uw, lw, sw, u3, l3, s3]
    return out


def test_chained_calls_match_synchronised_calls_bitwise():
    d = _inputs()
    ref = [t.clone() for t in _sequence(d, sync=True)]
    torch.cuda.synchronize()
    for _ in range(3):
        got = _sequence(d, sync=False)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    # the same sequence captured in one graph (outputs allocated by the capture's pool)
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        _sequence(d, sync=False)             # warm-up of the side stream
        with torch.cuda.graph(g, stream=cap):
            got = _sequence(d, sync=False)
    torch.cuda.current_stream().wait_stream(cap)
    for _ in range(3):
        for t in got:
            if t.dtype == torch.float64:
                t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    # the chained outputs are projections of what they were given: the second and third
    # projections of an already projected field return it (up to the solver tolerance)
    u1, u2, u3 = ref[0].cpu().numpy(), ref[3].cpu().numpy(), ref[14].cpu().numpy()
    np.testing.assert_allclose(u2, u1, rtol=0, atol=1e-9 * np.abs(u1).max())
    np.testing.assert_allclose(u3, u2, rtol=0, atol=1e-9 * np.abs(u1).max())
