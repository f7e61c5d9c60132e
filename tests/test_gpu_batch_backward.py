"""GPU tests of the uneven-batch adjoint (snap_batch_project_backward): one persistent launch
over instances of different families and sizes against the per-group snap_project_backward
launches (to rounding: the two kernels are compiled separately), bit-for-bit identical results
under every schedule and through the owned CUDA graph, the oracle's dense adjoint at its own
solution on the instances of a small mix, and sampled instances of the full uneven mix."""
import numpy as np
import pytest
import torch

from oracle import problems, solve
from paper_2607_00095_b300 import Batch, Problem, decode_stats, options, synthetic
from tests import gpu_helpers as H
from tests.test_gpu_batch import SCHEDULES, _fill, _small_mix

pytestmark = pytest.mark.gpu


def _fill_gbar(gbufs, gbar):
    for pi, g in gbufs.items():
        for j, i in enumerate(g["ids"]):
            g["gu"][j].copy_(torch.as_tensor(gbar[i]))


def _gbar(data, seed):
    return [synthetic.gen_gbar(seed + i, d[0].shape) for i, d in enumerate(data)]


def _bwd_outputs(gbufs):
    return {pi: (g["gh"].cpu().numpy().copy(), g["gp"].cpu().numpy().copy())
            for pi, g in gbufs.items()}


def _assert_same(a, b):
    for pi in a:
        np.testing.assert_array_equal(a[pi][0], b[pi][0])
        np.testing.assert_array_equal(a[pi][1], b[pi][1])


def _assert_close(a, b, rtol_h=1e-12, rtol_p=1e-9):
    """The same adjoint arithmetic in two separately compiled kernels, to rounding."""
    for pi in a:
        for x, y, rt in ((a[pi][0], b[pi][0], rtol_h), (a[pi][1], b[pi][1], rtol_p)):
            for s in range(x.shape[0]):
                den = max(np.abs(y[s]).max(), 1.0)
                assert np.abs(x[s] - y[s]).max() / den <= rt, (pi, s)


def _setup(seed, opts=None):
    specs, probs, inst, data = _small_mix(seed)
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    b.project(opts=opts)
    torch.cuda.synchronize()
    for pi, g in bufs.items():
        assert (decode_stats(g["st"].cpu().numpy())["status"] == 0).all(), specs[pi]
    gbufs = b.alloc_backward("cuda:0")
    gbar = _gbar(data, 5000 + seed)
    _fill_gbar(gbufs, gbar)
    return specs, probs, b, bufs, gbufs, data, gbar


def test_batch_backward_matches_per_group_every_schedule():
    specs, probs, b, bufs, gbufs, data, gbar = _setup(7)
    b.backward_grouped()
    torch.cuda.synchronize()
    ref = _bwd_outputs(gbufs)
    first = None
    for sch in SCHEDULES:
        b.set_schedule(**sch)
        for g in gbufs.values():
            g["gh"].fill_(np.nan)
            g["gp"].fill_(np.nan)
        b.backward()
        torch.cuda.synchronize()
        out = _bwd_outputs(gbufs)
        if first is None:
            first = out
            _assert_close(out, ref)
        else:
            _assert_same(out, first)
    # the owned graph replays the same launch
    b.capture_graph_backward()
    for g in gbufs.values():
        g["gh"].zero_()
        g["gp"].zero_()
    b.launch_graph_backward()
    torch.cuda.synchronize()
    _assert_same(_bwd_outputs(gbufs), out)


def test_batch_backward_against_oracle():
    """Every instance of a small mix (families A, B, C; nt below, at and above 32) against the
    oracle's dense adjoint at the oracle's own solution of the same inputs."""
    opts = options(tol_kkt=1e-13)
    specs, probs, b, bufs, gbufs, data, gbar = _setup(8, opts)
    b.backward()
    torch.cuda.synchronize()
    out = _bwd_outputs(gbufs)
    for pi, g in gbufs.items():
        f, nx, nt = specs[pi]
        ids = g["ids"]
        uh = np.stack([data[i][0] for i in ids])
        pr = np.stack([data[i][1] for i in ids])
        gb = np.stack([gbar[i] for i in ids])
        if f == "C":
            S = problems.structure_2d(nx, nt)
            ue, le, so = solve.project(S, problems.rhs_2d(nx, nt, pr), uh, tol_kkt=1e-13)
            assert (so["status"] == 0).all()
            a, bl = solve.adjoint(S, ue, le, gb)
            gpo = problems.grad_params_2d(nx, nt, pr, bl)
        else:
            a, gpo = H.oracle_adjoint_1d(f, nx, nt, pr, uh, gb, tol_kkt=1e-13)
        H.assert_adjoint_close(out[pi][0], a)
        H.assert_adjoint_close(out[pi][1], gpo)


def test_batch_backward_without_params_and_bad_samples():
    """No parameter gradients bound: dL/du_hat only.  A sample whose forward failed gets NaN
    gradients, the others are unaffected."""
    specs, probs, b, bufs, gbufs, data, gbar = _setup(9)
    b.backward()
    torch.cuda.synchronize()
    ref = _bwd_outputs(gbufs)
    # rebind without parameter gradients
    b.bind_backward(_rows(gbufs, "gu", b.n_inst), _rows(gbufs, "gh", b.n_inst), None)
    for g in gbufs.values():
        g["gh"].fill_(np.nan)
        g["gp"].fill_(-1.0)
    b.backward()
    torch.cuda.synchronize()
    for pi, g in gbufs.items():
        np.testing.assert_array_equal(g["gh"].cpu().numpy(), ref[pi][0])
        assert (g["gp"].cpu().numpy() == -1.0).all()
    # mark one instance of a 1-D and one of a 2-D group as failed in the forward statistics
    b.bind_backward(_rows(gbufs, "gu", b.n_inst), _rows(gbufs, "gh", b.n_inst),
                    _rows(gbufs, "gp", b.n_inst))
    pb = next(pi for pi in bufs if specs[pi][0] == "B")
    pc = next(pi for pi in bufs if specs[pi][0] == "C")
    marked = [(pb, 0), (pc, 0)]
    for pi, j in marked:
        bufs[pi]["st"][j, 8:12] = torch.tensor(list((2).to_bytes(4, "little")), dtype=torch.uint8)
    b.backward()
    torch.cuda.synchronize()
    for pi, g in gbufs.items():
        gh, gp = g["gh"].cpu().numpy(), g["gp"].cpu().numpy()
        for j in range(gh.shape[0]):
            if (pi, j) in marked:
                assert np.isnan(gh[j]).all() and np.isnan(gp[j]).all()
            else:
                np.testing.assert_array_equal(gh[j], ref[pi][0][j])
                np.testing.assert_array_equal(gp[j], ref[pi][1][j])


def _rows(gbufs, key, n):
    per = [None] * n
    for g in gbufs.values():
        for j, i in enumerate(g["ids"]):
            per[i] = g[key][j]
    return per


def test_uneven_full_size_backward():
    """The uneven mix (1024 instances, seed 1004): persistent adjoint against the per-group
    launches (to rounding), its graph bit for bit, and one sampled 1-D instance per group
    against the oracle's dense adjoint."""
    mix = synthetic.gen_uneven(**synthetic.WORKLOADS["uneven"])
    keys = sorted({(m["family"], m["nx"], m["nt"]) for m in mix})
    probs = [Problem(f, nx, nt) for f, nx, nt in keys]
    inst = np.array([keys.index((m["family"], m["nx"], m["nt"])) for m in mix], np.int32)
    data = [(m["u_hat"].reshape(-1), m["params"]) for m in mix]
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    b.project()
    torch.cuda.synchronize()
    gbufs = b.alloc_backward("cuda:0")
    gbar = _gbar(data, 9000)
    _fill_gbar(gbufs, gbar)
    b.backward()
    torch.cuda.synchronize()
    out = _bwd_outputs(gbufs)
    b.capture_graph_backward()
    for g in gbufs.values():
        g["gh"].zero_()
    b.launch_graph_backward()
    torch.cuda.synchronize()
    _assert_same(_bwd_outputs(gbufs), out)
    b.backward_grouped()
    torch.cuda.synchronize()
    ref = _bwd_outputs(gbufs)
    ok = {pi: decode_stats(g["st"].cpu().numpy())["status"] == 0 for pi, g in bufs.items()}
    for pi in out:
        sel = ok[pi]
        _assert_close({pi: (out[pi][0][sel], out[pi][1][sel])},
                      {pi: (ref[pi][0][sel], ref[pi][1][sel])})
    rng = np.random.default_rng(13)
    for pi, g in gbufs.items():
        f, nx, nt = keys[pi]
        if f == "C":
            continue
        cand = np.nonzero(ok[pi])[0]
        j = int(cand[rng.integers(0, len(cand))])
        i = g["ids"][j]
        a, gpo = H.oracle_adjoint_1d(f, nx, nt, data[i][1][None], data[i][0][None], gbar[i][None])
        H.assert_adjoint_close(out[pi][0][j:j + 1], a)
        H.assert_adjoint_close(out[pi][1][j:j + 1], gpo)
