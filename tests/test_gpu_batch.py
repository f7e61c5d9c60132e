"""GPU tests of the uneven batch (one persistent launch over instances of different grid sizes
and families): agreement with snap_project per group, bit-for-bit identical results under every
schedule, the oracle on sampled instances, the uneven mix at full size, timing stamps, the owned
CUDA graph, the autotuner and the error paths.

The batch kernel runs the same device code per slice / frame as snap_project, but the two
kernels are compiled separately and the compiler fuses multiplies and adds differently in them,
so batch and per-group results agree to rounding (u to 1e-12 relative per instance, lambda to
1e-9 per constraint type), not bit for bit.  Between schedules of the batch kernel itself they
agree bit for bit: a slice's arithmetic does not depend on the lane or warp that runs it."""
import itertools

import numpy as np
import pytest
import torch

from oracle import closed_form, problems, solve
from paper_2607_00095_b300 import Batch, Problem, _abi, decode_stats, options, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

SCHEDULES = [dict(ctas_per_sm=c, order=o, pack_1d=p, sort_1d=s)
             for c, o, p, s in itertools.product((1, 2), (0, 1), (0, 1), (0, 1))]


def _small_mix(seed):
    """Problems of several shapes (families A, B, C; nt below, at and above 32) and a seeded
    instance list over them, with inputs."""
    specs = [("B", 16, 3), ("B", 24, 40), ("A", 32, 5), ("B", 64, 33), ("C", 8, 2), ("C", 16, 3),
             ("B", 6, 2)]
    probs = [Problem(f, nx, nt) for f, nx, nt in specs]
    rng = np.random.default_rng(seed)
    inst = rng.integers(0, len(specs), size=41).astype(np.int32)
    inst[: len(specs)] = np.arange(len(specs))     # every problem present
    # enough nt = 2 instances that one 32-slice tile spans 17 of them
    inst = np.concatenate([inst, np.full(20, len(specs) - 1, np.int32)])
    data = []
    for i, pi in enumerate(inst):
        f, nx, nt = specs[pi]
        if f == "C":
            wh, pr = synthetic.gen_2d(seed * 1000 + i, 1, nx, nt, kmax=max(1, min(8, nx // 2 - 1)))
        else:
            wh, pr = synthetic.gen_1d(seed * 1000 + i, 1, nx, nt, f)
        data.append((wh.reshape(-1), pr[0]))
    return specs, probs, inst, data


def _fill(b, bufs, data):
    for pi, g in bufs.items():
        for j, i in enumerate(g["ids"]):
            g["uh"][j].copy_(torch.as_tensor(data[i][0]))
            g["pr"][j].copy_(torch.as_tensor(data[i][1]))


def _outputs(bufs):
    return {pi: (g["u"].cpu().numpy().copy(), g["lam"].cpu().numpy().copy(),
                 g["st"].cpu().numpy().copy()) for pi, g in bufs.items()}


def _reference(probs, bufs):
    """snap_project on each group's contiguous block."""
    out = {}
    for pi, g in bufs.items():
        u, lam, st = probs[pi].project(g["uh"], g["pr"])
        torch.cuda.synchronize()
        out[pi] = (u.cpu().numpy(), lam.cpu().numpy(), st.cpu().numpy())
    return out


def _assert_same(a, b):
    """Bit-for-bit equality of u, lambda and the statistics."""
    for pi in a:
        np.testing.assert_array_equal(a[pi][0], b[pi][0])
        np.testing.assert_array_equal(a[pi][1], b[pi][1])
        np.testing.assert_array_equal(a[pi][2], b[pi][2])


def _assert_close(a, b, probs):
    """Agreement to rounding of two runs of the same arithmetic in different kernels."""
    for pi in a:
        sa, sb = decode_stats(a[pi][2]), decode_stats(b[pi][2])
        np.testing.assert_array_equal(sa["status"], sb["status"])
        ok = sa["status"] == 0
        assert (sa["h_inf"][ok] <= H.H_TOL).all() and (sb["h_inf"][ok] <= H.H_TOL).all()
        # converged instances: the same point to rounding (an instance stopped at MAXITER sits
        # at an iterate that rounding moves)
        ua, ub = a[pi][0][ok], b[pi][0][ok]
        for s in range(ua.shape[0]):
            den = max(np.abs(ub[s]).max(), 1e-300)
            assert np.abs(ua[s] - ub[s]).max() / den <= 1e-12, (pi, s)
        p = probs[pi]
        S = (problems.structure_2d(p.nx, p.nt) if p.family == "C"
             else problems.structure_1d(p.family, p.nx, p.nt))
        H.assert_lam_close(S, a[pi][1][ok], b[pi][1][ok], rtol=1e-9)


def test_batch_matches_per_group_project_every_schedule():
    specs, probs, inst, data = _small_mix(7)
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    ref = _reference(probs, bufs)
    for pi in ref:
        st = decode_stats(ref[pi][2])
        assert (st["status"] == 0).all(), specs[pi]
    first = None
    for sch in SCHEDULES:
        b.set_schedule(**sch)
        for g in bufs.values():
            g["u"].fill_(np.nan)
            g["lam"].fill_(np.nan)
            g["st"].fill_(255)
        b.project()
        torch.cuda.synchronize()
        out = _outputs(bufs)
        if first is None:
            first = out
            _assert_close(out, ref, probs)
        else:
            _assert_same(out, first)
    # the grouped baseline is plain snap_project per group
    b.project_grouped()
    torch.cuda.synchronize()
    _assert_same(_outputs(bufs), ref)


def test_batch_tile_shapes():
    """Slices per 1-D item (16, 32, 64) do not change a slice's arithmetic: the same bits.
    Lanes per slice (2, 4, 8, for all groups or per group) sum the moments in a different
    order: the same point to rounding."""
    specs, probs, inst, data = _small_mix(10)
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    b.set_schedule(tile_1d=32, lanes_1d=4)
    b.project()
    torch.cuda.synchronize()
    ref = _outputs(bufs)
    for tile in (16, 64):
        b.set_schedule(tile_1d=tile)
        b.project()
        torch.cuda.synchronize()
        _assert_same(_outputs(bufs), ref)
    b.set_schedule(tile_1d=32)
    for lanes in (2, 8):
        b.set_schedule(lanes_1d=lanes)
        assert all(l == lanes for k, l in enumerate(b.group_lanes()) if specs[k][0] != "C")
        b.project()
        torch.cuda.synchronize()
        _assert_close(_outputs(bufs), ref, probs)
    mixed = [(2, 4, 8)[k % 3] if specs[k][0] != "C" else 0 for k in range(len(specs))]
    b.set_group_lanes(mixed)
    b.set_schedule(lanes_1d=0)
    assert b.group_lanes() == mixed
    b.project()
    torch.cuda.synchronize()
    _assert_close(_outputs(bufs), ref, probs)
    with pytest.raises(_abi.SnapError):
        b.set_schedule(tile_1d=48)
    with pytest.raises(_abi.SnapError):
        b.set_group_lanes([3] * len(specs))


def test_batch_against_oracle():
    specs, probs, inst, data = _small_mix(8)
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    b.project()
    torch.cuda.synchronize()
    out = _outputs(bufs)
    for pi, g in bufs.items():
        f, nx, nt = specs[pi]
        ids = g["ids"]
        uh = np.stack([data[i][0] for i in ids])
        pr = np.stack([data[i][1] for i in ids])
        u, lam, st = out[pi]
        st = decode_stats(st)
        assert (st["status"] == 0).all() and st["h_inf"].max() <= H.H_TOL
        if f == "C":
            S = problems.structure_2d(nx, nt)
            ue, le, so = solve.project(S, problems.rhs_2d(nx, nt, pr), uh)
        else:
            ue, le, so, S, _ = solve.project_1d(f, nx, nt, pr, uh)
        assert (so["status"] == 0).all()
        H.assert_u_close(u, ue)
        H.assert_lam_close(S, lam, le)


def test_uneven_full_size():
    """The uneven mix (1024 instances, seed 1004): 1-D family B on nx in {64..256}, nt in
    {50, 100, 200}; 2-D at 32 x 32 x 8.  Persistent launch == per-group launches bit for bit;
    every instance converged; sampled instances against the oracle."""
    mix = synthetic.gen_uneven(**synthetic.WORKLOADS["uneven"])
    keys = sorted({(m["family"], m["nx"], m["nt"]) for m in mix})
    probs = [Problem(f, nx, nt) for f, nx, nt in keys]
    inst = np.array([keys.index((m["family"], m["nx"], m["nt"])) for m in mix], np.int32)
    data = [(m["u_hat"].reshape(-1), m["params"]) for m in mix]
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    t = torch.zeros(len(mix), 2, dtype=torch.int64, device="cuda:0")
    b.project(t_ns=t)
    torch.cuda.synchronize()
    out = _outputs(bufs)
    ref = _reference(probs, bufs)
    _assert_close(out, ref, probs)
    b.project_grouped()
    torch.cuda.synchronize()
    _assert_same(_outputs(bufs), ref)
    tt = t.cpu().numpy()
    assert (tt[:, 0] > 0).all() and (tt[:, 1] >= tt[:, 0]).all()
    rng = np.random.default_rng(11)
    n_bad = 0
    for pi, g in bufs.items():
        st = decode_stats(out[pi][2])
        f, nx, nt = keys[pi]
        ok = st["status"] == 0
        assert (st["h_inf"][ok] <= H.H_TOL).all(), keys[pi]
        for j in np.nonzero(~ok)[0]:
            # a slice the method itself does not solve under the globalisation used: the oracle
            # reports the same outcome (one family-B instance of this seed stalls at MAXITER)
            n_bad += 1
            i = g["ids"][j]
            assert f != "C"
            _, _, so, _, _ = solve.project_1d(f, nx, nt, data[i][1][None], data[i][0][None])
            assert so["status"][0] == st["status"][j] == 1, (keys[pi], i)
        j = int(rng.integers(0, len(g["ids"])))
        i = g["ids"][j]
        uh, pr = data[i]
        if f == "C":
            wc, lc = closed_form.project_2d(uh.reshape(1, nt, 2, nx, nx), pr[None])
            H.assert_u_close(out[pi][0][j:j + 1], wc.reshape(1, -1))
            H.assert_lam_close(problems.structure_2d(nx, nt), out[pi][1][j:j + 1], lc)
        else:
            if not ok[j]:
                continue
            ue, le, so, S, _ = solve.project_1d(f, nx, nt, pr[None], uh[None])
            assert (so["status"] == 0).all()
            H.assert_u_close(out[pi][0][j:j + 1], ue)
            H.assert_lam_close(S, out[pi][1][j:j + 1], le)
    assert n_bad <= 2


def test_graph_autotune_and_rebind():
    specs, probs, inst, data = _small_mix(9)
    b = Batch(probs, inst)
    bufs = b.alloc("cuda:0")
    _fill(b, bufs, data)
    sch, ms = b.autotune(reps=2)
    base = {k: sch[k] for k in ("ctas_per_sm", "order", "pack_1d", "sort_1d")}
    assert base in SCHEDULES and ms > 0
    assert sch["tile_1d"] in (16, 32, 64) and sch["lanes_1d"] == 0
    assert b.schedule() == sch
    lanes = b.group_lanes()
    assert all((l in (2, 4, 8)) if specs[k][0] != "C" else l == 0 for k, l in enumerate(lanes))
    b.project()
    torch.cuda.synchronize()
    ref = _outputs(bufs)
    b.capture_graph()
    for g in bufs.values():
        g["u"].zero_()
    b.launch_graph()
    torch.cuda.synchronize()
    _assert_same(_outputs(bufs), ref)
    # rebind to fresh buffers (same inputs): the captured graph follows the pointer table
    bufs2 = b.alloc("cuda:0")
    _fill(b, bufs2, data)
    b.launch_graph()
    torch.cuda.synchronize()
    _assert_same(_outputs(bufs2), ref)
    info = b.info()
    assert info["groups"] == len(specs) and info["frames_2d"] > 0 and info["tiles_1d"] > 0


def test_batch_errors():
    p1 = Problem("B", 16, 3)
    p2 = Problem("C", 8, 2)
    b = Batch([p1, p2], [0, 1, 0])
    with pytest.raises(_abi.SnapError) as ei:
        b.project()                              # not bound yet
    assert ei.value.code == 6
    bufs = b.alloc("cuda:0")
    with pytest.raises(_abi.SnapError) as ei:
        b.set_schedule(ctas_per_sm=3)
    assert ei.value.code == 1
    # workspace too small
    ws = torch.empty(16, dtype=torch.uint8, device="cuda:0")
    import ctypes as C
    with pytest.raises(_abi.SnapError) as ei:
        _abi.check(_abi.lib().snap_batch_project(b._h, C.byref(options()), None,
                                                 C.c_void_p(ws.data_ptr()), 16, None))
    assert ei.value.code == 5
    # non-contiguous group: the grouped baseline refuses, the persistent launch works
    u = [torch.zeros(p1.n_vars + 2, dtype=torch.float64, device="cuda:0")[2:] for _ in range(3)]
    uh = [bufs[0]["uh"][0], bufs[1]["uh"][0], bufs[0]["uh"][1]]
    pr = [bufs[0]["pr"][0], bufs[1]["pr"][0], bufs[0]["pr"][1]]
    lam = [bufs[0]["lam"][0], bufs[1]["lam"][0], bufs[0]["lam"][1]]
    st = [bufs[0]["st"][0], bufs[1]["st"][0], bufs[0]["st"][1]]
    outs = [u[0], bufs[1]["u"][0], u[2]]
    b.bind(uh, pr, outs, lam, st)
    with pytest.raises(_abi.SnapError) as ei:
        b.project_grouped()
    assert ei.value.code == 2
    # 1-D outputs must be 16-byte aligned
    bad = [torch.zeros(p1.n_vars + 1, dtype=torch.float64, device="cuda:0")[1:], outs[1], outs[2]]
    with pytest.raises(_abi.SnapError) as ei:
        b.bind(uh, pr, bad, lam, st)
    assert ei.value.code == 1
    with pytest.raises(_abi.SnapError) as ei:
        Batch([Problem("toy", 3, 3)], [0])
    assert ei.value.code == 2
    e = Batch([p1], [])
    e.bind([], [], [], [], [])
    e.project()
