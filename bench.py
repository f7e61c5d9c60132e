#!/usr/bin/env python3
"""Benchmark: converged projections/s on the Burgers-type 1-D projection workload.

Workload (synthetic, seeded; the paper's trained flow models and PDE datasets are not
available): family B (IC + per-slice mass + energy + boundary invariant), B = 512 samples,
nx = 128, nt = 100, FP64.  A step is one snap_project call over one batch of 512 samples
(parameter derivation, the moment-path Newton-KKT kernel, per-sample statistics).  Four
distinct input/output sets rotate between steps so the working set (4 x 107 MB) exceeds the
126 MB L2.  A sample counts as converged when its status is OK and ||h||_inf <= 1e-8 over all
nominal rows, recomputed after the timed region from the written u (snap_constraint_residual).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank projects its own 512-sample shard (weak scaling, no collective on
the data path); timing is the max over ranks.  --impl reference times the oracle (dense
Newton-KKT on the host cores) on bounded samples of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged projections/s (‖h‖∞≤1e-8), 1D Burgers B=512; adjoint/forward time"
UNIT = "projections/s"
WORKLOAD = dict(name="burgers_1d", family="B", B=512, nx=128, nt=100, seed=1001)
H_TOL = 1e-8
ROTATE = 4
# the forward path's tile kernel (moments, slice solves, write-back; the prepare and
# statistics kernels around it overlap it by programmatic dependent launch)
KERNELS = ("k1d_mixed",)
KERNEL = "+".join(KERNELS)
KERNEL_SOURCES = ("paper_2607_00095_b300/csrc/kern_1d_mixed.cu", "paper_2607_00095_b300/csrc/tile_1d.cuh",
                  "paper_2607_00095_b300/csrc/slice_newton.cuh", "paper_2607_00095_b300/csrc/df64.cuh",
                  "paper_2607_00095_b300/csrc/snap_internal.h", "paper_2607_00095_b300/csrc/snap_bounds.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 2-D, uneven-batch and sampling-loop measurements beside the headline")
    ap.add_argument("--extra-only", action="store_true",
                    help="run only the 2-D, uneven-batch and sampling-loop measurements (one JSON line)")
    return ap.parse_args()


def shard_seed(seed, r, rank):
    """Seed of rotation set r on rank `rank`: every rank projects its own samples (weak
    scaling; the batches of different ranks are independent problems)."""
    return seed + 7919 * r + 104729 * rank


def reduce_over_ranks(elapsed_ms, converged, device):
    """Whole-job timing and count over all ranks: the slowest rank's time, the sum of the
    converged samples (one all-reduce each; nothing on the data path)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(converged)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def sources_digest(sources):
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, src), "rb").read())
    return h.hexdigest()


def link_ceiling(uh_h, pr_h, u_h, lam_h, st_h, d_in, d_out, reps):
    """Plain pinned-memory copies of one step's bytes: host -> device alone, device -> host
    alone, and both directions at once on two streams (ms per step and GB/s)."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def up():
        with torch.cuda.stream(s1):
            d_in[0].copy_(uh_h, non_blocking=True)
            d_in[1].copy_(pr_h, non_blocking=True)

    def down():
        with torch.cuda.stream(s2):
            u_h.copy_(d_out[0], non_blocking=True)
            lam_h.copy_(d_out[1], non_blocking=True)
            st_h.copy_(d_out[2], non_blocking=True)

    def timed(fns):
        for f in fns:
            f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for f in fns:
                f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / reps

    up_ms, down_ms, both_ms = timed([up]), timed([down]), timed([up, down])
    h2d = uh_h.numel() * 8 + pr_h.numel() * 8
    d2h = u_h.numel() * 8 + lam_h.numel() * 8 + st_h.numel()
    return {"h2d_gbs": h2d / (up_ms * 1e6), "d2h_gbs": d2h / (down_ms * 1e6), "both_ms": both_ms}


def kernel_traffic(name, sources):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != sources_digest(sources):
        return None
    return rec.get("traffic_bytes_per_launch_full_size")


# ---------------------------------------------------------------------------------------
# oracle timing (cpu baseline / reference arm)
# ---------------------------------------------------------------------------------------
def oracle_rate(uh, pr, budget_s=10.0, chunk=8, nthreads=0):
    """Run the oracle on chunks of samples until budget_s elapses; converged samples / s."""
    from oracle import solve
    w = WORKLOAD
    t0 = time.perf_counter()
    done = conv = 0
    while done < uh.shape[0]:
        sl = slice(done, min(done + chunk, uh.shape[0]))
        _, _, st, _, _ = solve.project_1d(w["family"], w["nx"], w["nt"], pr[sl], uh[sl], nthreads=nthreads)
        conv += int(((st["status"] == 0) & (st["h_inf"] <= H_TOL)).sum())
        done = sl.stop
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return conv / el, done, el


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import solve
    from paper_2607_00095_b300 import synthetic
    w = WORKLOAD
    uh, pr = synthetic.gen_1d(w["seed"], w["B"], w["nx"], w["nt"], w["family"])
    chunk = 8
    nthreads = solve.max_threads()
    for s in range(args.warmup):
        i = (s * chunk) % w["B"]
        solve.project_1d(w["family"], w["nx"], w["nt"], pr[i:i + chunk], uh[i:i + chunk])
    conv = 0
    t0 = time.perf_counter()
    for s in range(args.steps):
        i = ((args.warmup + s) * chunk) % w["B"]
        _, _, st, _, _ = solve.project_1d(w["family"], w["nx"], w["nt"], pr[i:i + chunk], uh[i:i + chunk])
        conv += int(((st["status"] == 0) & (st["h_inf"] <= H_TOL)).sum())
    el = time.perf_counter() - t0
    value = conv / el
    sample = f"{chunk} samples of the {w['name']} workload per step (rotating through the 512), dense Newton-KKT"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w["name"], "family": w["family"], "B": w["B"], "nx": w["nx"],
                       "nt": w["nt"], "samples_per_step": chunk},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2607_00095_b300 import Problem, api, decode_stats, options, synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.extra_only:
        hbm0 = measured_peaks().get("hbm_gbs") or 6400.0
        print(json.dumps({"div_2d": measure_div2d(dev, hbm0), "uneven": measure_uneven(dev),
                          "pcfm": measure_pcfm(dev),
                          "vorticity_2d": measure_vorticity(dev, hbm0),
                          "burgers_bc_1d": measure_burgers_bc(dev, hbm0),
                          "burgers_flux_1d": measure_burgers_flux(dev, hbm0, 5),
                          "heat2_1d": measure_heat(dev, hbm0)}), flush=True)
        return 0
    w = WORKLOAD
    B, nx, nt = w["B"], w["nx"], w["nt"]
    p = Problem(w["family"], nx, nt)
    opts = options()

    # rotating input / output sets (different seeds per set and per rank)
    sets = []
    host0 = None
    for r in range(ROTATE):
        seed = shard_seed(w["seed"], r, rank)
        uh, pr = synthetic.gen_1d(seed, B, nx, nt, w["family"])
        if r == 0:
            host0 = (uh, pr)
        d_uh = torch.as_tensor(uh.reshape(B, -1), device=dev)
        d_pr = torch.as_tensor(pr, device=dev)
        out = (torch.empty_like(d_uh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        sets.append((d_uh, d_pr, out))
    ws = p.workspace(B, dev)

    # the C-ABI call with its arguments marshalled once per rotation set (the timed loop then
    # costs one ctypes call per step on the host)
    import ctypes as C
    L = api.lib()
    stream = api._stream()
    calls = []
    for d_uh, d_pr, out in sets:
        calls.append((p.handle, B, api._ptr(d_uh), api._ptr(d_pr), None, api._ptr(out[0]),
                      api._ptr(out[1]), api._ptr(out[2]), C.byref(opts), api._ptr(ws),
                      ws.numel(), stream))

    def step(i):
        api.check(L.snap_project(*calls[i % ROTATE]))
        return L.snap_last_launch_count()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    # eager C-ABI loop (host launch overhead included), with the library's per-kernel CUDA
    # events around every launch of the dominant kernel
    api.profile_reset()
    api.profile_enable(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        step(i)
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / args.steps
    k_parts = {name: api.profile_read(name) for name in KERNELS}
    k_ms = sum(ms for ms, _ in k_parts.values())
    k_n = min(n for _, n in k_parts.values())
    api.profile_enable(0)
    api.profile_reset()

    # the production form: one CUDA graph per rotation set (a graph holds one whole step)
    cap_stream = torch.cuda.Stream()
    graphs = []
    launches_per_step = 0
    with torch.cuda.stream(cap_stream):
        for r in range(ROTATE):
            call = calls[r][:-1] + (api._stream(cap_stream),)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap_stream):
                api.check(L.snap_project(*call))
                launches_per_step = L.snap_last_launch_count()
            graphs.append(g)
    for g in graphs:
        g.replay()
    torch.cuda.synchronize()
    # one step per graph, for comparison (the launch gap between graphs included)
    graphs[0].replay()
    e0.record()
    for i in range(args.steps):
        graphs[i % ROTATE].replay()
    e1.record()
    torch.cuda.synchronize()
    single_graph_ms = e0.elapsed_time(e1) / args.steps
    # the timed form: one graph holds ROTATE consecutive steps (one per rotation set), so the
    # prepare kernel of each step is launched as a programmatic dependent of the previous
    # step's statistics kernel instead of behind a graph launch
    g_multi = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(g_multi, stream=cap_stream):
            for r in range(ROTATE):
                api.check(L.snap_project(*(calls[r][:-1] + (api._stream(cap_stream),))))
    g_multi.replay()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # an untimed lead-in graph keeps the GPU busy while the host enqueues the timed ones: the
    # start event is then not recorded on an idle stream that waits for the first submission
    g_multi.replay()
    e0.record()
    for _ in range(args.steps // ROTATE):
        g_multi.replay()
    for i in range(args.steps % ROTATE):
        graphs[i].replay()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    steps_timed = args.steps
    launches = args.steps * launches_per_step

    # converged samples of each set, from the written u (untimed)
    conv_per_set = []
    for d_uh, d_pr, out in sets:
        _, hinf = p.residual(out[0], d_pr, want_rows=False)
        st = decode_stats(out[2])
        ok = (st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)
        conv_per_set.append(int(ok.sum()))
    conv = sum(conv_per_set[i % ROTATE] for i in range(steps_timed))
    if world > 1:
        elapsed_ms, conv = reduce_over_ranks(elapsed_ms, conv, dev)
    value = conv / (elapsed_ms / 1e3)

    # adjoint / forward time (differentiation workload: same shapes, dL/du ~ N(0, 1))
    gbar = torch.as_tensor(synthetic.gen_gbar(1002, (B, nt * nx)), device=dev)
    d_uh, d_pr, out = sets[0]
    reps = 20

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        fn()                    # untimed lead-in, as in the timed loop
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    u0, lam0, st0 = out
    fwd_ms = timed(lambda: p.project(d_uh, d_pr, opts=opts, out=out, workspace=ws))
    bwd_ms = timed(lambda: p.backward(gbar, u0, lam0, d_pr, stats=st0))
    # the adjoint's tile kernel against the forward's, from the same kind of events
    api.profile_reset()
    api.profile_enable(1)
    for _ in range(reps):
        p.project(d_uh, d_pr, opts=opts, out=out, workspace=ws)
        p.backward(gbar, u0, lam0, d_pr, stats=st0)
    torch.cuda.synchronize()
    kf_ms, kf_n = api.profile_read("k1d_mixed")
    kb_ms, kb_n = api.profile_read("k1d_bwd_mixed")
    api.profile_enable(0)
    kf_us, kb_us = 1e3 * kf_ms / max(kf_n, 1), 1e3 * kb_ms / max(kb_n, 1)

    # end to end through the public API with host buffers: every step copies its inputs from
    # pinned host memory and reads its result back; three buffer sets and three streams
    # (copy in, project, copy out) let step i+1's upload and step i-1's download run while
    # step i projects (PCIe is full duplex)
    e2e = None
    if not args.no_e2e:
        NS = 3
        uh_h = torch.as_tensor(host0[0].reshape(B, -1)).pin_memory()
        pr_h = torch.as_tensor(host0[1]).pin_memory()
        u_h = [torch.empty_like(uh_h).pin_memory() for _ in range(NS)]
        lam_h = [torch.empty(B, p.n_rows, dtype=torch.float64).pin_memory() for _ in range(NS)]
        st_h = [torch.empty(B, 40, dtype=torch.uint8).pin_memory() for _ in range(NS)]
        d_in = [(torch.empty_like(d_uh), torch.empty_like(d_pr)) for _ in range(NS)]
        d_out = [(torch.empty_like(d_uh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
                  torch.empty(B, 40, dtype=torch.uint8, device=dev)) for _ in range(NS)]
        s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(NS)]
        ev_c = [torch.cuda.Event() for _ in range(NS)]
        ev_out = [torch.cuda.Event() for _ in range(NS)]
        for j in range(NS):
            for ev in (ev_c[j], ev_out[j]):
                ev.record(s_c)

        def e2e_step(i):
            j = i % NS
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_c[j])            # the set's inputs were consumed
                d_in[j][0].copy_(uh_h, non_blocking=True)
                d_in[j][1].copy_(pr_h, non_blocking=True)
                ev_in[j].record(s_in)
            with torch.cuda.stream(s_c):
                s_c.wait_event(ev_in[j])
                s_c.wait_event(ev_out[j])           # the set's last result was read back
                p.project(d_in[j][0], d_in[j][1], opts=opts, out=d_out[j], workspace=ws,
                          stream=s_c)
                ev_c[j].record(s_c)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_c[j])
                u_h[j].copy_(d_out[j][0], non_blocking=True)
                lam_h[j].copy_(d_out[j][1], non_blocking=True)
                st_h[j].copy_(d_out[j][2], non_blocking=True)
                ev_out[j].record(s_out)

        for i in range(6):
            e2e_step(i)
        torch.cuda.synchronize()
        n_e2e = max(9, min(args.steps, 30))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s_in)
        for i in range(n_e2e):
            e2e_step(i)
        s_out.wait_stream(s_in)
        s_out.wait_stream(s_c)
        b.record(s_out)
        torch.cuda.synchronize()
        e2e_ms = a.elapsed_time(b) / n_e2e
        st = np.frombuffer(st_h[(n_e2e - 1) % NS].numpy().tobytes(), dtype=api.STATS_DTYPE)
        conv_e2e = int(((st["status"] == 0) & (st["h_inf"] <= H_TOL)).sum())
        h2d = int(uh_h.numel() * 8 + pr_h.numel() * 8)
        d2h = int(u_h[0].numel() * 8 + lam_h[0].numel() * 8 + st_h[0].numel())
        # the link itself: the same bytes moved by plain pinned copies, each direction alone
        # and both at once (the ceiling an end-to-end step can reach)
        link = link_ceiling(uh_h, pr_h, u_h[0], lam_h[0], st_h[0], d_in[0], d_out[0], n_e2e)
        e2e = {"value": conv_e2e * world / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e2e_ms,
               "link_gbs_h2d": link["h2d_gbs"], "link_gbs_d2h": link["d2h_gbs"],
               "link_ms_both": link["both_ms"],
               "link_frac": link["both_ms"] / e2e_ms,
               "pipeline": "3 buffer sets: upload / project / download of consecutive steps overlap"}

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6400.0
    bytes_per_sample = 8 * (2 * p.n_vars + p.n_rows + p.n_params) + 40
    launch_bytes = bytes_per_sample * B
    k_avg_ms = k_ms / max(k_n, 1)
    fma_launch = B * (nt - 1) * (nx - 2)        # interior values of the slices k >= 1
    achieved = launch_bytes / (k_avg_ms / 1e3) / 1e9
    traffic = kernel_traffic(KERNEL, KERNEL_SOURCES)
    fp64 = api.measure_fp64_rate(local)

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        extra["div_2d"] = measure_div2d(dev, hbm)
        extra["uneven"] = measure_uneven(dev)
        extra["pcfm"] = measure_pcfm(dev)
        extra["vorticity_2d"] = measure_vorticity(dev, hbm)
        extra["burgers_bc_1d"] = measure_burgers_bc(dev, hbm)
        extra["burgers_flux_1d"] = measure_burgers_flux(dev, hbm, 5)
        extra["burgers_flux10_1d"] = measure_burgers_flux(dev, hbm, 10)
        extra["heat2_1d"] = measure_heat(dev, hbm)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import solve
        cores = solve.max_threads()
        # the same oracle on one host core (a shorter sample of the same samples), then on all
        # of them (the thread count is a setting of the oracle library that persists)
        rate1, n_s1, el1 = oracle_rate(*host0, budget_s=4.0, nthreads=1)
        rate, n_s, el = oracle_rate(*host0, budget_s=10.0, nthreads=cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {n_s} samples of the {w['name']} workload (seed {w['seed']}), "
                         f"dense Newton-KKT per connected component, {el:.1f} s",
               "one_core": {"value": rate1, "unit": UNIT, "cores": 1,
                            "sample": f"first {n_s1} samples, {el1:.1f} s"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps_timed,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / steps_timed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "family": "B (IC, mass, energy, boundary invariant)",
                       "B_per_gpu": B, "nx": nx, "nt": nt, "path": "mixed",
                       "l2": f"{ROTATE} rotating input/output sets of {launch_bytes / 1e6:.0f} MB (> 126 MB L2)"},
            "converged_per_step": conv / steps_timed,
            "timing": (f"one CUDA graph per {ROTATE} consecutive steps (one step per input set; "
                       f"an untimed lead-in graph runs ahead of the start event; "
                       f"{single_graph_ms:.4f} ms/step with one graph per step); eager C-ABI loop "
                       f"{eager_ms:.4f} ms/step, in which the kernel events were taken"),
            "ms_per_step_one_graph_per_step": single_graph_ms,
            "adjoint_forward_ratio": bwd_ms / fwd_ms,
            "adjoint": {"forward_ms": fwd_ms, "backward_ms": bwd_ms,
                        "forward_kernel_us": kf_us, "backward_kernel_us": kb_us,
                        "kernel_ratio": kb_us / kf_us if kf_us > 0 else None,
                        "workspace_bytes": p.workspace_bytes(B),
                        "note": "the adjoint rebuilds the slice factors from (u, lambda)"},
            "roofline": {"bound": "hbm", "kernel": KERNEL, "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                         "algorithmic_bytes_per_launch": launch_bytes, "kernel_ms": k_avg_ms,
                         "kernel_ms_parts": {n: ms / max(c, 1) for n, (ms, c) in k_parts.items()},
                         "peak_source": peak_src,
                         # the co-bound: one FP64 FMA per written interior value (the write-back
                         # u = a u_hat + c), against the FP64 FMA rate measured by the library
                         "fp64": {"fma_per_launch": fma_launch,
                                  "achieved_fma_per_s": fma_launch / (k_avg_ms * 1e-3),
                                  "peak_fma_per_s": fp64,
                                  "frac": fma_launch / (k_avg_ms * 1e-3) / fp64 if fp64 else None}},
            "fp64_fma_per_s": fp64,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _event_ms(fn, reps):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    fn()                        # untimed lead-in: the start event is not taken on an idle stream
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_div2d(dev, hbm, reps=50):
    """The 2-D velocity workload: B=64 samples of (u, v) on 64 x 64 x 16 frames (divergence
    rows + kinetic energy); two rotating sets (2 x 134 MB in + out > L2), CUDA graphs."""
    import torch

    from paper_2607_00095_b300 import Problem, api, decode_stats, synthetic
    w = synthetic.WORKLOADS["div_2d"]
    B, N, nt = w["B"], w["N"], w["nt"]
    p = Problem("C", N, nt)
    sets = []
    for r in range(2):
        wh, pr = synthetic.gen_2d(w["seed"] + 7919 * r, B, N, nt)
        d_wh = torch.as_tensor(wh.reshape(B, -1), device=dev)
        d_pr = torch.as_tensor(pr, device=dev)
        out = (torch.empty_like(d_wh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        sets.append((d_wh, d_pr, out))
    ws = p.workspace(B, dev)
    for d_wh, d_pr, out in sets:
        p.project(d_wh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    api.profile_reset()
    api.profile_enable(1)
    for i in range(10):
        d_wh, d_pr, out = sets[i % 2]
        p.project(d_wh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    k_ms, k_n = api.profile_read("k2d_frame")
    api.profile_enable(0)
    api.profile_reset()
    cap = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(cap):
        for d_wh, d_pr, out in sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                p.project(d_wh, d_pr, out=out, workspace=ws, stream=cap)
            graphs.append(g)
    for g in graphs:
        g.replay()
    it = [0]

    def step():
        graphs[it[0] % 2].replay()
        it[0] += 1
    ms = _event_ms(step, reps)
    conv = 0
    for d_wh, d_pr, out in sets:
        _, hinf = p.residual(out[0], d_pr, want_rows=False)
        st = decode_stats(out[2])
        conv += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
    conv /= 2
    bytes_per_call = (8 * (2 * p.n_vars + p.n_rows + p.n_params) + 40) * B
    kavg = k_ms / max(k_n, 1)
    return {"workload": "div_2d", "B": B, "N": N, "nt": nt, "ms_per_call": ms,
            "converged_per_call": conv, "projections_per_s": conv / (ms / 1e3),
            "kernel": "k2d_frame", "kernel_ms": kavg,
            "hbm_frac_of_measured": bytes_per_call / (kavg / 1e3) / 1e9 / hbm,
            "algorithmic_bytes_per_call": bytes_per_call,
            "note": "FP32-pipe bound (four M x M products per class per refinement round)"}


def measure_uneven(dev, reps=30):
    """The uneven mix: 1024 instances (seed 1004), 75 % family B with nx in {64, 96, 128, 192,
    256} and nt in {50, 100, 200}, the rest 2-D at 32 x 32 x 8; inputs 140 MB (> L2).  One
    persistent launch (autotuned schedule, library-owned CUDA graph) against one plain launch
    per (family, size) group (the same calls captured in a CUDA graph)."""
    import numpy as np
    import torch

    from paper_2607_00095_b300 import Batch, Problem, decode_stats, synthetic
    mix = synthetic.gen_uneven(**synthetic.WORKLOADS["uneven"])
    keys = sorted({(m["family"], m["nx"], m["nt"]) for m in mix})
    probs = [Problem(f, nx, nt) for f, nx, nt in keys]
    inst = np.array([keys.index((m["family"], m["nx"], m["nt"])) for m in mix], np.int32)
    b = Batch(probs, inst)
    bufs = b.alloc(dev)
    in_bytes = 0
    for pi, g in bufs.items():
        g["uh"].copy_(torch.as_tensor(np.stack([mix[i]["u_hat"].reshape(-1) for i in g["ids"]])))
        g["pr"].copy_(torch.as_tensor(np.stack([mix[i]["params"] for i in g["ids"]])))
        in_bytes += g["uh"].numel() * 8
    sched, tune_ms = b.autotune(reps=5)
    group_lanes = {f"{f} {nx}x{nt}": l for (f, nx, nt), l in zip(keys, b.group_lanes())}
    n = len(mix)
    t_ns = torch.zeros(n, 2, dtype=torch.int64, device=dev)
    b.capture_graph(t_ns=t_ns)
    for _ in range(3):
        b.launch_graph()
    ms_p = _event_ms(b.launch_graph, reps)
    tt = t_ns.cpu().numpy().astype(np.float64)
    lat_us = (tt[:, 1] - tt[:, 0]) / 1e3
    makespan_us = (tt[:, 1].max() - tt[:, 0].min()) / 1e3

    def converged():
        c = 0
        for pi, g in bufs.items():
            _, hinf = probs[pi].residual(g["u"], g["pr"], want_rows=False)
            st = decode_stats(g["st"])
            c += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
        return c
    conv_p = converged()
    cap = torch.cuda.Stream()
    b.project_grouped()
    torch.cuda.synchronize()
    with torch.cuda.stream(cap):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            b.project_grouped(stream=cap)
    g.replay()
    ms_g = _event_ms(g.replay, reps)
    conv_g = converged()
    # the adjoint of the mix (dL/du ~ N(0, 1)): one persistent launch (owned graph) against one
    # snap_project_backward launch per group (the same calls captured in a graph)
    b.launch_graph()
    gbufs = b.alloc_backward(dev)
    for pi, gb in gbufs.items():
        gb["gu"].copy_(torch.as_tensor(np.stack([synthetic.gen_gbar(2004 + int(i), mix[i]["u_hat"].size)
                                                 for i in gb["ids"]])))
    b.capture_graph_backward()
    b.launch_graph_backward()
    bms_p = _event_ms(b.launch_graph_backward, reps)
    b.backward_grouped()
    torch.cuda.synchronize()
    with torch.cuda.stream(cap):
        gbw = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gbw, stream=cap):
            b.backward_grouped(stream=cap)
    gbw.replay()
    bms_g = _event_ms(gbw.replay, reps)
    return {"workload": "uneven", "instances": n, "groups": len(keys),
            "schedule": sched, "lanes_per_slice_by_group": group_lanes,
            "autotune_best_ms": tune_ms,
            "persistent_ms_per_call": ms_p, "grouped_ms_per_call": ms_g,
            "speedup_vs_grouped": ms_g / ms_p,
            "converged_persistent": conv_p, "converged_grouped": conv_g,
            "projections_per_s": conv_p / (ms_p / 1e3),
            "grouped_projections_per_s": conv_g / (ms_g / 1e3),
            "latency_us_p50": float(np.percentile(lat_us, 50)),
            "latency_us_p99": float(np.percentile(lat_us, 99)),
            "makespan_us": makespan_us, "input_bytes": in_bytes,
            "backward_persistent_ms_per_call": bms_p, "backward_grouped_ms_per_call": bms_g,
            "backward_speedup_vs_grouped": bms_g / bms_p,
            "persistent_launches_per_call": 1,
            "grouped_launches_per_call": sum(2 if f == "C" else 3 for f, _, _ in keys)}


def measure_vorticity(dev, hbm, reps=50):
    """The 2-D vorticity constraints of the Navier-Stokes problem (IC, total vorticity,
    enstrophy per frame): B = 512 samples of 16 x 16 x 50 frames; four rotating sets (> L2),
    CUDA graphs."""
    import torch

    from paper_2607_00095_b300 import api, decode_stats, synthetic, vorticity_problem
    w = synthetic.WORKLOADS["vorticity_2d"]
    B, N, nt = w["B"], w["N"], w["nt"]
    p = vorticity_problem(N, nt)
    sets = []
    for r in range(4):
        uh, pr = synthetic.gen_vorticity(w["seed"] + 7919 * r, B, N, nt)
        d_uh = torch.as_tensor(uh.reshape(B, -1), device=dev)
        d_pr = torch.as_tensor(pr, device=dev)
        out = (torch.empty_like(d_uh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        sets.append((d_uh, d_pr, out))
    ws = p.workspace(B, dev)
    for d_uh, d_pr, out in sets:
        p.project(d_uh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    cap = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(cap):
        for d_uh, d_pr, out in sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                p.project(d_uh, d_pr, out=out, workspace=ws, stream=cap)
            graphs.append(g)
    for g in graphs:
        g.replay()
    it = [0]

    def step():
        graphs[it[0] % 4].replay()
        it[0] += 1
    ms = _event_ms(step, reps)
    conv = 0
    for d_uh, d_pr, out in sets:
        _, hinf = p.residual(out[0], d_pr, want_rows=False)
        st = decode_stats(out[2])
        conv += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
    conv /= 4
    bytes_per_call = (8 * (2 * p.n_vars + p.n_rows + p.n_params) + 40) * B
    return {"workload": "vorticity_2d", "B": B, "N": N, "nt": nt, "ms_per_call": ms,
            "converged_per_call": conv, "projections_per_s": conv / (ms / 1e3),
            "hbm_frac_of_measured_step": bytes_per_call / (ms / 1e3) / 1e9 / hbm,
            "path": "family A rows on flattened frames (nx = N^2), mixed-pipe tile kernel"}


def measure_burgers_flux(dev, hbm, K, reps=50):
    """Family E, the Burgers IC regime with Godunov flux rows: B = 512 samples of
    nx = nt = 101, IC + mass + Flux(K); four rotating sets (> L2), CUDA graphs."""
    import torch

    from paper_2607_00095_b300 import Problem, api, decode_stats, synthetic
    w = synthetic.WORKLOADS["burgers_flux_1d"]
    B, nx, nt = w["B"], w["nx"], w["nt"]
    p = Problem("E", nx, nt, n_flux=K)
    sets = []
    for r in range(4):
        uh, g = synthetic.gen_burgers_flux(w["seed"] + 7919 * r, B, nx, nt)
        d_uh = torch.as_tensor(uh.reshape(B, -1), device=dev)
        d_pr = torch.as_tensor(g, device=dev)
        out = (torch.empty_like(d_uh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        sets.append((d_uh, d_pr, out))
    ws = p.workspace(B, dev)
    for d_uh, d_pr, out in sets:
        p.project(d_uh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    api.profile_reset()
    api.profile_enable(1)
    for i in range(12):
        d_uh, d_pr, out = sets[i % 4]
        p.project(d_uh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    k_ms, k_n = api.profile_read("k1dflux_forward")
    api.profile_enable(0)
    api.profile_reset()
    cap = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(cap):
        for d_uh, d_pr, out in sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                p.project(d_uh, d_pr, out=out, workspace=ws, stream=cap)
            graphs.append(g)
    for g in graphs:
        g.replay()
    it = [0]

    def step():
        graphs[it[0] % 4].replay()
        it[0] += 1
    ms = _event_ms(step, reps)
    conv = 0
    for d_uh, d_pr, out in sets:
        _, hinf = p.residual(out[0], d_pr, want_rows=False)
        st = decode_stats(out[2])
        conv += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
    conv /= 4
    bytes_per_call = (8 * (2 * p.n_vars + p.n_rows + p.n_params) + 40) * B
    kavg = k_ms / max(k_n, 1)
    # the adjoint (dL/du_hat and dL/dg) on the first set, kernel time from the same events
    gbar = torch.as_tensor(synthetic.gen_gbar(w["seed"] + 1, (B, p.n_vars)), device=dev)
    d_uh, d_pr, out = sets[0]
    for _ in range(3):
        p.backward(gbar, out[0], out[1], d_pr, stats=out[2])
    torch.cuda.synchronize()
    api.profile_reset()
    api.profile_enable(1)
    for _ in range(12):
        p.backward(gbar, out[0], out[1], d_pr, stats=out[2])
    torch.cuda.synchronize()
    b_ms, b_n = api.profile_read("k1dflux_backward")
    api.profile_enable(0)
    api.profile_reset()
    bavg = b_ms / max(b_n, 1)
    return {"workload": f"burgers_flux_1d (Flux({K}))", "B": B, "nx": nx, "nt": nt, "n_flux": K,
            "ms_per_call": ms, "converged_per_call": conv,
            "projections_per_s": conv / (ms / 1e3), "kernel": "k1dflux_forward",
            "kernel_ms": kavg, "hbm_frac_of_measured": bytes_per_call / (kavg / 1e3) / 1e9 / hbm,
            "algorithmic_bytes_per_call": bytes_per_call, "backward_kernel_ms": bavg,
            "adjoint_forward_ratio": bavg / kavg}


def measure_heat(dev, hbm, reps=30):
    """Family F, the heat problem's second constraint regime (IC, mass, Crank-Nicolson PDE
    residual, energy evolution): B = 512 samples of nx = nt = 100; four rotating sets, CUDA
    graphs.  Forward (u by the time chain, lambda by backward substitution, statistics) and
    the adjoint (dL/d(g, alpha)) kernel times."""
    import torch

    from paper_2607_00095_b300 import Problem, api, decode_stats, synthetic
    w = synthetic.WORKLOADS["heat2_1d"]
    B, nx, nt = w["B"], w["nx"], w["nt"]
    p = Problem("F", nx, nt)
    sets = []
    for r in range(4):
        uh, pr = synthetic.gen_heat(w["seed"] + 7919 * r, B, nx, nt)
        d_uh = torch.as_tensor(uh.reshape(B, -1), device=dev)
        d_pr = torch.as_tensor(pr, device=dev)
        out = (torch.empty_like(d_uh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        sets.append((d_uh, d_pr, out))
    for d_uh, d_pr, out in sets:
        p.project(d_uh, d_pr, out=out)
    torch.cuda.synchronize()
    api.profile_reset()
    api.profile_enable(1)
    for i in range(8):
        d_uh, d_pr, out = sets[i % 4]
        p.project(d_uh, d_pr, out=out)
    torch.cuda.synchronize()
    k_ms, k_n = api.profile_read("k_heat_forward")
    api.profile_enable(0)
    api.profile_reset()
    cap = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(cap):
        for d_uh, d_pr, out in sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                p.project(d_uh, d_pr, out=out, stream=cap)
            graphs.append(g)
    for g in graphs:
        g.replay()
    it = [0]

    def step():
        graphs[it[0] % 4].replay()
        it[0] += 1
    ms = _event_ms(step, reps)
    conv = 0
    for d_uh, d_pr, out in sets:
        _, hinf = p.residual(out[0], d_pr, want_rows=False)
        st = decode_stats(out[2])
        conv += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
    conv /= 4
    bytes_per_call = (8 * (2 * p.n_vars + p.n_rows + p.n_params) + 40) * B
    kavg = k_ms / max(k_n, 1)
    gbar = torch.as_tensor(synthetic.gen_gbar(w["seed"] + 1, (B, p.n_vars)), device=dev)
    d_uh, d_pr, out = sets[0]
    for _ in range(3):
        p.backward(gbar, out[0], out[1], d_pr, stats=out[2])
    torch.cuda.synchronize()
    api.profile_reset()
    api.profile_enable(1)
    for _ in range(8):
        p.backward(gbar, out[0], out[1], d_pr, stats=out[2])
    torch.cuda.synchronize()
    b_ms, b_n = api.profile_read("k_heat_backward")
    api.profile_enable(0)
    api.profile_reset()
    bavg = b_ms / max(b_n, 1)
    # the forward is two sequential chains of nt - 1 periodic solves per sample (u, then lambda),
    # the adjoint one: the kernels are bound by the chain's latency, so the time per chain step
    # is the figure to compare (the solve alone is ~1.4k cycles of double-float latency)
    return {"workload": "heat2_1d", "B": B, "nx": nx, "nt": nt, "ms_per_call": ms,
            "converged_per_call": conv, "projections_per_s": conv / (ms / 1e3),
            "kernel": "k_heat_forward", "kernel_ms": kavg,
            "hbm_frac_of_measured": bytes_per_call / (kavg / 1e3) / 1e9 / hbm,
            "algorithmic_bytes_per_call": bytes_per_call,
            "bound": "latency of the per-sample time chain (double-float, FP32 pipe)",
            "forward_us_per_chain_step": 1e3 * kavg / (2 * (nt - 1)),
            "backward_kernel_ms": bavg, "backward_us_per_chain_step": 1e3 * bavg / (nt - 1),
            "adjoint_forward_ratio": bavg / kavg}


def measure_burgers_bc(dev, hbm, reps=50):
    """Family D, the Burgers boundary-condition regime: B = 512 samples of nx = nt = 101
    (Dirichlet, mass and Neumann rows per slice); four rotating sets (> L2), CUDA graphs."""
    import torch

    from paper_2607_00095_b300 import Problem, api, decode_stats, synthetic
    w = synthetic.WORKLOADS["burgers_bc_1d"]
    B, nx, nt = w["B"], w["nx"], w["nt"]
    p = Problem("D", nx, nt)
    sets = []
    for r in range(4):
        uh, pr = synthetic.gen_burgers_bc(w["seed"] + 7919 * r, B, nx, nt)
        d_uh = torch.as_tensor(uh.reshape(B, -1), device=dev)
        d_pr = torch.as_tensor(pr, device=dev)
        out = (torch.empty_like(d_uh), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        sets.append((d_uh, d_pr, out))
    ws = p.workspace(B, dev)
    for d_uh, d_pr, out in sets:
        p.project(d_uh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    api.profile_reset()
    api.profile_enable(1)
    for i in range(12):
        d_uh, d_pr, out = sets[i % 4]
        p.project(d_uh, d_pr, out=out, workspace=ws)
    torch.cuda.synchronize()
    k_ms, k_n = api.profile_read("k1dbc_forward")
    api.profile_enable(0)
    api.profile_reset()
    cap = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(cap):
        for d_uh, d_pr, out in sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                p.project(d_uh, d_pr, out=out, workspace=ws, stream=cap)
            graphs.append(g)
    for g in graphs:
        g.replay()
    it = [0]

    def step():
        graphs[it[0] % 4].replay()
        it[0] += 1
    ms = _event_ms(step, reps)
    conv = 0
    for d_uh, d_pr, out in sets:
        _, hinf = p.residual(out[0], d_pr, want_rows=False)
        st = decode_stats(out[2])
        conv += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
    conv /= 4
    bytes_per_call = (8 * (2 * p.n_vars + p.n_rows + p.n_params) + 40) * B
    kavg = k_ms / max(k_n, 1)
    return {"workload": "burgers_bc_1d", "B": B, "nx": nx, "nt": nt, "ms_per_call": ms,
            "converged_per_call": conv, "projections_per_s": conv / (ms / 1e3),
            "kernel": "k1dbc_forward", "kernel_ms": kavg,
            "hbm_frac_of_measured": bytes_per_call / (kavg / 1e3) / 1e9 / hbm,
            "algorithmic_bytes_per_call": bytes_per_call}


def measure_pcfm(dev, reps=20):
    """The sampling loop: one PCFM pass (10 shoot / project / pull-back steps) over B = 512
    Burgers samples, captured in one CUDA graph; two rotating input sets (> L2)."""
    import torch

    from paper_2607_00095_b300 import Problem, decode_stats, synthetic
    w = synthetic.WORKLOADS["pcfm_1d"]
    B, nx, nt, N, s0 = w["B"], w["nx"], w["nt"], w["n_steps"], w["sigma0"]
    p = Problem(w["family"], nx, nt)
    sets = []
    for r in range(2):
        u0, x1, xi, pr = synthetic.gen_pcfm(w["seed"] + 7919 * r, B, nx, nt, w["family"])
        d = [torch.as_tensor(a, device=dev) for a in (u0, x1, xi, pr)]
        out = (torch.empty_like(d[0]), torch.empty(B, p.n_rows, dtype=torch.float64, device=dev),
               torch.empty(B, 40, dtype=torch.uint8, device=dev))
        p.pcfm_sample(*d, n_steps=N, sigma0=s0, out=out)
        sets.append((d, out))
    torch.cuda.synchronize()
    cap = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(cap):
        for d, out in sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                p.pcfm_sample(*d, n_steps=N, sigma0=s0, out=out, stream=cap)
            graphs.append(g)
    for g in graphs:
        g.replay()
    it = [0]

    def step():
        graphs[it[0] % 2].replay()
        it[0] += 1
    ms = _event_ms(step, reps)
    conv = 0
    for d, out in sets:
        _, hinf = p.residual(out[0], d[3], want_rows=False)
        st = decode_stats(out[2])
        conv += int(((st["status"] == 0) & (hinf.cpu().numpy() <= H_TOL)).sum())
    conv /= 2
    return {"workload": "pcfm_1d", "B": B, "nx": nx, "nt": nt, "n_steps": N, "sigma0": s0,
            "ms_per_pass": ms, "converged_samples_per_pass": conv,
            "samples_per_s": conv / (ms / 1e3), "projections_per_s": B * N / (ms / 1e3),
            "velocity": "analytic: (x1 - u0) + sigma0 (1 - tau) xi"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
