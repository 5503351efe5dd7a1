"""Benchmark: coarse-grid correction throughput (GB/s) on one GB300 (replicas on N GPUs).

One step is one coarse-grid correction of Alg. 2 on the 32^4 lattice with 4^4
blocks (8^4 coarse sites) and N_tv = 20, FP64 setup and FP32 storage:
restriction y_c = R y, restarted FGMRES(30) on D_c to relative residual 0.05
(at most 200 applications), prolongation x = P x_c.  The value is the step's
algorithmic bytes (every byte each kernel must move at least once: R twice,
D_c once per application, the vectors of the Krylov basis for the
Gram-Schmidt) divided by the step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L = (32, 32, 32, 32)
B = (4, 4, 4, 4)
NTV = 20
EPS, M0, CSW = 0.3, -0.3, 1.0
SEED = 20151204 + 2
TOL, RESTART, MAX_APPLIES = 0.05, 30, 200
# FGMRES(30) reaches 0.05 on this workload's coarse system in 2 applications (the GPU arm measures
# it: config.applies_per_step); the reference arm's oracle sample runs the same count
APPLIES_PER_STEP = 2
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the 32^4 workload, from
# the ncu captures of the 24^4 case summarised under profiles/ scaled by the number of blocks /
# coarse sites (the per-unit work is the same); valid for the kernels as captured.
TRAFFIC = {"restrict": 2124549284, "prolong": 2124409312, "apply": 483471208}
# the same for the 48^3 x 96 tensor-core workload (captures of the 24^3 x 48 case, x16; the apply
# figure is the tensor-core kernel alone, without the FP32 -> BF16 conversion launch)
TRAFFIC_TC16 = {"restrict": 20641533184, "prolong": 19751972864, "apply": 3679113216}
TC16_KERNELS = {"restrict": "restrict_tc_kernel<16> (Y_c = R Y, BF16 R, 16 RHS)",
                "apply": "xc_to_bf16_kernel<16> + apply_tc_kernel<16> (D_c X_c, BF16 D_c, 16 RHS)",
                "prolong": "prolong_tc_kernel<16> (X = P X_c, BF16 R, 16 RHS)"}
# DRAM bytes of one FP16 coarse application at 32^3 x 64, Ntv = 24 (ncu capture of the full size,
# profiles/apply_mrhs_fp16_32x3x64_ntv24.md)
TRAFFIC_FP16_APPLY = 692893440
# DRAM bytes of one FP32 16-column tcgen05 apply at 32^3 x 64, Ntv = 24: the 16^3 x 32 capture
# (profiles/apply_tc5_fp32_16x3x32_ntv24_nrhs16.md, 90,586.9 KB for 512 sites) x 16 sites
TRAFFIC_MRHS_FP32 = 1449390080
# DRAM traffic / algorithmic bytes of the fused batch launch, from the reduced-volume capture
# (profiles/batch_kernel_small_mixed.md); the full launch's traffic is taken in that proportion
BATCH_TRAFFIC_RATIO = 0.990
# DRAM traffic / algorithmic bytes of one SAP half sweep, from the 16^4 capture (profiles/sap_16x4.md:
# 35.56 MB for 65,536 sites x 504 B); the 32^4 launch is taken in proportion
SAP_TRAFFIC_RATIO = 1.077
METRIC = "coarse-grid correction GB/s & % HBM roofline; batched-mixed vs plain speedup"
WORKLOAD = "fp32_32^4_b4_ntv20: 32^4 Wilson-clover, 4^4 blocks -> 8^4 coarse, Ntv=20, 1 RHS, " \
           "FP64 setup, FP32 R and D_c; step = R y, FGMRES(30) to 0.05 (<=200 applies), P x_c"


def geometry():
    V = int(np.prod(L))
    Vb = int(np.prod(B))
    Vc = V // Vb
    nc = 2 * NTV
    return V, Vb, Vc, nc


def bytes_model(applies, cycles_iters, elem=8):
    """Algorithmic bytes of one step (FP32 complex = 8 B)."""
    V, Vb, Vc, nc = geometry()
    vec_c = Vc * nc * elem
    vec_f = V * 12 * elem
    R = Vc * 2 * NTV * 6 * Vb * elem
    restrict = R + vec_f + vec_c
    prolong = R + vec_c + vec_f
    apply_ = Vc * 9 * nc * nc * elem + 2 * vec_c
    # Arnoldi step j: dots read w and V_0..V_j, update reads w, V_0..V_j and writes w, scale r/w
    gs = sum((2 * (j + 1) + 4) * vec_c for j in cycles_iters)
    return restrict + prolong + applies * apply_ + gs, {"restrict": restrict, "apply": apply_, "prolong": prolong}


def arnoldi_iterations(applies):
    """Arnoldi step indices j of the FGMRES(RESTART) run with `applies` applications."""
    its = []
    left = applies
    while left > 0:
        m = min(RESTART, left)
        its += list(range(m))
        left -= m + 1  # one residual application per restart
    return its


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.samples = []
        if self.proc is None:
            return
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                self.samples.append(f)

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def e2e_pipelined(amg, h, y, x, stream, steps):
    """Seconds for `steps` coarse-grid corrections through amg_cgc with every step's input copied
    from pinned host memory and its result copied back, step k + 1's input copy and step k - 1's
    result copy overlapping step k on their own streams."""
    import torch
    yh = [y.cpu().pin_memory() for _ in range(2)]
    xh = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for _ in range(2)]
    yd = [torch.empty_like(y) for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(h2d):
        yd[0].copy_(yh[0], non_blocking=True)
        ev_in[0].record(h2d)
    for k in range(steps):
        b = k % 2
        if k + 1 < steps:  # next input into the other buffer once step k - 1 has consumed it
            with torch.cuda.stream(h2d):
                if k >= 1:
                    h2d.wait_event(ev_done[1 - b])
                yd[1 - b].copy_(yh[1 - b], non_blocking=True)
                ev_in[1 - b].record(h2d)
        stream.wait_event(ev_in[b])
        if k >= 2:
            stream.wait_event(ev_out[b])  # xd[b] read back by the copy of step k - 2
        amg.amg_cgc(h, yd[b], xd[b], 1, TOL, RESTART, MAX_APPLIES, stream, info=False)
        ev_done[b].record(stream)
        with torch.cuda.stream(d2h):
            d2h.wait_event(ev_done[b])
            xh[b].copy_(xd[b], non_blocking=True)
            ev_out[b].record(d2h)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def max_over_ranks(vals, dist, device):
    """Elementwise maximum of per-rank timings over all ranks (replicas: the job ends with the
    slowest rank)."""
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_gbs(world, step_bytes, steps, seconds):
    """Whole-job throughput: every rank moved step_bytes per step (weak scaling)."""
    return world * step_bytes * steps / seconds / 1e9


FP64_TFLOPS = 1.25  # GB300 FP64 peak (nominal; an FMA-chain probe on this pool measured 1.258)


def setup_report(setup_ms, V, ntv):
    """Setup phase times; the assembly's rank-6 contractions (4 hops over all 2Ntv x 2Ntv entries,
    the self term over the two chirality-diagonal quadrants) as FP64-equivalent flops (8 per
    complex multiply-add) against the FP64 peak."""
    nc = 2 * ntv
    flop = 8.0 * V * 6 * (4 * nc * nc + 2 * ntv * ntv)
    rate = flop / (setup_ms[2] * 1e-3) / 1e12
    return {"clover": round(setup_ms[0], 2), "gram_schmidt": round(setup_ms[1], 2),
            "assembly": round(setup_ms[2], 2), "quantise": round(setup_ms[3], 2),
            "assembly_arith": "f32pair", "assembly_tflop": round(flop / 1e12, 3),
            "assembly_fp64_equiv_tflops": round(rate, 3), "fp64_peak_tflops": FP64_TFLOPS}


def run_gpu(args):
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    V, Vb, Vc, nc = geometry()
    stream = torch.cuda.current_stream()
    seed = SEED + 1000 * rank  # independent replica per rank
    U = sd.links(seed, EPS, L)
    tv = sd.test_vectors(seed, NTV, L)
    p = amg.make_params(L, B, NTV, 1, M0, CSW, amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32,
                        setup_arith=amg.AMG_SETUP_F32PAIR)
    h, _ = amg.amg_setup_coarse(p, U, tv, stream)
    setup_ms = amg.amg_setup_timings(h)
    del U, tv
    torch.cuda.empty_cache()
    y = sd.fine_rhs(seed, 1, L, torch.complex64)
    x = torch.empty_like(y)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        return amg.amg_cgc(h, y, x, 1, TOL, RESTART, MAX_APPLIES, stream, info=False)

    info = amg.amg_cgc(h, y, x, 1, TOL, RESTART, MAX_APPLIES, stream, info=True)
    applies = info[0][0]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # ---- device-resident timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = amg.amg_kernel_launches(h)
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = amg.amg_kernel_launches(h) - launches0
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(ms) / 1000.0
    step_bytes, parts = bytes_model(applies, arnoldi_iterations(applies))
    # ---- per-kernel live timing (events around each launch on the launching stream)
    yc = torch.empty((Vc, 2, NTV, 1), dtype=torch.complex64, device="cuda")
    zc = torch.empty_like(yc)
    amg.amg_restrict(h, y, yc, 1, stream)

    def timed(fn, n):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for _ in range(3):
            fn()
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / n / 1000.0

    t_apply = timed(lambda: amg.amg_coarse_apply(h, yc, zc, 1, stream), 50)
    t_restrict = timed(lambda: amg.amg_restrict(h, y, yc, 1, stream), 20)
    t_prolong = timed(lambda: amg.amg_prolong(h, yc, x, 1, stream), 20)
    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region:
    # every step copies its input host -> device and its result device -> host; the copies of
    # neighbouring steps overlap the coarse-grid correction on two copy streams (double buffers)
    t_e2e = e2e_pipelined(amg, h, y, x, stream, args.steps)
    evenodd = None
    if world == 1 and not args.no_evenodd:
        evenodd = evenodd_comparison(amg, h, y, x, yc, flush, stream, applies, t_total / args.steps, timed)
    status = amg.amg_sync_status(h)
    amg.amg_destroy(h)
    if status != amg.AMG_OK:
        raise RuntimeError("device error: %s" % amg.amg_status_string(status))
    if dist:
        t_total, t_e2e = max_over_ranks([t_total, t_e2e], dist, "cuda")
    value = whole_job_gbs(world, step_bytes, args.steps, t_total)
    e2e_value = whole_job_gbs(world, step_bytes, args.steps, t_e2e)
    peaks, src = measured_peaks()
    # dominant kernel of the step: largest (launches per step x live launch time)
    live = {"restrict": (t_restrict, 1, parts["restrict"], "restrict y_c = R y (FP32 R)"),
            "prolong": (t_prolong, 1, parts["prolong"], "prolong x = P x_c (FP32 R)"),
            "apply": (t_apply, applies, parts["apply"], "coarse apply y_c = D_c x_c (FP32 links)")}
    dom = max(live, key=lambda k: live[k][0] * live[k][1])
    t_dom, _, dom_bytes, dom_name = live[dom]
    achieved = dom_bytes / t_dom / 1e9
    result = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1000.0 * t_total / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": dict(workload_config(applies), parallelism="replicas" if world > 1 else "single"),
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1),
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                     "peak_source": src, "traffic": TRAFFIC.get(dom),
                     "bytes_per_launch": dom_bytes, "avg_launch_us": round(t_dom * 1e6, 2),
                     "step_share": round(t_dom * live[dom][1] / (t_total / args.steps), 3)},
        "kernels": {
            "restrict": {"GB/s": round(parts["restrict"] / t_restrict / 1e9, 1), "us": round(t_restrict * 1e6, 1),
                         "frac": round(parts["restrict"] / t_restrict / 1e9 / peaks["hbm_gbs"], 4)},
            "apply": {"GB/s": round(parts["apply"] / t_apply / 1e9, 1), "us": round(t_apply * 1e6, 1),
                      "frac": round(parts["apply"] / t_apply / 1e9 / peaks["hbm_gbs"], 4)},
            "prolong": {"GB/s": round(parts["prolong"] / t_prolong / 1e9, 1), "us": round(t_prolong * 1e6, 1),
                        "frac": round(parts["prolong"] / t_prolong / 1e9 / peaks["hbm_gbs"], 4)},
        },
        "setup_ms": setup_report(setup_ms, V, NTV),
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": V * 12 * 8,
                "d2h_bytes_per_step": V * 12 * 8},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if evenodd is not None:
        result["evenodd"] = evenodd
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(applies)
    if not args.no_speedup:
        result["batched_mixed_vs_plain"] = speedup_mixed()
    if rank == 0 and world == 1 and not args.no_workloads and not args.lattice:
        # the other workloads, each with its own step time, algorithmic bytes, roofline and clocks
        result["workloads"] = {name: sub_line(fn(args)) for name, fn in
                               (("tc16", run_tc16), ("fp16", run_fp16), ("mrhs", run_mrhs),
                                ("batch", run_batch), ("vcycle", run_vcycle))}
    if dist:
        dist.destroy_process_group()
    return result, rank


SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "roofline", "kernels",
            "setup_ms", "outer_solve", "clocks")


def sub_line(res):
    """A workload's own JSON line reduced to what the default line carries for it."""
    import torch
    torch.cuda.empty_cache()
    return {k: res[k] for k in SUB_KEYS if k in res}


def evenodd_comparison(amg, h, y, x, yc, flush, stream, applies, ms_plain, timed):
    """The even/odd-reduced coarse solve on the same handle: bandwidth of one Schur-complement
    application (three half-lattice passes; algorithmic bytes = D_c with the odd self blocks
    replaced by their inverses, plus x_e and y_e), and the coarse-grid correction with the reduced
    solve against the plain one at the workload's tolerance 0.05 and at 1e-6."""
    import torch
    V, Vb, Vc, nc = geometry()
    t0 = time.perf_counter()
    amg.amg_setup_evenodd(h, stream)
    setup_ms = (time.perf_counter() - t0) * 1e3
    xe = torch.randn((Vc // 2, nc, 1), dtype=torch.complex64, device="cuda")
    ye = torch.empty_like(xe)
    t_schur = timed(lambda: amg.amg_schur_apply(h, xe, ye, 1, stream), 50)
    schur_bytes = Vc * 9 * nc * nc * 8 + Vc * nc * 8
    peaks, _ = measured_peaks()

    def cgc_ms(fn, n=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / n

    out = {"setup_ms": round(setup_ms, 2), "schur_apply_us": round(t_schur * 1e6, 1),
           "schur_GB/s": round(schur_bytes / t_schur / 1e9, 1),
           "schur_frac": round(schur_bytes / t_schur / 1e9 / peaks["hbm_gbs"], 4)}
    for tol, key in ((TOL, "tol_0.05"), (1e-6, "tol_1e-6")):
        ip = amg.amg_cgc(h, y, x, 1, tol, RESTART, 2000, stream, info=True)
        ie = amg.amg_cgc_eo(h, y, x, 1, tol, RESTART, 2000, stream, info=True)
        mp = cgc_ms(lambda: amg.amg_cgc(h, y, x, 1, tol, RESTART, 2000, stream, info=False))
        me = cgc_ms(lambda: amg.amg_cgc_eo(h, y, x, 1, tol, RESTART, 2000, stream, info=False))
        out[key] = {"plain_applies": ip[0][0], "plain_ms": round(mp, 3), "eo_schur_applies": ie[0][0],
                    "eo_ms": round(me, 3), "speedup": round(mp / me, 2)}
    return out


def speedup_mixed(seed=20151204 + 3):
    """Batched mixed precision against plain FP32, per right-hand side, at coarse accuracy 1e-4.

    Workload: 32^3 x 64 lattice, 4^4 blocks (8^3 x 16 coarse), Ntv = 24, 16 right-hand sides.
    Plain: FP32 D_c, single-RHS FGMRES(30) to relative residual 1e-4, one right-hand side after
    the other.  Batched mixed: all 16 right-hand sides at once, FGMRES(30) to 0.05 on the BF16
    (tensor-core) or FP16 D_c, refined with the FP32 D_c until the true residual is <= 1e-4.
    """
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd
    L3, ntv, nrhs = (32, 32, 32, 64), 24, 16
    st = torch.cuda.current_stream()
    U = sd.links(seed, EPS, L3)
    tv = sd.test_vectors(seed, ntv, L3)
    hs = {}
    for name, link in (("fp32", amg.AMG_FP32), ("fp16", amg.AMG_FP16_SCALED), ("bf16", amg.AMG_BF16)):
        p = amg.make_params(L3, B, ntv, nrhs, M0, CSW, link, amg.AMG_FP32, amg.AMG_FP32)
        hs[name], _ = amg.amg_setup_coarse(p, U, tv, st)
    del U, tv
    Vc = int(np.prod(L3)) // int(np.prod(B))
    b = sd.coarse_vector(seed, ntv, nrhs, Vc, torch.complex64)
    cols = [b[..., r:r + 1].contiguous() for r in range(nrhs)]
    x1 = torch.empty_like(cols[0])
    x = torch.empty_like(b)
    res = {}
    try:
        def plain():
            out = []
            for r in range(nrhs):
                out.append(amg.amg_coarse_solve(hs["fp32"], cols[r], x1, 1, 1e-4, 30, 2000, st, info=True)[0])
            return out
        def mixed(name):
            return amg.amg_coarse_solve_mixed(hs["fp32"], hs[name], b, x, nrhs, 1e-4, 0.05, 30, 400, 30, st)
        for fn in (plain, lambda: mixed("bf16"), lambda: mixed("fp16")):
            fn()  # warm-up
        def timed(fn, reps=3):
            best_t, best_info = None, None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                info = fn()
                e1.record(st)
                torch.cuda.synchronize()
                el = e0.elapsed_time(e1) / 1000.0
                if best_t is None or el < best_t:
                    best_t, best_info = el, info
            return best_t, best_info
        tp, ip = timed(plain)
        tb, ib = timed(lambda: mixed("bf16"))
        th, ih = timed(lambda: mixed("fp16"))
        res = {
            "workload": "32^3x64, 4^4 blocks, Ntv=24, 16 RHS; coarse relative residual <= 1e-4",
            "plain_fp32_ms_per_rhs": round(1000 * tp / nrhs, 3),
            "plain_applies_per_rhs": float(np.mean([a for a, _ in ip])),
            "mixed_bf16_tc_ms_per_rhs": round(1000 * tb / nrhs, 3),
            "mixed_bf16_inner_applies": float(np.mean([a for a, _, _ in ib])),
            "mixed_bf16_max_true_residual": max(r for _, _, r in ib),
            "mixed_fp16_ms_per_rhs": round(1000 * th / nrhs, 3),
            "mixed_fp16_max_true_residual": max(r for _, _, r in ih),
            "speedup_bf16": round(tp / tb, 2),
            "speedup_fp16": round(tp / th, 2),
            "timing": "CUDA events around the whole solve (host synchronisations included), best of 3",
        }
    finally:
        for h in hs.values():
            amg.amg_destroy(h)
    return res


SAMPLE_L = (16, 16, 16, 16)  # the oracle's sample lattice: 1/16 of the 32^4 workload, same blocks and N_tv
THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
_SAMPLE = None
_BARRIER = None


def _make_sample(seed):
    """Random orthonormal R and random D_c blocks on the sample lattice (the cost of the oracle's
    loops does not depend on the values) and a fine right-hand side."""
    from oracle import lattice as lat
    Lc = lat.coarse_dims(SAMPLE_L, B)
    Vc = int(np.prod(Lc))
    Vb = int(np.prod(B))
    rng = np.random.default_rng(seed)
    W = rng.normal(size=(Vc, 2, 6 * Vb, NTV)) + 1j * rng.normal(size=(Vc, 2, 6 * Vb, NTV))
    Q = np.linalg.qr(W)[0]
    Dc = (rng.normal(size=(Vc, 9, 2 * NTV, 2 * NTV)) + 1j * rng.normal(size=(Vc, 9, 2 * NTV, 2 * NTV))) / 40
    Dc[:, 0] += 4 * np.eye(2 * NTV)
    y = rng.normal(size=SAMPLE_L[::-1] + (4, 3)) + 1j * rng.normal(size=SAMPLE_L[::-1] + (4, 3))
    return Q, Dc, y, Lc


def _sample_step(applies):
    """One step of the workload on the sample: the oracle's R y, FGMRES(RESTART) with `applies`
    D_c applications (tolerance 0, so the count is fixed), P x_c."""
    from oracle import coarse, krylov
    Q, Dc, y, Lc = _SAMPLE
    yc = coarse.restrict(Q, y, B)
    xc, _, _ = krylov.fgmres(lambda v: coarse.coarse_apply(Dc, v, Lc), yc, tol=0.0, restart=RESTART,
                             max_applies=applies)
    coarse.prolong(Q, xc, SAMPLE_L, B)


def _worker_init(barrier):
    global _SAMPLE, _BARRIER
    _BARRIER = barrier
    _SAMPLE = _make_sample(os.getpid())


def _worker_run(applies, target_s):
    """All workers start together (the barrier holds one task per worker), then each repeats the
    sample step until target_s seconds have passed (at least once)."""
    _BARRIER.wait()
    reps, t0 = 0, time.perf_counter()
    while True:
        _sample_step(applies)
        reps += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            return reps, el


class OraclePool:
    """One single-threaded oracle process per host core (spawn-started), each on its own sample."""

    def __init__(self):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.cores = len(os.sched_getaffinity(0))
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in THREAD_VARS}
        os.environ.update({k: "1" for k in THREAD_VARS})
        try:
            self.ex = cf.ProcessPoolExecutor(max_workers=self.cores, mp_context=ctx, initializer=_worker_init,
                                             initargs=(ctx.Barrier(self.cores),))
            self.round(APPLIES_PER_STEP, 0.0)  # spawn and build every worker's sample
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def round(self, applies, target_s):
        """(sample steps done by all workers, wall seconds of the round)."""
        t0 = time.perf_counter()
        res = [f.result() for f in [self.ex.submit(_worker_run, applies, target_s) for _ in range(self.cores)]]
        return sum(r for r, _ in res), time.perf_counter() - t0

    def close(self):
        self.ex.shutdown()


def sample_step_bytes(applies):
    """Algorithmic bytes of one sample step in the workload's byte model (FP32 data), scaled from
    the workload's volume to the sample's."""
    step, _ = bytes_model(applies, arnoldi_iterations(applies))
    return step * int(np.prod(SAMPLE_L)) / int(np.prod(L))


def sample_description(cores, applies):
    return ("the oracle (numpy FP64) on %d host cores, one single-threaded process per core, each on its own "
            "16^4 sample of the workload (4^4 blocks, Ntv=20, 1/16 of the 32^4 volume): R y, FGMRES(%d) with %d "
            "D_c applications (the workload's count), P x_c; GB/s in the workload's FP32 byte model scaled to "
            "the sample volume" % (cores, RESTART, applies))


def cpu_baseline(applies, target_s=2.0):
    pool = OraclePool()
    try:
        reps, el = pool.round(applies, target_s)
    finally:
        pool.close()
    return {"value": round(reps * sample_step_bytes(applies) / el / 1e9, 3), "unit": "GB/s", "cores": pool.cores,
            "threads": pool.cores, "kind": "oracle",
            "sample": sample_description(pool.cores, applies) + "; %d steps in %.1f s" % (reps, el)}


def workload_config(applies):
    """config of the default workload (both arms)."""
    V, Vb, Vc, nc = geometry()
    step_bytes, parts = bytes_model(applies, arnoldi_iterations(applies))
    return {"workload": WORKLOAD, "L": list(L), "B": list(B), "ntv": NTV, "nrhs": 1,
            "coarse_solve": "FGMRES(%d) to %g, max %d applies" % (RESTART, TOL, MAX_APPLIES),
            "applies_per_step": applies, "bytes_per_step": step_bytes,
            "l2": "inputs larger than L2 (R %.2f GB, D_c %.2f GB) and a 256 MB flush before each step"
                  % (parts["restrict"] / 1e9, Vc * 9 * nc * nc * 8 / 1e9),
            "parallelism": "single"}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return None, rank
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.round(APPLIES_PER_STEP, 0.0)
        steps = [pool.round(APPLIES_PER_STEP, 0.0) for _ in range(args.steps)]
    finally:
        pool.close()
    reps = sum(r for r, _ in steps)
    tot = sum(t for _, t in steps)
    value = reps * sample_step_bytes(APPLIES_PER_STEP) / tot / 1e9
    cfg = workload_config(APPLIES_PER_STEP)
    cfg["parallelism"] = "replicas" if world > 1 else "single"
    res = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1000 * tot / max(1, len(steps)), 2),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": pool.cores, "threads": pool.cores,
                         "kind": "oracle",
                         "sample": sample_description(pool.cores, APPLIES_PER_STEP)
                         + "; one sample step per core per timed step"},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return res, rank


def _kernel_time(fn, n, stream):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for _ in range(3):
        fn()
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / n / 1000.0


def _timed_steps(step, steps, warmup, stream, flush=None):
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with Clocks(torch.cuda.current_device()) as clk:
        for a, b in ev:
            if flush is not None:
                flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / 1000.0, clk.summary()


def run_vcycle(args):
    """The two-level method on the default workload's lattice (32^4, 4^4 blocks, Ntv = 20, FP32
    vectors, FP32 R and D_c): one V-cycle (Alg. 1) = the coarse-grid correction (FGMRES(30) to 0.05)
    followed by 4 SAP cycles (Alg. 3) of 4 MR steps per block; the fine Wilson-clover D on its own;
    and the outer FGMRES(30) preconditioned with the V-cycle to relative residual 1e-5 (Sec. 1).

    Algorithmic bytes (FP32 complex = 8 B) per fine site: D reads 4 links (288 B), the clover
    (two Hermitian 6x6 blocks as upper triangles, 336 B), psi (96 B) and writes out (96 B) = 816 B;
    one SAP half sweep reads, per site of its colour, the links, the clover, y and x and writes x
    (912 B), and reads x on the other colour's sites once (96 B): 504 B per fine site of the
    lattice."""
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd
    n_smoother, n_mr = 4, 4
    V, Vb, Vc, nc = geometry()
    st = torch.cuda.current_stream()
    U = sd.links(SEED, EPS, L)
    tv = sd.test_vectors(SEED, NTV, L)
    p = amg.make_params(L, B, NTV, 1, M0, CSW, amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32)
    h, _ = amg.amg_setup_coarse(p, U, tv, st)
    amg.amg_setup_fine(h, U, st)
    del U, tv
    torch.cuda.empty_cache()
    vp = amg.make_vcycle_params(coarse_tol=TOL, coarse_restart=RESTART, coarse_max_applies=MAX_APPLIES,
                                n_smoother=n_smoother, n_mr=n_mr)
    y = sd.fine_rhs(SEED, 1, L, torch.complex64)
    x = torch.empty_like(y)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    info = amg.amg_cgc(h, y, x, 1, TOL, RESTART, MAX_APPLIES, st, info=True)
    applies = info[0][0]
    t, clk = _timed_steps(lambda: amg.amg_vcycle(h, vp, y, x, 1, st), args.steps, args.warmup, st, flush)
    t_d = _kernel_time(lambda: amg.amg_dirac_apply(h, y, x, 1, st), 20, st)
    t_sap = _kernel_time(lambda: amg.amg_sap(h, y, x, 1, 1, n_mr, st), 10, st) / 2  # one half sweep
    u = torch.empty_like(y)
    t0 = time.perf_counter()
    sinfo = amg.amg_solve(h, vp, y, u, 1, tol=1e-5, restart=30, max_applies=200, stream=st)
    t_solve = time.perf_counter() - t0
    # Three levels: the coarse lattice in 2^4 blocks (Ntv2 = 8 random level-1 test vectors), one
    # two-grid cycle on level 1 (2 MR steps on D_c before and after, level-2 FGMRES(30) to 0.05) in
    # place of the coarse FGMRES of every V-cycle.
    B2, ntv2, n_mr2 = (2, 2, 2, 2), 8, 2
    Lc = tuple(L[m] // B[m] for m in range(4))
    tv2 = sd.coarse_vector(SEED + 2, NTV, ntv2, Vc, torch.complex128)
    p2 = amg.make_params(Lc, B2, ntv2, 1, M0, CSW, amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2, _ = amg.amg_setup_level2(h, p2, tv2, st)
    t_setup2 = time.perf_counter() - t0
    del tv2
    amg.amg_attach_level2(h, h2, amg.make_level2_params(n_mr=n_mr2, restart=RESTART, max_applies=MAX_APPLIES,
                                                        tol=TOL))
    t3, _ = _timed_steps(lambda: amg.amg_vcycle(h, vp, y, x, 1, st), args.steps, args.warmup, st, flush)
    t0 = time.perf_counter()
    sinfo3 = amg.amg_solve(h, vp, y, u, 1, tol=1e-5, restart=30, max_applies=200, stream=st)
    t_solve3 = time.perf_counter() - t0
    amg.amg_attach_level2(h, None)
    status = amg.amg_sync_status(h)
    if status == amg.AMG_OK:
        status = amg.amg_sync_status(h2)
    amg.amg_destroy(h2)
    amg.amg_destroy(h)
    if status != amg.AMG_OK:
        raise RuntimeError(amg.amg_status_string(status))
    d_bytes = V * 816
    half_bytes = V * 504
    cgc_bytes, _ = bytes_model(applies, arnoldi_iterations(applies))
    step_bytes = cgc_bytes + 2 * n_smoother * half_bytes
    peaks, src = measured_peaks()
    d_gbs = d_bytes / t_d / 1e9
    sap_gbs = half_bytes / t_sap / 1e9
    ms = 1000 * t / args.steps
    return {
        "value": round(step_bytes * args.steps / t / 1e9, 2), "unit": "GB/s", "ms_per_step": round(ms, 4),
        "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
        "config": {"workload": "vcycle_32^4_b4_ntv20: one V-cycle (Alg. 1) on the default workload: CGC "
                               "(FGMRES(30) to 0.05) + %d SAP cycles of %d MR steps per 4^4 block; FP32" % (n_smoother, n_mr),
                   "bytes_per_step": step_bytes, "coarse_applies": applies, "n_smoother": n_smoother, "n_mr": n_mr,
                   "l2": "256 MB flush before each step"},
        "roofline": {"bound": "hbm", "kernel": "sap_smem_kernel (one half sweep: residual + %d MR steps per block, "
                     "links and clover in shared memory)" % n_mr, "achieved": round(sap_gbs, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(sap_gbs / peaks["hbm_gbs"], 4), "peak_source": src,
                     "traffic": round(SAP_TRAFFIC_RATIO * half_bytes) if SAP_TRAFFIC_RATIO and not args.lattice else None,
                     "traffic_note": "16^4 capture's traffic / algorithmic bytes x this launch's bytes",
                     "bytes_per_launch": half_bytes, "avg_launch_us": round(t_sap * 1e6, 2),
                     "step_share": round(2 * n_smoother * t_sap / (t / args.steps), 3)},
        "kernels": {"dirac": {"us": round(t_d * 1e6, 1), "GB/s": round(d_gbs, 1),
                              "frac": round(d_gbs / peaks["hbm_gbs"], 4), "bytes_per_launch": d_bytes},
                    "sap_half_sweep": {"us": round(t_sap * 1e6, 1), "GB/s": round(sap_gbs, 1),
                                       "frac": round(sap_gbs / peaks["hbm_gbs"], 4)}},
        "outer_solve": {"tol": 1e-5, "applies_of_D": sinfo[0][0], "relres": sinfo[0][1],
                        "seconds": round(t_solve, 4), "restart": 30},
        "three_level": {"level2": "%dx%dx%dx%d coarse lattice in 2^4 blocks -> %dx%dx%dx%d, Ntv2 = %d random level-1 "
                                  "test vectors" % (Lc + tuple(Lc[m] // B2[m] for m in range(4)) + (ntv2,)),
                        "cycle": "one two-grid cycle on level 1 per V-cycle: %d MR steps on D_c before and after, "
                                 "level-2 FGMRES(%d) to %g" % (n_mr2, RESTART, TOL),
                        "setup2_ms": round(1000 * t_setup2, 2), "vcycle_ms": round(1000 * t3 / args.steps, 4),
                        "outer_solve": {"tol": 1e-5, "applies_of_D": sinfo3[0][0], "relres": sinfo3[0][1],
                                        "seconds": round(t_solve3, 4), "restart": 30}},
        "clocks": clk,
    }


def run_mrhs(args):
    """Coarse applications with many right-hand sides at 32^3 x 64, 4^4 blocks (8^3 x 16 coarse
    sites), Ntv = 24: FP32 D_c and FP16 D_c with block scales, 16 and 4 columns, one pass on the
    tensor cores (tcgen05).  Algorithmic bytes: D_c once (FP32: 8 B per complex entry; FP16: 4 B
    plus one FP32 scale per block) and the input and output coarse vectors (FP32)."""
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd
    Lt, ntv, seed = (32, 32, 32, 64), 24, 20151204 + 3
    if args.lattice:
        Lt = tuple(int(v) for v in args.lattice.split(","))
    Vc = int(np.prod(Lt)) // int(np.prod(B))
    nc = 2 * ntv
    st = torch.cuda.current_stream()
    peaks, src = measured_peaks()
    kern, t_total, bytes_total, steps = {}, 0.0, 0, 0
    clk = None
    for name, link, eb, extra in (("fp32", amg.AMG_FP32, 8, 0), ("fp16", amg.AMG_FP16_SCALED, 4, Vc * 9 * 4)):
        U = sd.links(seed, EPS, Lt)
        tv = sd.test_vectors(seed, ntv, Lt)
        h, _ = amg.amg_setup_coarse(amg.make_params(Lt, B, ntv, 16, M0, CSW, link, amg.AMG_FP32, amg.AMG_FP32),
                                    U, tv, st)
        del U, tv
        torch.cuda.empty_cache()
        for nrhs in (16, 4):
            x = sd.coarse_vector(seed + nrhs, ntv, nrhs, Vc, torch.complex64)
            y = torch.empty_like(x)
            t, clk = _timed_steps(lambda: amg.amg_coarse_apply(h, x, y, nrhs, st), args.steps, args.warmup, st)
            b = Vc * 9 * nc * nc * eb + extra + 2 * Vc * nc * nrhs * 8
            us = 1e6 * t / args.steps
            kern["%s_%d" % (name, nrhs)] = {"us": round(us, 1), "GB/s": round(b / us / 1e3, 1),
                                            "frac": round(b / us / 1e3 / peaks["hbm_gbs"], 4), "bytes_per_launch": b}
            t_total += t
            bytes_total += b * args.steps
            steps += args.steps
        status = amg.amg_sync_status(h)
        amg.amg_destroy(h)
        if status != amg.AMG_OK:
            raise RuntimeError(amg.amg_status_string(status))
    dom = kern["fp32_16"]
    return {
        "value": round(bytes_total / t_total / 1e9, 2), "unit": "GB/s",
        "ms_per_step": round(1000 * t_total / steps, 4), "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
        "config": {"workload": ("mrhs_32^3x64_b4_ntv24: D_c x_c with 16 and 4 columns, FP32 and FP16-scaled "
                                "D_c, tcgen05 one-pass apply; inputs larger than L2 (FP32 D_c 1.36 GB)")
                               if Lt == (32, 32, 32, 64) else "%dx%dx%dx%d variant of mrhs" % Lt},
        "roofline": {"bound": "hbm", "kernel": "apply_tc5_kernel<48, true> (FP32 D_c, 16 columns)",
                     "achieved": dom["GB/s"], "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": dom["frac"],
                     "peak_source": src, "traffic": TRAFFIC_MRHS_FP32 if Lt == (32, 32, 32, 64) else None,
                     "bytes_per_launch": dom["bytes_per_launch"], "avg_launch_us": dom["us"]},
        "kernels": kern, "clocks": clk,
    }


def run_tc16(args):
    """48^3 x 96, 4^4 blocks (12^3 x 24 coarse), Ntv = 24, 16 right-hand sides, BF16 tensor cores.

    Step: restriction of 16 BF16 right-hand sides, FGMRES(30) to 0.05 on the BF16 D_c (all 16
    right-hand sides), prolongation to BF16; the same byte accounting as the default workload
    (BF16 R and D_c: 4 B per complex entry; fine vectors BF16, coarse vectors FP32)."""
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd
    Lt, ntv, nrhs, seed = (48, 48, 48, 96), 24, 16, 20151204 + 4
    if args.lattice:
        Lt = tuple(int(v) for v in args.lattice.split(","))
    V = int(np.prod(Lt))
    Vb = int(np.prod(B))
    Vc = V // Vb
    nc = 2 * ntv
    st = torch.cuda.current_stream()
    U = sd.links(seed, EPS, Lt)
    tv = sd.test_vectors(seed, ntv, Lt)
    p = amg.make_params(Lt, B, ntv, nrhs, M0, CSW, amg.AMG_BF16, amg.AMG_BF16, amg.AMG_BF16,
                        setup_arith=amg.AMG_SETUP_F32PAIR)
    h, _ = amg.amg_setup_coarse(p, U, tv, st)
    setup_ms = amg.amg_setup_timings(h)
    del U, tv
    torch.cuda.empty_cache()
    y32 = sd.fine_rhs(seed, nrhs, Lt, torch.complex64)
    y = torch.view_as_real(y32).to(torch.bfloat16)
    del y32
    torch.cuda.empty_cache()
    x = torch.empty_like(y)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    info = amg.amg_cgc(h, y, x, nrhs, TOL, RESTART, MAX_APPLIES, st, info=True)
    applies = max(a for a, _ in info)
    t, clk = _timed_steps(lambda: amg.amg_cgc(h, y, x, nrhs, TOL, RESTART, MAX_APPLIES, st, info=False),
                          args.steps, args.warmup, st, flush)
    Rb = Vc * 2 * ntv * 6 * Vb * 4
    vf = V * 12 * nrhs * 4
    vc = Vc * nc * nrhs * 8
    parts = {"restrict": Rb + vf + vc, "prolong": Rb + vc + vf, "apply": Vc * 9 * nc * nc * 4 + 2 * vc}
    flops = {"restrict": 8.0 * Vc * 2 * ntv * 6 * Vb * nrhs, "prolong": 8.0 * Vc * 2 * ntv * 6 * Vb * nrhs,
             "apply": 8.0 * Vc * 9 * nc * nc * nrhs}
    gs = sum((2 * (j + 1) + 4) * vc for j in arnoldi_iterations(applies))
    step_bytes = parts["restrict"] + parts["prolong"] + applies * parts["apply"] + gs
    yc = torch.empty((Vc, 2, ntv, nrhs), dtype=torch.complex64, device="cuda")
    zc = torch.empty_like(yc)
    amg.amg_restrict(h, y, yc, nrhs, st)
    tk = {"restrict": _kernel_time(lambda: amg.amg_restrict(h, y, yc, nrhs, st), 5, st),
          "apply": _kernel_time(lambda: amg.amg_coarse_apply(h, yc, zc, nrhs, st), 20, st),
          "prolong": _kernel_time(lambda: amg.amg_prolong(h, yc, x, nrhs, st), 5, st)}
    status = amg.amg_sync_status(h)
    amg.amg_destroy(h)
    if status != amg.AMG_OK:
        raise RuntimeError(amg.amg_status_string(status))
    peaks, src = measured_peaks()
    counts = {"restrict": 1, "prolong": 1, "apply": applies}
    dom = max(tk, key=lambda k: tk[k] * counts[k])
    kern = {k: {"us": round(tk[k] * 1e6, 1), "GB/s": round(parts[k] / tk[k] / 1e9, 1),
                "frac": round(parts[k] / tk[k] / 1e9 / peaks["hbm_gbs"], 4),
                "TFLOP/s": round(flops[k] / tk[k] / 1e12, 1),
                "tensor_frac": round(flops[k] / tk[k] / 1e12 / peaks["bf16_tflops"], 4)} for k in tk}
    return {
        "metric": METRIC, "value": round(step_bytes * args.steps / t / 1e9, 2), "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * t / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": ("tc16_48^3x96_b4_ntv24: 48^3x96 Wilson-clover, 4^4 blocks -> 12^3x24 coarse, "
                                "Ntv=24, 16 RHS, BF16 R / D_c / fine vectors on the tensor cores, FP32 "
                                "accumulation and coarse vectors; step = R Y, FGMRES(30) to 0.05, P X_c")
                               if Lt == (48, 48, 48, 96) else "%dx%dx%dx%d variant of tc16" % Lt,
                   "applies_per_step": applies, "bytes_per_step": step_bytes},
        "roofline": {"bound": "hbm", "kernel": TC16_KERNELS[dom], "achieved": kern[dom]["GB/s"],
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": kern[dom]["frac"], "peak_source": src,
                     "traffic": TRAFFIC_TC16.get(dom) if Lt == (48, 48, 48, 96) else None,
                     "bytes_per_launch": parts[dom], "avg_launch_us": kern[dom]["us"],
                     "step_share": round(tk[dom] * counts[dom] / (t / args.steps), 3)},
        "kernels": kern, "setup_ms": setup_report(setup_ms, V, ntv), "clocks": clk,
    }


def run_fp16(args):
    """32^3 x 64, 4^4 blocks (8^3 x 16 coarse), Ntv = 24, FP16 D_c with per-block FP32 scales, one
    right-hand side: 200 D_c applications of FGMRES(30) (tolerance 0 so the budget is spent);
    error of one FP16 application against the FP64 application of the same D_c."""
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd
    Lt, ntv, seed = (32, 32, 32, 64), 24, 20151204 + 3
    Vc = int(np.prod(Lt)) // int(np.prod(B))
    nc = 2 * ntv
    st = torch.cuda.current_stream()
    U = sd.links(seed, EPS, Lt)
    tv = sd.test_vectors(seed, ntv, Lt)
    h16, _ = amg.amg_setup_coarse(amg.make_params(Lt, B, ntv, 1, M0, CSW, amg.AMG_FP16_SCALED, amg.AMG_FP32,
                                                  amg.AMG_FP32), U, tv, st)
    h64, _ = amg.amg_setup_coarse(amg.make_params(Lt, B, ntv, 1, M0, CSW, amg.AMG_FP64, amg.AMG_FP64,
                                                  amg.AMG_FP64), U, tv, st)
    del U, tv
    b = sd.coarse_vector(seed, ntv, 1, Vc, torch.complex64)
    x = torch.empty_like(b)
    y16 = torch.empty_like(b)
    y64 = torch.empty((Vc, 2, ntv, 1), dtype=torch.complex128, device="cuda")
    amg.amg_coarse_apply(h16, b, y16, 1, st)
    amg.amg_coarse_apply(h64, b.to(torch.complex128), y64, 1, st)
    torch.cuda.synchronize()
    err = float((y16.to(torch.complex128) - y64).norm() / y64.norm())
    t, clk = _timed_steps(lambda: amg.amg_coarse_solve(h16, b, x, 1, 0.0, RESTART, 200, st, info=False),
                          args.steps, args.warmup, st)
    apply_bytes = Vc * 9 * nc * nc * 4 + Vc * 9 * 4 + 2 * Vc * nc * 8
    ta = _kernel_time(lambda: amg.amg_coarse_apply(h16, b, y16, 1, st), 50, st)
    gs = sum((2 * (j + 1) + 4) * Vc * nc * 8 for j in arnoldi_iterations(200))
    step_bytes = 200 * apply_bytes + gs
    amg.amg_destroy(h16)
    amg.amg_destroy(h64)
    peaks, src = measured_peaks()
    return {
        "metric": METRIC, "value": round(step_bytes * args.steps / t / 1e9, 2), "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * t / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": "fp16_32^3x64_b4_ntv24: 8^3x16 coarse, Ntv=24, FP16 D_c + FP32 scale per "
                               "block, 1 RHS; step = 200 D_c applications of FGMRES(30)",
                   "bytes_per_step": step_bytes, "fp16_apply_rel_error_vs_fp64": err},
        "roofline": {"bound": "hbm", "kernel": "apply_mrhs_kernel<__half2,1> (D_c x_c, FP16 D_c + block scales)",
                     "achieved": round(apply_bytes / ta / 1e9, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(apply_bytes / ta / 1e9 / peaks["hbm_gbs"], 4), "peak_source": src,
                     "traffic": TRAFFIC_FP16_APPLY, "bytes_per_launch": apply_bytes,
                     "avg_launch_us": round(ta * 1e6, 2), "step_share": round(200 * ta / (t / args.steps), 3)},
        "clocks": clk,
    }


def run_batch(args):
    """The uneven batch in one persistent launch, captured in a CUDA graph: lattices 16^4 (Ntv=16,
    1 RHS), 24^3 x 48 (Ntv=20, 4 RHS), 32^3 x 64 (Ntv=24, 12 RHS), 4^4 blocks, eps 0.2 / 0.3 / 0.4;
    step = x_k = P_k D_ck R_k y_k for all three; launch shape from the autotuner.  Precision
    (--batch-precision): "mixed" = the 1-RHS lattice in FP32, the multi-RHS lattices in BF16 on the
    tensor cores (BF16 R, D_c and fine vectors); "fp32" = all FP32.  Algorithmic bytes in the
    storage precision of each lattice (BF16 rows of y_c: 4 B per complex entry)."""
    import torch
    import paper_1512_04506_gb300 as amg
    from synth import device as sd
    spec = [((16, 16, 16, 16), 16, 1, 0.2), ((24, 24, 24, 48), 20, 4, 0.3), ((32, 32, 32, 64), 24, 12, 0.4)]
    if args.lattice == "small":  # the three lattices at 1/2, 1/4 and 1/4 of the volume, for ncu captures
        spec = [((8, 16, 16, 16), 16, 1, 0.2), ((24, 24, 12, 24), 20, 4, 0.3), ((16, 32, 32, 32), 24, 12, 0.4)]
    st = torch.cuda.current_stream()
    hs, ys, xs, nr = [], [], [], []
    step_bytes = 0
    precs = []
    for k, (Lk, ntv, nrhs, eps) in enumerate(spec):
        seed = 20151204 + 5 + 10 * k
        U = sd.links(seed, eps, Lk)
        tv = sd.test_vectors(seed, ntv, Lk)
        bf = args.batch_precision == "mixed" and nrhs in (4, 8, 12, 16)
        pr = amg.AMG_BF16 if bf else amg.AMG_FP32
        h, _ = amg.amg_setup_coarse(amg.make_params(Lk, B, ntv, nrhs, M0, CSW, pr, pr, pr), U, tv, st)
        del U, tv
        y = sd.fine_rhs(seed, nrhs, Lk, torch.complex64)
        if bf:
            y = torch.view_as_real(y).to(torch.bfloat16)
            torch.cuda.empty_cache()
        hs.append(h)
        ys.append(y)
        xs.append(torch.empty_like(y))
        nr.append(nrhs)
        precs.append("bf16" if bf else "fp32")
        V = int(np.prod(Lk))
        Vc = V // int(np.prod(B))
        nc = 2 * ntv
        e = 4 if bf else 8  # bytes per complex entry of R, D_c, fine vectors and y_c
        step_bytes += 2 * Vc * 2 * ntv * 6 * int(np.prod(B)) * e + 2 * V * 12 * nrhs * e \
            + Vc * 9 * nc * nc * e + 2 * Vc * nc * nrhs * e + 2 * Vc * nc * nrhs * 8
    torch.cuda.empty_cache()
    amg.amg_batch_cgc(hs, ys, xs, nr, st)
    best = amg.amg_batch_autotune(hs, ys, xs, nr, st) if not args.no_autotune else None
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(st)
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            amg.amg_batch_cgc(hs, ys, xs, nr, s2)
    st.wait_stream(s2)
    t, clk = _timed_steps(g.replay, args.steps, args.warmup, st)
    status = amg.amg_sync_status(hs[0])
    for h in hs:
        amg.amg_destroy(h)
    if status != amg.AMG_OK:
        raise RuntimeError(amg.amg_status_string(status))
    peaks, src = measured_peaks()
    gbs = step_bytes * args.steps / t / 1e9
    return {
        "metric": METRIC, "value": round(gbs, 2), "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1000 * t / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32" if "bf16" in precs else "f32",
        "data": "synthetic",
        "config": {"workload": ("batch: 16^4 (Ntv 16, 1 RHS) + 24^3x48 (Ntv 20, 4 RHS) + 32^3x64 (Ntv 24, "
                                "12 RHS), 4^4 blocks; one persistent launch per step, CUDA graph; inputs "
                                "larger than L2") if args.lattice != "small" else "reduced-volume variant of batch",
                   "precision": dict(zip(["16^4", "24^3x48", "32^3x64"], precs)),
                   "bytes_per_step": step_bytes,
                   "autotuned_ms": round(best, 4) if best is not None else "default launch shape"},
        "roofline": {"bound": "hbm", "kernel": "batch_kernel<true> (fused R, D_c, P over the three lattices)",
                     "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(gbs / peaks["hbm_gbs"], 4), "peak_source": src,
                     "traffic": round(BATCH_TRAFFIC_RATIO * step_bytes) if args.lattice != "small" else None,
                     "traffic_note": "reduced-volume capture's traffic / algorithmic bytes x this launch's bytes",
                     "bytes_per_launch": step_bytes, "avg_launch_us": round(1e6 * t / args.steps, 2),
                     "step_share": 1.0},
        "clocks": clk,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-speedup", action="store_true",
                    help="skip the batched-mixed vs plain FP32 coarse-solve comparison")
    ap.add_argument("--workload", default="fp32", choices=["fp32", "tc16", "fp16", "mrhs", "batch", "vcycle"],
                    help="fp32: the default 32^4 workload; tc16: 48^3x96 with 16 RHS on the tensor cores; "
                         "fp16: 200 FP16 coarse applications at 32^3x64; batch: the uneven batch")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch workload: keep the default launch shape (for ncu captures of it)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default workload: skip the tc16, fp16 and batch sub-objects")
    ap.add_argument("--no-evenodd", action="store_true",
                    help="skip the even/odd-reduced coarse solve comparison of the default workload")
    ap.add_argument("--batch-precision", default="mixed", choices=["mixed", "fp32"],
                    help="batch workload: BF16 tensor cores for the multi-RHS lattices (mixed) or all FP32")
    ap.add_argument("--lattice", default=None,
                    help="Lx,Ly,Lz,Lt override of the 32^4 lattice (smaller cases for ncu captures); "
                         "'small' for the batch workload")
    args = ap.parse_args()
    if args.lattice and args.workload != "batch":
        global L, WORKLOAD
        L = tuple(int(v) for v in args.lattice.split(","))
        WORKLOAD = "%dx%dx%dx%d variant of %s" % (L + (WORKLOAD,))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        res, rank = run_reference(args)
    elif args.workload == "tc16":
        res, rank = run_tc16(args), 0
    elif args.workload == "fp16":
        res, rank = run_fp16(args), 0
    elif args.workload == "batch":
        res, rank = run_batch(args), 0
    elif args.workload == "vcycle":
        res, rank = run_vcycle(args), 0
    elif args.workload == "mrhs":
        res, rank = run_mrhs(args), 0
    else:
        res, rank = run_gpu(args)
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
