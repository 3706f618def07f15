"""Benchmark: Tucker-compressed FMM aggregation + disaggregation on one GB300.

One step = one aggregation (Fig. 2b) + one disaggregation (Fig. 3b) of every
group of the workload, i.e. one far-field matvec without the translation
stage.  Default workload: PEC sphere of diameter 30 lambda (icosphere nu = 180:
648,000 triangles, 972,000 RWGs), 2-lambda boxes, 6-digit FMM (L = 39, 40 x 80
directions), Tucker tolerance 1e-6, one CN(0, 1) right-hand side.

Printed (rank 0, one JSON line): ms per matvec of the Tucker path with inputs
resident in HBM (`value`), the same through the host-buffer C-ABI call (`e2e`),
the dense-far-field comparator on the same GPU, the roofline of the dominant
kernel, the FP64 oracle timed on the host cores (`cpu_baseline`) and the SM
clocks seen during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sphere30] [--no-dense] [--no-cpu-baseline]
Under torchrun every rank runs an independent replica on its own GPU (the
aggregation / disaggregation of one problem needs no exchange between GPUs).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agg+disagg ms/matvec & HBM GB/s: Tucker vs dense far-fields, 1 GB300, rel err≤1e-6"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere30")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-groups", type=int, default=5)
    ap.add_argument("--graph", dest="graph", action="store_true", default=True,
                    help="replay one captured CUDA graph of the two stages per step (default)")
    ap.add_argument("--no-graph", dest="graph", action="store_false", help="launch the two stages eagerly per step")
    ap.add_argument("--sweep", action="store_true",
                    help="parameter sweep on the 20-lambda sphere (box x tolerance x digits, 16 RHS): "
                         "one JSON line per point")
    ap.add_argument("--sweep-boxes", default="0.5,1,2,4")
    ap.add_argument("--sweep-tols", default="1e-3,1e-4,1e-6,1e-8")
    ap.add_argument("--sweep-digits", default="3,6")
    ap.add_argument("--translate", action="store_true",
                    help="also time the translation stage (FMM-FFT, tfmm_translate) between the two stages and "
                         "report the far-field matvec aggregate -> translate -> disaggregate")
    ap.add_argument("--svd", action="store_true",
                    help="also build the truncated-SVD comparator (Sec. II.C) of the workload and time it: "
                         "the Table III analogue (dense / SVD / Tucker memory and ms) on one GPU")
    ap.add_argument("--tuning", default="",
                    help="KEY=VALUE[,KEY=VALUE...] fields of tfmm_tuning set on the plan before timing "
                         "(e.g. dis_threads=384,dis_ctas_per_sm=2)")
    ap.add_argument("--mrhs-precision", type=int, default=None,
                    help="R > 1: 0 FP32 CUDA cores, 2 / 3 tensor cores with 2- / 3-term split BF16 (default 3)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def whole_job_ms(total_ms, steps, world, device=None):
    """The slowest replica's timed total (max over ranks) and the whole job's ms per matvec.

    Replicas run side by side, one per GPU, each doing one matvec per step, so the job
    finishes steps * world matvecs in the slowest rank's time.
    """
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, total_ms / (steps * world)


def workload_desc(w, L=None, n_theta=None, n_phi=None, G=None):
    if w.shape == "trihedral":
        d = (f"PEC square trihedral corner reflector, {w.diameter:g}-lambda plates, {w.nu}x{w.nu} squares per plate "
             f"({w.n_tri} triangles, {w.n_rwg} RWGs), {w.box:g}-lambda boxes, d0={w.digits} digits")
    else:
        d = (f"PEC sphere D={w.diameter:g} lambda, icosphere nu={w.nu} ({w.n_tri} triangles, {w.n_rwg} RWGs), "
             f"{w.box:g}-lambda boxes, d0={w.digits} digits")
    if L is not None:
        d += f" (L={L}, {n_theta}x{n_phi} directions, {G} groups)"
    if w.rhs == "planewave_sweep":
        d += f", Tucker tol {w.tol:g}, {w.nrhs} RWG-tested plane waves theta_inc = pi i/{w.nrhs - 1}, phi_inc = 0, theta-polarised"
    elif w.rhs == "planewave_corner":
        d += (f", N_phi = 2L+1, Tucker tol {w.tol:g}, RWG-tested plane wave theta_inc = 135 deg, phi_inc = 225 deg, "
              f"theta-polarised")
    else:
        d += f", Tucker tol {w.tol:g}, {w.nrhs} RHS CN(0,1) seed {w.seed}"
    return d


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def mark(self, on):
        self.marks.append((time.time(), on))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        windows = []
        for i in range(0, len(self.marks) - 1, 2):
            windows.append((self.marks[i][0], self.marks[i + 1][0]))
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if not any(a <= t <= b for a, b in windows):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------- cpu baseline
def size_quantile_groups(sizes, count):
    """Group ids at evenly spaced quantiles of the group size (smallest and largest included)."""
    order = np.argsort(np.asarray(sizes), kind="stable")
    q = np.linspace(0, len(order) - 1, max(count, 1)).round().astype(int)
    return sorted({int(order[i]) for i in q})


def oracle_sample(w, verts, tris, n_groups_sample, seed):
    """Oracle far-fields + T-HOSVD for a few groups of the workload (setup, untimed).

    The groups sit at evenly spaced quantiles of the group size, so that the
    per-group times span the whole size range the scaling below extrapolates over.
    """
    import oracle
    P = oracle.problem.build(verts, tris, k=2 * math.pi, box=w.box, digits=w.digits, tol=w.tol,
                             nphi_rule="2L+1" if w.nphi_rule == 0 else "2L+2", compress=False, keep_tensors=False)
    pick = size_quantile_groups([len(m) for m in P.groups.members], n_groups_sample)
    tuck, dense = {}, {}
    for g in pick:
        At, Ap = P.group_tensors(g)
        dense[g] = (At, Ap)
        tuck[g] = (oracle.hosvd.thosvd(At, w.tol), oracle.hosvd.thosvd(Ap, w.tol))
    x = None
    return P, pick, tuck, dense


def oracle_group_step(P, g, tuck, x):
    """Oracle Tucker aggregation + disaggregation of one group (complex128)."""
    from oracle import apply
    xg = x[P.groups.members[g]]
    F = [apply.tucker_aggregate(tuck[g][a], xg) for a in range(2)]
    return sum(apply.tucker_disaggregate(tuck[g][a], F[a], P.grid.weights) for a in range(2))


def scale_group_times(sizes_sample, times_sample, sizes_all):
    """Whole-problem time from per-group times of a size-quantile sample.

    Fits t = a + b n_beta by least squares over the sampled groups (the oracle's
    cost per group is affine in its size: the n_beta r_beta terms grow with n_beta,
    the core and angular terms do not) and sums the fit over every group.  Falls
    back to scaling by the groups' share of RWGs when the fit is degenerate.
    """
    n = np.asarray(sizes_sample, float)
    t = np.asarray(times_sample, float)
    N = np.asarray(sizes_all, float)
    if len(set(n.tolist())) >= 2:
        b, a = np.polyfit(n, t, 1)
        pred = a + b * N
        if np.all(pred > 0):
            return float(pred.sum())
    return float(t.sum() * N.sum() / n.sum())


def time_oracle(P, pick, tuck, x, steps, warmup, budget_s=None):
    """ms per whole-problem Tucker agg + disagg, extrapolated from the sampled groups."""
    for _ in range(warmup):
        for g in pick:
            oracle_group_step(P, g, tuck, x)
    per = {g: [] for g in pick}
    n = 0
    t0 = time.perf_counter()
    while True:
        for g in pick:
            s = time.perf_counter()
            oracle_group_step(P, g, tuck, x)
            per[g].append(time.perf_counter() - s)
        n += 1
        if budget_s is None and n >= steps:
            break
        if budget_s is not None and (time.perf_counter() - t0 >= budget_s and n >= 3):
            break
    sizes = [len(m) for m in P.groups.members]
    total_s = scale_group_times([sizes[g] for g in pick], [statistics.median(per[g]) for g in pick], sizes)
    return 1e3 * total_s, n


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        if info:
            return max(i.get("num_threads", 1) for i in info)
    except Exception:
        pass
    return os.cpu_count()


# ---------------------------------------------------------------- reference
def run_reference(args, w, world, rank):
    if rank != 0:
        return
    from paper_2103_05822_gb300.inputs import complex_gaussian, workload_mesh
    verts, tris = workload_mesh(w)
    P, pick, tuck, _ = oracle_sample(w, verts, tris, args.oracle_groups, w.seed)
    R = w.nrhs
    x = complex_gaussian((P.n_rwg, R) if R > 1 else P.n_rwg, w.seed)  # timing does not depend on the values
    ms, n = time_oracle(P, pick, tuck, x, args.steps, args.warmup)
    cores = cpu_threads()
    sample = (f"{len(pick)} of {P.groups.n_groups} groups at size quantiles (oracle far-field + T-HOSVD untimed); "
              f"median of {n} timings per group of Tucker agg+disagg of {R} column(s), extrapolated to every "
              f"group by a least-squares fit of time vs group size")
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "complex128", "data": "synthetic",
        "config": {"workload": workload_desc(w, P.grid.L, P.grid.n_theta, P.grid.n_phi, P.groups.n_groups)},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours
def launches_per_step(tfmm, plan, R, dev):
    """Kernels one aggregate + disaggregate pair launches: one persistent kernel per stage
    for one RHS (three per stage on the split path, taken by plans with fewer work items
    than twice the SMs), the tensor-core chain for many (operand prep and four kernels
    for aggregation, four for disaggregation)."""
    import torch
    t = tfmm.tfmm_plan_tuning_get(plan)
    if R == 1:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        split = t["single_rhs_split"] == 1 or (t["single_rhs_split"] == 0 and 2 * plan.info["n_groups"] < 2 * sms)
        return 6 if split else 2
    return 8


def traffic_record(kernel, factor_bytes):
    """DRAM bytes per launch from a committed ncu capture (scaled by the factor bytes streamed),
    if the kernel source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    src = os.path.join(ROOT, "paper_2103_05822_gb300", "csrc", "apply.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    ent = rec.get(kernel)
    if not ent or ent.get("apply_cu_sha256") != sha or "dram_bytes_per_factor_byte" not in ent:
        return None
    return round(ent["dram_bytes_per_factor_byte"] * factor_bytes)


def run_ours(args, w, world, rank, local):
    import torch
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import complex_gaussian, workload_mesh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    R = w.nrhs
    use_dense = not args.no_dense and R <= 8  # the dense comparator streams 16 N N_dir bytes per column
    verts, tris = workload_mesh(w)
    t0 = time.perf_counter()
    mesh = tfmm.tfmm_mesh_create(verts, tris)
    mp = args.mrhs_precision if args.mrhs_precision is not None else (3 if R > 1 else 0)
    prm = tfmm.tfmm_params_default(k=2 * math.pi, box=w.box, digits=float(w.digits), tol=w.tol, nphi_rule=w.nphi_rule,
                                   keep_dense=1 if use_dense else 0, max_rhs=R, mrhs_precision=mp)
    stream = torch.cuda.current_stream()
    plan = tfmm.tfmm_plan_create(mesh, prm, stream=stream)
    setup_s = time.perf_counter() - t0
    if args.tuning:
        kv = dict(item.split("=") for item in args.tuning.split(","))
        tfmm.tfmm_plan_tuning_set(plan, stream=stream, **{k.strip(): int(v) for k, v in kv.items()})
    info = plan.info
    N, G, nd = info["n_rwg"], info["n_groups"], info["n_dir"]

    if w.rhs == "planewave_sweep":
        th = np.pi * np.arange(R) / max(R - 1, 1)
        kh = np.stack([np.sin(th), np.zeros(R), np.cos(th)], axis=1)
        pol = np.stack([np.cos(th), np.zeros(R), -np.sin(th)], axis=1)
        xv = torch.empty((R, N), dtype=torch.complex64, device=dev)
        tfmm.tfmm_planewave(plan, kh, pol, xv, stream=stream)
        torch.cuda.synchronize()
        x_host = xv.cpu().numpy()
    elif w.rhs == "planewave_corner":
        # Sec. III.A: k_inc at theta = 135 deg, phi = 225 deg, theta-polarised
        th, ph = math.radians(135.0), math.radians(225.0)
        kh = np.array([[math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)]])
        pol = np.array([[math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)]])
        xv = torch.empty((1, N), dtype=torch.complex64, device=dev)
        tfmm.tfmm_planewave(plan, kh, pol, xv, stream=stream)
        torch.cuda.synchronize()
        x_host = xv.cpu().numpy().reshape(N)
    else:
        x_host = complex_gaussian((R, N) if R > 1 else N, w.seed).astype(np.complex64)
    x = torch.from_numpy(x_host).to(dev)
    spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device=dev)
    y = torch.empty((R, N) if R > 1 else N, dtype=torch.complex64, device=dev)

    def step_tucker(ev=None):
        if ev is not None:
            ev[0].record(stream)
        tfmm.tfmm_aggregate(plan, x, spec, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        tfmm.tfmm_disaggregate(plan, spec, y, stream=stream)
        if ev is not None:
            ev[2].record(stream)

    def step_dense(ev=None):
        if ev is not None:
            ev[0].record(stream)
        tfmm.tfmm_aggregate_dense(plan, x, spec, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        tfmm.tfmm_disaggregate_dense(plan, spec, y, stream=stream)
        if ev is not None:
            ev[2].record(stream)

    graph = None
    if args.graph:
        step_tucker()  # first call for this R builds the chain's problem lists and scratch
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            cap = torch.cuda.current_stream()
            tfmm.tfmm_aggregate(plan, x, spec, stream=cap)
            tfmm.tfmm_disaggregate(plan, spec, y, stream=cap)
        torch.cuda.synchronize()

        def step_graph(ev=None):
            if ev is not None:
                ev[0].record(stream)
            graph.replay()
            if ev is not None:
                ev[1].record(stream)
                ev[2].record(stream)

    def timed(step, K, W):
        for _ in range(W):
            step()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        clocks.mark(True)
        start.record(stream)
        for k in range(K):
            step(evs[k])
        end.record(stream)
        torch.cuda.synchronize()
        clocks.mark(False)
        barrier()
        total = start.elapsed_time(end)
        agg = [e[0].elapsed_time(e[1]) for e in evs]
        dis = [e[1].elapsed_time(e[2]) for e in evs]
        return total, agg, dis

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # untimed soak so that clocks settle under load
    for _ in range(max(args.warmup, 3)):
        step_tucker()
    torch.cuda.synchronize()

    total, agg, dis = timed(step_graph if graph is not None else step_tucker, args.steps, args.warmup)
    ms_step = total / args.steps
    if graph is not None:  # per-stage split from an eager pass
        _, agg, dis = timed(step_tucker, args.steps, args.warmup)
    total, value = whole_job_ms(total, args.steps, world, dev)

    dense = None
    if use_dense:
        dtot, dagg, ddis = timed(step_dense, args.steps, args.warmup)
        dense = {"ms_per_matvec": dtot / args.steps, "aggregate_ms": statistics.mean(dagg),
                 "disaggregate_ms": statistics.mean(ddis)}

    # end to end through the host-buffer C-ABI call: H2D x, agg, disagg, D2H y, sync
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty(x_host.shape, dtype=torch.complex64).pin_memory()
    for _ in range(args.warmup):
        tfmm.tfmm_matvec_host(plan, xh, yh, R=R, stream=stream)
    torch.cuda.synchronize()
    barrier()
    clocks.mark(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tfmm.tfmm_matvec_host(plan, xh, yh, R=R, stream=stream)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    clocks.mark(False)
    barrier()
    clocks.stop()

    # accuracy of this run against the dense-far-field GPU path (same x)
    rel = None
    if dense is not None:
        ref = torch.empty_like(spec)
        tfmm.tfmm_aggregate(plan, x, spec, stream=stream)
        tfmm.tfmm_aggregate_dense(plan, x, ref, stream=stream)
        torch.cuda.synchronize()
        rel = float(torch.linalg.vector_norm(spec - ref) / torch.linalg.vector_norm(ref))

    trans_rec = None
    if args.translate:
        spec_in = torch.empty_like(spec)
        t1 = time.perf_counter()
        tfmm.tfmm_translate(plan, spec, spec_in, stream=stream)  # first call builds the transform of T_L
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t1

        def step_far(ev=None):
            if ev is not None:
                ev[0].record(stream)
            tfmm.tfmm_aggregate(plan, x, spec, stream=stream)
            tfmm.tfmm_translate(plan, spec, spec_in, stream=stream)
            if ev is not None:
                ev[1].record(stream)
            tfmm.tfmm_disaggregate(plan, spec_in, y, stream=stream)
            if ev is not None:
                ev[2].record(stream)

        ftot, fa, fd = timed(step_far, args.steps, args.warmup)
        trans_rec = {"far_matvec_ms": ftot / args.steps, "aggregate_plus_translate_ms": statistics.mean(fa),
                     "disaggregate_ms": statistics.mean(fd), "build_s": build_s}
        trans_rec["translate_ms"] = trans_rec["aggregate_plus_translate_ms"] - statistics.mean(agg)
        del spec_in

    svd_rec = None
    if args.svd:
        # the same workload compressed by the truncated SVD of each aggregation matrix at gamma
        t1 = time.perf_counter()
        prm_s = tfmm.tfmm_params_default(k=2 * math.pi, box=w.box, digits=float(w.digits), tol=w.tol,
                                         nphi_rule=w.nphi_rule, keep_dense=0, max_rhs=R, compression=tfmm.SVD)
        plan_s = tfmm.tfmm_plan_create(mesh, prm_s, stream=stream)
        setup_svd = time.perf_counter() - t1
        spec_s = torch.empty_like(spec)

        def step_svd(ev=None):
            if ev is not None:
                ev[0].record(stream)
            tfmm.tfmm_aggregate(plan_s, x, spec_s, stream=stream)
            if ev is not None:
                ev[1].record(stream)
            tfmm.tfmm_disaggregate(plan_s, spec_s, y, stream=stream)
            if ev is not None:
                ev[2].record(stream)

        stot, sagg, sdis = timed(step_svd, args.steps, args.warmup)
        info_s = plan_s.info
        rel_s = None
        if dense is not None:
            ref = torch.empty_like(spec)
            tfmm.tfmm_aggregate(plan_s, x, spec_s, stream=stream)
            tfmm.tfmm_aggregate_dense(plan, x, ref, stream=stream)
            torch.cuda.synchronize()
            rel_s = float(torch.linalg.vector_norm(spec_s - ref) / torch.linalg.vector_norm(ref))
        sb = info_s["tucker_bytes_alg"]
        svd_rec = {"ms_per_matvec": stot / args.steps, "aggregate_ms": statistics.mean(sagg),
                   "disaggregate_ms": statistics.mean(sdis), "bytes": sb, "compression": 8 * 2 * N * nd / sb,
                   "aggregate_gbs": (sb + 8 * N * R + 16 * G * nd * R) / statistics.mean(sagg) / 1e6,
                   "max_rank_beta": info_s["max_rank"][2], "rel_err_vs_dense_gpu": rel_s, "setup_s": setup_svd}
        del plan_s, spec_s
        torch.cuda.empty_cache()

    # roofline of the dominant kernel (algorithmic bytes or flops per launch / mean launch time)
    fac = info["tucker_bytes_alg"]
    bytes_agg = fac + 8 * N * R + 16 * G * nd * R
    bytes_dis = fac + 16 * G * nd * R + 8 * N * R
    agg_ms, dis_ms = statistics.mean(agg), statistics.mean(dis)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    if R == 1:
        if agg_ms >= dis_ms:
            kern, ms_k, bytes_k = "tucker_aggregate_kernel", agg_ms, bytes_agg
        else:
            kern, ms_k, bytes_k = "tucker_disaggregate_kernel", dis_ms, bytes_dis
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = bytes_k / (ms_k * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "traffic": traffic_record(kern, fac), "algorithmic_bytes": bytes_k}
    else:
        # the R-column chains: complex multiply-adds of Figs. 2b / 3b, 8 real flops each
        cm = 0
        for g in range(G):
            for a in range(2):
                nb, (rt, rp, rb) = tfmm.tfmm_plan_group(plan, g, a)
                cm += nb * rb + rt * rp * rb + info["n_phi"] * rp * rt + nd * rt
        flops = 8.0 * cm * R
        side = "aggregate" if agg_ms >= dis_ms else "disaggregate"
        ms_k = max(agg_ms, dis_ms)
        achieved = flops / (ms_k * 1e-3) / 1e12
        if mp in (2, 3):
            # split-BF16 on tcgen05: each complex product is 4 real MMAs per retained term pair
            products = 3 if mp == 2 else 6
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            roof = {"bound": "tensor", "kernel": f"tc_gemm_kernel<{mp},*> ({side} chain)", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "measured bf16 sustained" if "bf16_tflops_sustained" in peaks else "fallback",
                    "executed_tensor_tflops": achieved * products,
                    "frac_executed": achieved * products / peak,
                    "traffic": None, "algorithmic_flops": flops, "algorithmic_bytes": bytes_agg}
        else:
            sm_clock = 2.07e9
            peak = 152 * 128 * 2 * sm_clock / 1e12  # FP32 FMA lanes x 2 flops x max SM clock
            roof = {"bound": "alu", "kernel": f"mr_gemm_kernel ({side} chain)", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flops x 2.07 GHz",
                    "traffic": None, "algorithmic_flops": flops, "algorithmic_bytes": bytes_agg}

    cpu = None
    err_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        P, pick, tuck, dense_o = oracle_sample(w, verts, tris, args.oracle_groups, w.seed)
        xo = x_host.astype(np.complex128)
        xo = xo.T if R > 1 else xo  # the oracle takes columns
        # the spectra of the timed run on the sampled groups against the oracle's own FP64
        # far-fields and dense Eq. 3, per right-hand side
        from oracle import apply as oapply
        idx = torch.tensor(pick, device=dev)
        got = spec.index_select(1, idx).cpu().numpy()  # (R, len(pick), 2, N_dir)
        worst = 0.0
        for r in range(R):
            num = den = 0.0
            xr = xo[:, r] if R > 1 else xo
            for k, g in enumerate(pick):
                xg = xr[P.groups.members[g]]
                for a in range(2):
                    ref = oapply.dense_aggregate(dense_o[g][a], xg)
                    num += float(np.sum(np.abs(got[r, k, a] - ref) ** 2))
                    den += float(np.sum(np.abs(ref) ** 2))
            worst = max(worst, math.sqrt(num / den))
        err_oracle = {"max_per_rhs": worst, "groups": pick,
                      "what": "aggregation spectra vs the oracle's FP64 far-fields and dense Eq. 3"}
        ms_cpu, n = time_oracle(P, pick, tuck, xo, 0, 1, budget_s=10.0)
        cpu = {"value": ms_cpu, "unit": "ms", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{len(pick)} of {G} groups at size quantiles, oracle Tucker agg+disagg (complex128) "
                         f"timed {n} times per group (~10 s), extrapolated to every group by a least-squares "
                         f"fit of time vs group size; oracle setup untimed"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
            "config": {"workload": workload_desc(w, info["L"], info["n_theta"], info["n_phi"], G),
                       "l2": ("no flush: Tucker factors ({:.2f} GB) exceed the 129 MB L2".format(fac / 1e9) if fac > 129e6
                              else "Tucker factors ({:.3f} GB) fit in the 129 MB L2: no flush, timings are "
                                   "L2-resident".format(fac / 1e9)),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "stages": {"aggregate_ms": agg_ms, "disaggregate_ms": dis_ms,
                       "aggregate_gbs": bytes_agg / agg_ms / 1e6, "disaggregate_gbs": bytes_dis / dis_ms / 1e6},
            "dense": dense,
            "speedup_vs_dense": (dense["ms_per_matvec"] / ms_step) if dense else None,
            "svd": svd_rec,
            "translation": trans_rec,
            "rel_err_vs_dense_gpu": rel, "rel_err_vs_oracle": err_oracle,
            "memory": {"tucker_bytes": info["tucker_bytes"], "tucker_bytes_alg": fac,
                       "dense_bytes": 8 * 2 * N * nd, "compression": 8 * 2 * N * nd / fac,
                       "max_rank": info["max_rank"], "max_n_beta": info["max_n_beta"]},
            "setup_s": setup_s, "setup_ms": info["setup_ms"],
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 8 * N * R, "d2h_bytes_per_step": 8 * N * R},
            "gpu_launches": launches_per_step(tfmm, plan, R, dev) * args.steps,
            "nrhs": R, "graph": bool(args.graph), "mrhs_precision": mp if R > 1 else None,
            "tuning": tfmm.tfmm_plan_tuning_get(plan),
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep(args):
    """Box size x Tucker tolerance x digits on the 20-lambda sphere with 16 CN(0,1) RHS.

    Per point: setup, autotuner (R = 16), event-timed aggregation + disaggregation,
    compression, roofline fractions, and the per-RHS error of the aggregation against the
    oracle's own FP64 far-fields and dense Eq. 3 on the two smallest groups.
    """
    import torch
    import oracle
    from oracle import apply
    from paper_2103_05822_gb300 import tfmm
    from paper_2103_05822_gb300.inputs import WORKLOADS, complex_gaussian, icosphere
    w = WORKLOADS["sphere20_sweep"]
    R = w.nrhs
    verts, tris = icosphere(w.diameter, w.nu)
    mesh = tfmm.tfmm_mesh_create(verts, tris)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    tensor = peaks.get("bf16_tflops_sustained", 1700.0)
    fp32 = 152 * 128 * 2 * 2.07e9 / 1e12
    stream = torch.cuda.current_stream()
    oracle_cache = {}
    boxes = [float(v) for v in args.sweep_boxes.split(",")]
    tols = [float(v) for v in args.sweep_tols.split(",")]
    digits = [int(v) for v in args.sweep_digits.split(",")]
    for d0 in digits:
        for box in sorted(boxes):
            for tol in sorted(tols, reverse=True):
                t0 = time.perf_counter()
                prm = tfmm.tfmm_params_default(k=2 * math.pi, box=box, digits=float(d0), tol=tol, max_rhs=R,
                                               mrhs_precision=3)
                plan = tfmm.tfmm_plan_create(mesh, prm, stream=stream)
                setup_s = time.perf_counter() - t0
                info = plan.info
                N, G, nd = info["n_rwg"], info["n_groups"], info["n_dir"]
                tune = tfmm.tfmm_autotune(plan, R=R, budget_ms=3000.0, stream=stream)
                X = complex_gaussian((R, N), w.seed)
                x = torch.from_numpy(X.astype(np.complex64)).cuda()
                spec = torch.empty((R, G, 2, nd), dtype=torch.complex64, device="cuda")
                y = torch.empty((R, N), dtype=torch.complex64, device="cuda")
                for _ in range(3):
                    tfmm.tfmm_aggregate(plan, x, spec, stream=stream)
                    tfmm.tfmm_disaggregate(plan, spec, y, stream=stream)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                agg, dis = [], []
                for _ in range(10):
                    ev[0].record(stream)
                    tfmm.tfmm_aggregate(plan, x, spec, stream=stream)
                    ev[1].record(stream)
                    tfmm.tfmm_disaggregate(plan, spec, y, stream=stream)
                    ev[2].record(stream)
                    torch.cuda.synchronize()
                    agg.append(ev[0].elapsed_time(ev[1]))
                    dis.append(ev[1].elapsed_time(ev[2]))
                tfmm.tfmm_sync(plan, stream=stream)
                a_ms, d_ms = statistics.median(agg), statistics.median(dis)
                cm = 0
                sizes = []
                for g in range(G):
                    nb_g = 0
                    for a in range(2):
                        nb, (rt, rp, rb) = tfmm.tfmm_plan_group(plan, g, a)
                        nb_g = nb
                        cm += nb * rb + rt * rp * rb + info["n_phi"] * rp * rt + nd * rt
                    sizes.append((nb_g, g))
                flops = 8.0 * cm * R
                fac = info["tucker_bytes_alg"]
                bytes_agg = fac + 8 * N * R + 16 * G * nd * R
                dense_bytes = 16 * N * nd
                engine = {0: "fp32_chain", 1: "fp32_columns", 2: "tc_split_bf16_2", 3: "tc_split_bf16_3"}[tune["mrhs_precision"]]
                fl_peak = tensor if tune["mrhs_precision"] in (2, 3) else fp32
                # oracle: its own far-fields of the two smallest groups, dense FP64 Eq. 3
                pick = [g for _, g in sorted(sizes)[:2]]
                key = (box, d0)
                if key not in oracle_cache:  # the far-fields do not depend on the tolerance
                    oracle_cache.clear()
                    oracle_cache[key] = oracle.problem.build(verts, tris, k=2 * math.pi, box=box, digits=d0, tol=tol,
                                                             compress=False, keep_tensors=True, groups_subset=pick)
                P = oracle_cache[key]
                S = spec.cpu().numpy()
                err = 0.0
                for r in range(R):
                    num = den = 0.0
                    for g in pick:
                        xg = X[r][P.groups.members[g]]
                        A_t, A_p = P.group_tensors(g)
                        for a, A in enumerate((A_t, A_p)):
                            ref = apply.dense_aggregate(A, xg)
                            num += float(np.sum(np.abs(S[r, g, a] - ref) ** 2))
                            den += float(np.sum(np.abs(ref) ** 2))
                    err = max(err, math.sqrt(num / den))
                line = {
                    "point": {"box_lambda": box, "tol": tol, "digits": d0},
                    "L": info["L"], "n_theta": info["n_theta"], "n_phi": info["n_phi"], "groups": G,
                    "max_rank": info["max_rank"], "max_n_beta": info["max_n_beta"],
                    "compression": dense_bytes / fac, "tucker_gb": fac / 1e9, "dense_gb": dense_bytes / 1e9,
                    "ms_per_matvec": a_ms + d_ms, "aggregate_ms": a_ms, "disaggregate_ms": d_ms,
                    "nrhs": R, "engine": engine, "tuning": tune,
                    "hbm_frac": bytes_agg / (max(a_ms, d_ms) * 1e-3) / 1e9 / hbm,
                    "flop_frac": flops / (max(a_ms, d_ms) * 1e-3) / 1e12 / fl_peak,
                    "rel_err_vs_oracle_dense": err, "oracle_groups": pick, "setup_s": setup_s,
                }
                print(json.dumps(line), flush=True)
                del plan, x, spec, y
                torch.cuda.empty_cache()


def main():
    args = parse()
    if args.sweep:
        run_sweep(args)
        return
    from paper_2103_05822_gb300.inputs import WORKLOADS
    w = WORKLOADS[args.workload]
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, w, world, rank)
    else:
        run_ours(args, w, world, rank, local)


if __name__ == "__main__":
    main()
