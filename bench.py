"""Benchmark of the matrix-free NGF + curvature registration on B300.

One step = one full multilevel Gauss-Newton registration (register_multilevel:
image pyramid, per level 10 Gauss-Newton steps each with gradient, Jacobi
diagonal, 20 PCG iterations of gn_hessvec and an Armijo line search, and the
prolongation between levels).  The default workload is the synthetic
512x512x900 thorax-abdomen pair (0.8x0.8x1.0 mm, 129x129x225 nodes, 5 levels),
the largest single-GPU configuration; `--workload lung_ct` times the
256x256x120 lung-CT pair (1x1x2.5 mm, 129x129x61 nodes, 4 levels) the same
way.  Inputs are resident in HBM when the timed region starts; L2 is flushed
(a 256 MB write) before every timed step.

value = image voxels processed by gn_hessvec over the whole registration
(sum over levels of voxels x Hessian-vector products) / step time, in
Gvoxel/s: the Hessian-vector throughput of the whole job, every other part
of the registration included.  `ms_per_step` is the full-registration time.

`--impl reference` times the FP64 CPU oracle instead (bounded samples of the
same workload on the host cores).  Under torchrun every rank runs an
independent replica (the path has no exchange step); value sums all ranks'
voxels over the slowest rank's time.  Other workloads (batch_64, conv3d,
learned, oracle_timing) print their own JSON lines.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "thorax_abd"
REG_WORKLOADS = ("thorax_abd", "lung_ct")
GN_ITERS, PCG_ITERS = 10, 20
LBFGS_ITERS = 50  # L-BFGS steps per level of the comparison run
# algorithmic cost of one gn_hessvec image-grid pass per voxel (see design notes):
# P u and P p (separable) 30, warp + dT 50, 12 differences + N, A, B 40, rho_hat 25,
# v = dr s and t = dr^T v 28, q_hat 3, P^T 25  ->  200 FP32 flop (FMA = 2 flop)
HESS_FLOP_PER_VOXEL = 200.0
FP32_LANES_PER_SM = 128
METRIC = "gn_hessvec Gvoxel/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def reduce_max_sum(values_max, values_sum, ws):
    """(max over ranks of values_max, sum over ranks of values_sum)."""
    if ws == 1:
        return values_max, values_sum
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    a = torch.tensor([float(values_max)], dtype=torch.float64, device=dev)
    b = torch.tensor([float(values_sum)], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def image_pass_source_hash():
    """sha256 of the Hessian image pass's source (kernel body, its helpers and
    the tile, parameter and shared-memory layouts; not the diagonal pass's),
    to tell whether a stored DRAM traffic figure still describes the kernel
    that runs."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1804_10541_b300", "csrc")
    with open(os.path.join(csrc, "ngf_kernels.cu")) as f:
        cu = f.read()
    end = cu.index("image_pass<MODE_HESS, ImgSmemC>(P, blockIdx.x, blockIdx.y, blockIdx.z);")
    with open(os.path.join(csrc, "ngf_kernels.cuh")) as f:
        cuh = f.read()
    tiles = cuh[cuh.index("constexpr int TX"):cuh.index("// x-node window of one warp row in the diagonal kernel")]
    layouts = cuh[cuh.index("enum Mode"):cuh.index("constexpr int IMG_FILL")]
    return hashlib.sha256((cu[:end] + tiles + layouts).encode()).hexdigest()


def stored_traffic(workload):
    """DRAM bytes per launch of k_image_hess on the workload's finest level
    from the committed ncu summary, or None when the kernel source changed
    since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", f"k_image_hess_{workload}.md")) as f:
            txt = f.read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in txt.splitlines()
                  if line.startswith(("traffic_bytes_per_launch: ", "image_pass_source_sha256: ")))
    if fields.get("image_pass_source_sha256") != image_pass_source_hash():
        return None
    try:
        return float(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def oracle_sample(workload, R, T, w, planes=64):
    """A bounded piece of the workload for the FP64 oracle: the whole pair
    when it is small, else the z-slab of `planes` central image planes of R
    and T with its own node grid at the workload's voxels-per-cell ratio (the
    full 512x512x900 grid would need about 47 GB of host memory in the
    oracle's staged arrays).  Returns (m, h, n, R, T, description) with R, T
    float64 numpy arrays."""
    m, h, n = list(w["m"]), w["h"], list(w["n"])
    if m[2] > 2 * planes and m[0] * m[1] * m[2] > 32 * 1024 * 1024:
        z0 = (m[2] - planes) // 2
        plane = m[0] * m[1]
        ratio = (m[2]) / (n[2] - 1)
        Rh = R[z0 * plane:(z0 + planes) * plane].double().cpu().numpy()
        Th = T[z0 * plane:(z0 + planes) * plane].double().cpu().numpy()
        nz = max(2, int(round(planes / ratio)) + 1)
        desc = (f"z-slab of {planes} central planes ({m[0]}x{m[1]}x{planes}, nodes {n[0]}x{n[1]}x{nz}) of the "
                f"{m[0]}x{m[1]}x{m[2]} {workload} pair")
        return (m[0], m[1], planes), h, (n[0], n[1], nz), Rh, Th, desc
    return tuple(m), h, tuple(n), R.double().cpu().numpy(), T.double().cpu().numpy(), \
        f"the full {m[0]}x{m[1]}x{m[2]} {workload} grid"


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline_leg(workload, R, T, w, seconds_budget=20.0, max_calls=5):
    """Time the FP64 oracle's gn_hessvec (as it stands) on the host cores on a
    bounded sample of the same workload (see oracle_sample)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    from paper_1804_10541_b300 import synth
    m, h, n, Rh, Th, desc = oracle_sample(workload, R, T, w)
    L = O.level(m, h, n, w["alpha"], w["tau"], w["rho"])
    N = n[0] * n[1] * n[2]
    u, p = synth.random_fields(N, 5, amp=0.5 * min(h))
    uh, ph = u.double().numpy(), p.double().numpy()
    O.hessvec(L, Rh, Th, uh, ph)  # first call pages the arrays in; not timed
    times = []
    t0 = time.perf_counter()
    while len(times) < max_calls:
        t1 = time.perf_counter()
        O.hessvec(L, Rh, Th, uh, ph)
        times.append(time.perf_counter() - t1)
        if time.perf_counter() - t0 > seconds_budget:
            break
    M = m[0] * m[1] * m[2]
    med = statistics.median(times)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": M / med / 1e9, "unit": "Gvoxel/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"median of {len(times)} FP64 oracle gn_hessvec calls on the {desc} "
                      f"({med:.2f} s per call, OpenMP over z)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed as it stands on the host, on
    a bounded sample of the bench's workload (one gn_hessvec per step)."""
    ws, rank = _dist()
    if rank != 0:
        return 0
    import torch
    from paper_1804_10541_b300 import synth
    workload = args.workload if args.workload in REG_WORKLOADS else WORKLOAD
    R, T, _, w = synth.make(workload, device="cuda" if torch.cuda.is_available() else "cpu")
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    m, h, n, Rh, Th, desc = oracle_sample(workload, R, T, w)
    del R, T
    L = O.level(m, h, n, w["alpha"], w["tau"], w["rho"])
    N = n[0] * n[1] * n[2]
    u, p = synth.random_fields(N, 5, amp=0.5 * min(h))
    uh, ph = u.double().numpy(), p.double().numpy()
    for _ in range(args.warmup):
        O.hessvec(L, Rh, Th, uh, ph)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.hessvec(L, Rh, Th, uh, ph)
        times.append(time.perf_counter() - t0)
    M = m[0] * m[1] * m[2]
    total = sum(times)
    value = M * args.steps / total / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    wm = w["m"]
    line = {"metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{workload} {wm[0]}x{wm[1]}x{wm[2]} at {h[0]}x{h[1]}x{h[2]} mm; one step = one "
                                   f"FP64 oracle gn_hessvec on the {desc}",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "Gvoxel/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{args.steps} timed FP64 oracle gn_hessvec calls on the {desc}"},
            "e2e": {"value": value, "unit": "Gvoxel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    from paper_1804_10541_b300 import ngf, synth

    workload = args.workload
    R, T, _, w = synth.make(workload, device=dev)
    m, h, n, levels = w["m"], w["h"], w["n"], w["levels"]
    M = m[0] * m[1] * m[2]
    N = n[0] * n[1] * n[2]
    desc = ngf.level_desc(m, h, n, w["alpha"], w["tau"], w["rho"])
    opts = ngf.options(levels=levels, gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True)
    stream = torch.cuda.Stream(device=dev)
    u = torch.empty(3 * N, device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev, dtype=torch.float32)  # 256 MB > 126 MB L2

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            rep = ngf.register_multilevel(desc, opts, R, T, u, stream)
    stream.synchronize()

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = ngf.ngf_launch_count()
    voxels = 0
    reps = []
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            rep = ngf.register_multilevel(desc, opts, R, T, u, stream)
            ev[k][1].record(stream)
            voxels += rep.hessvec_voxels
            reps.append(rep)
    stream.synchronize()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = ngf.ngf_launch_count() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    t_max, vox_all = reduce_max_sum(t_local, voxels, ws)
    value = vox_all / t_max / 1e9

    # fixed cost of a registration call (allocations, plans, pyramid, objective
    # evaluations): the same call with zero Gauss-Newton steps
    opts0 = ngf.options(levels=levels, gn_iters=0, pcg_iters=PCG_ITERS, use_graph=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ngf.register_multilevel(desc, opts0, R, T, u, stream)
        e0.record(stream)
        ngf.register_multilevel(desc, opts0, R, T, u, stream)
        e1.record(stream)
    stream.synchronize()
    fixed_ms = e0.elapsed_time(e1)

    # ---- L-BFGS registration of the same pair (Sec. 2.3.2), for comparison
    opts_l = ngf.options(levels=levels, gn_iters=LBFGS_ITERS, method=ngf.NGF_METHOD_LBFGS, lbfgs_memory=5)
    ul = torch.empty(3 * N, device=dev)
    with torch.cuda.stream(stream):
        ngf.register_multilevel(desc, opts_l, R, T, ul, stream)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep_l = ngf.register_multilevel(desc, opts_l, R, T, ul, stream)
        e1.record(stream)
    stream.synchronize()
    lbfgs = {"registration_ms": e0.elapsed_time(e1), "steps_per_level": LBFGS_ITERS, "memory": 5,
             "final_J": rep_l.J, "steps": rep_l.gn_done, "ls_trials": rep_l.ls_trials,
             "J_rel_to_gauss_newton": (rep_l.J - reps[-1].J) / abs(reps[-1].J)}

    # ---- end to end through the public API with host buffers (pinned)
    Rp = torch.empty(M, dtype=torch.float32, pin_memory=True)
    Tp = torch.empty(M, dtype=torch.float32, pin_memory=True)
    Up = torch.empty(3 * N, dtype=torch.float32, pin_memory=True)
    Rp.copy_(R.cpu())
    Tp.copy_(T.cpu())
    e2e_times, e2e_vox = [], 0
    for k in range(max(1, min(args.steps, 5))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ngf.register_multilevel(desc, opts, Rp, Tp, Up, stream)
        e2e_times.append(time.perf_counter() - t0)
        e2e_vox += rep.hessvec_voxels
    e2e_t, e2e_v = reduce_max_sum(sum(e2e_times), e2e_vox, ws)
    e2e = {"value": e2e_v / e2e_t / 1e9, "unit": "Gvoxel/s", "h2d_bytes_per_step": 2 * M * 4,
           "d2h_bytes_per_step": 3 * N * 4}

    # ---- live roofline of the dominant kernel (Hessian image pass) at the
    # finest level, same plan configuration and inputs as inside the step
    gen = torch.Generator(device="cpu").manual_seed(11)
    uu = (0.5 * min(h) * torch.randn(3 * N, generator=gen)).to(dev)
    pp = torch.randn(3 * N, generator=gen).to(dev)
    q = torch.empty(3 * N, device=dev)
    nh = GN_ITERS * PCG_ITERS
    with torch.cuda.stream(stream), ngf.Plan(desc, stream) as pl:
        for _ in range(20):
            ngf.gn_hessvec(pl.handle, R, T, uu, pp, q)
        ngf.ngf_profile_enable(pl.handle, True)
        ngf.ngf_profile_read(pl.handle, ngf.NGF_K_HESSVEC)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nh):
            ngf.gn_hessvec(pl.handle, R, T, uu, pp, q)
        e1.record(stream)
        ms_img, nl = ngf.ngf_profile_read(pl.handle, ngf.NGF_K_HESSVEC)
        stream.synchronize()
        ms_call = e0.elapsed_time(e1) / nh
    t_launch = ms_img / nl / 1e3
    peaks = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    alu_peak = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s
    achieved = HESS_FLOP_PER_VOXEL * M / t_launch / 1e12
    bytes_per_voxel = 8.0 + 36.0 * N / M  # R, T + u, p read and q written, per voxel
    roofline = {"bound": "alu", "kernel": "k_image_hess", "achieved": achieved, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": stored_traffic(workload),
                "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz",
                "flop_per_voxel": HESS_FLOP_PER_VOXEL, "launch_us": t_launch * 1e6,
                "hessvec_call_us": ms_call * 1e3,
                "hbm": {"algorithmic_bytes": bytes_per_voxel * M,
                        "achieved_gbs": bytes_per_voxel * M / t_launch / 1e9,
                        "peak_gbs": peaks.get("hbm_gbs"),
                        "frac": (bytes_per_voxel * M / t_launch / 1e9) / peaks["hbm_gbs"] if "hbm_gbs" in peaks else None},
                "kernel_gvoxel_s": M / t_launch / 1e9,
                "measured_limiter": "instruction issue and latency, not the FP32 pipes or HBM: ncu shows issue "
                                    "active 61-63%, FMA pipe 28%, DRAM 3-4% of peak, top stalls long "
                                    "scoreboard (template gathers) and barrier "
                                    "(profiles/k_image_hess_<workload>.md)"}

    if rank == 0:
        cpu = None if (args.no_cpu_baseline or ws > 1) else cpu_baseline_leg(workload, R, T, w)
        r0 = reps[-1]
        line = {"metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{workload} {m[0]}x{m[1]}x{m[2]} at {h[0]}x{h[1]}x{h[2]} mm, nodes "
                                       f"{n[0]}x{n[1]}x{n[2]}, {levels} levels, {GN_ITERS} GN x {PCG_ITERS} PCG; "
                                       f"one step = one full register_multilevel",
                           "jacobi_preconditioner": "exact GN diagonal, computed at each level's first "
                                                    "Gauss-Newton step and kept for the level",
                           "parallelism": f"replicas x{ws}", "l2": "flushed before every step (256 MB write)",
                           "registration_ms": 1e3 * t_max / args.steps, "final_J": r0.J,
                           "gn_done": r0.gn_done, "pcg_total": r0.pcg_total, "ls_trials": r0.ls_trials,
                           "fixed_ms_per_registration": fixed_ms, "status": r0.status,
                           "torch_allocated_peak_gb": torch.cuda.max_memory_allocated(dev) / 1e9,
                           "parity": "operators match the FP64 oracle element-wise (gradient and Hessian-vector "
                                     "product 1e-5 relative L2, objective 1e-6) on crops with this workload's "
                                     "spacing and grid ratio; full registrations match the oracle's u within "
                                     "0.01 voxel after 3 GN steps per level and its final J within 1e-3 after "
                                     "10 (an Armijo decision within rounding can flip later)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "lbfgs": lbfgs,
                "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_kernel_case(args):
    """Kernel-only driver (for profiling): `calls` gn_hessvec products on the
    finest level of a workload, timed with CUDA events."""
    import torch
    from paper_1804_10541_b300 import ngf, synth
    if args.slab:
        # central z-slab of the thorax-abdomen phantom with its own node grid
        # at the workload's voxels-per-cell ratio: a smaller case of the same
        # kernel for multi-pass profiler captures (inputs still above L2)
        assert args.kernel_case == "thorax_abd"
        w = dict(synth.WORKLOADS["thorax_abd"])
        m, h, n = w["m"], w["h"], w["n"]
        z0 = (m[2] - args.slab) // 2
        R, T, _ = synth.thorax_pair(m, h, seed=w["seed"], device="cuda", zrange=(z0, z0 + args.slab))
        nz = max(2, int(round(args.slab * (n[2] - 1) / m[2])) + 1)
        m, n = (m[0], m[1], args.slab), (n[0], n[1], nz)
    else:
        R, T, _, w = synth.make(args.kernel_case, device="cuda")
        m, h, n = w["m"], w["h"], w["n"]
    torch.cuda.empty_cache()
    N = n[0] * n[1] * n[2]
    dist = ngf.NGF_DIST_SSD if args.distance == "ssd" else ngf.NGF_DIST_NGF
    desc = ngf.level_desc(m, h, n, w["alpha"], w["tau"], w["rho"], distance=dist)
    u, p = synth.random_fields(N, 5, amp=0.5 * min(h), device="cuda")
    q = torch.empty(3 * N, device="cuda")
    g = torch.empty(3 * N, device="cuda")
    dg = torch.empty(3 * N, device="cuda")
    times = {}
    with ngf.Plan(desc) as pl:
        ops = {"hessvec": lambda: ngf.gn_hessvec(pl.handle, R, T, u, p, q),
               "gradient": lambda: ngf.ngf_gradient(pl.handle, R, T, u, g, want_scalars=False),
               "diagonal": lambda: ngf.ngf_gn_diagonal(pl.handle, R, T, u, dg)}
        for name, op in ops.items():
            op()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.calls):
                op()
            e1.record()
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1) / args.calls
    M = m[0] * m[1] * m[2]
    print(json.dumps({"kernel_case": args.kernel_case, "m": list(m), "n": list(n), "distance": args.distance,
                      "calls": args.calls,
                      "ms": times, "hessvec_gvoxel_s": M / times["hessvec"] / 1e6}), flush=True)
    return 0


def shard_pairs(sizes, ws, rank):
    """Indices of the pairs rank `rank` of `ws` registers: largest first to
    the least-loaded rank (ties to the lower rank), by voxel count."""
    load = [0] * ws
    mine = []
    for k in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(ws), key=lambda j: (load[j], j))
        load[r] += sizes[k]
        if r == rank:
            mine.append(k)
    return sorted(mine)


def run_batch_sharded(args, ws, rank):
    """batch_64 over several GPUs: the pairs are independent, so each rank
    registers its share (balanced by voxels) with no data-path collective;
    the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    from paper_1804_10541_b300 import ngf, synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    pairs = synth.batch_pairs(device=dev)
    mine = shard_pairs([w["m"][0] * w["m"][1] * w["m"][2] for _, _, w in pairs], ws, rank)
    pairs = [pairs[k] for k in mine]
    descs = [ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"]) for _, _, w in pairs]
    R, T = [p[0] for p in pairs], [p[1] for p in pairs]
    U = [torch.zeros(3 * w["n"][0] * w["n"][1] * w["n"][2], device=dev) for _, _, w in pairs]
    opts = ngf.options(levels=2, gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ngf.register_batch(descs, opts, R, T, U, stream=stream)
    stream.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    voxels = 0
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            reps = ngf.register_batch(descs, opts, R, T, U, stream=stream)
            voxels += sum(r.hessvec_voxels for r in reps)
        e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    dist.barrier()
    t_max, vox_all = reduce_max_sum(e0.elapsed_time(e1) / 1e3, voxels, ws)
    if rank == 0:
        print(json.dumps({"workload": "batch_64 sharded by pairs", "metric": METRIC, "value": vox_all / t_max / 1e9,
                          "unit": "Gvoxel/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * t_max / args.steps, "scaling": "strong",
                          "pairs_on_rank0": len(mine), "dtype": "f32", "data": "synthetic"}), flush=True)
    dist.destroy_process_group()
    return 0


def run_batch(args):
    """Batched form on 64 blob pairs of uneven cubic size (64..192 voxels per
    side, 2 levels, 10 GN x 20 PCG): one register_batch call per step, against
    the same 64 pairs registered one after another with register_multilevel
    (equal decisions per pair, so equal final NGF); plus the per-pair error of
    the batched gn_hessvec against the FP64 oracle at the finest level."""
    import numpy as np
    import torch
    from paper_1804_10541_b300 import ngf, synth
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    dev = torch.device("cuda", 0)
    pairs = synth.batch_pairs(device=dev)
    descs = [ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"]) for _, _, w in pairs]
    R = [p[0] for p in pairs]
    T = [p[1] for p in pairs]
    nn = [3 * w["n"][0] * w["n"][1] * w["n"][2] for _, _, w in pairs]
    U = [torch.zeros(k, device=dev) for k in nn]
    opts = ngf.options(levels=2, gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev, dtype=torch.float32)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ngf.register_batch(descs, opts, R, T, U, stream=stream)
    stream.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = ngf.ngf_launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            reps = ngf.register_batch(descs, opts, R, T, U, stream=stream)
            ev[k][1].record(stream)
    stream.synchronize()
    launches = ngf.ngf_launch_count() - launches0
    clocks = sampler.stop()
    batch_ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    voxels = sum(r.hessvec_voxels for r in reps)
    # with the tile autotuner (z-chunk length chosen per level)
    Ua = [torch.zeros(k, device=dev) for k in nn]
    with torch.cuda.stream(stream):
        flush.fill_(0.5)
        ea0, ea1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea0.record(stream)
        reps_a = ngf.register_batch(descs, opts, R, T, Ua, autotune=True, stream=stream)
        ea1.record(stream)
    stream.synchronize()
    auto_ms = ea0.elapsed_time(ea1)
    # the same pairs one at a time, each with its own default z-chunk model
    U1 = [torch.zeros(k, device=dev) for k in nn]
    with torch.cuda.stream(stream):
        flush.fill_(0.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps1 = [ngf.register_multilevel(d, opts, r, t, u, stream) for d, r, t, u in zip(descs, R, T, U1)]
        e1.record(stream)
    stream.synchronize()
    seq_ms = e0.elapsed_time(e1)
    same_u = all(torch.equal(a, b) for a, b in zip(U, U1))
    j_rel = max(abs(a.J - b.J) / abs(b.J) for a, b in zip(reps, reps1))
    # at equal final NGF: one common z-chunk for both arms on every level, so
    # every pair takes identical decisions (bitwise equal u); several common
    # chunk lengths are timed and the one that is best for the sequential
    # arm is quoted (a long chunk starves a single small pair of CTAs)
    with ngf.Batch(descs, 0, stream) as b0:
        zc_batch = ngf.ngf_batch_zc(b0.handle)
    eq_rows = []
    for zc_c in sorted({8, 16, 32, zc_batch}):
        opts_eq = ngf.options(levels=2, gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True, zc=zc_c)
        Ue = [torch.zeros(k, device=dev) for k in nn]
        Us = [torch.zeros(k, device=dev) for k in nn]
        with torch.cuda.stream(stream):
            ngf.register_batch(descs, opts_eq, R, T, Ue, stream=stream)  # warm-up (plans, graphs)
            flush.fill_(0.5)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            reps_e = ngf.register_batch(descs, opts_eq, R, T, Ue, stream=stream)
            b_.record(stream)
            flush.fill_(0.25)
            es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            es0.record(stream)
            reps_s = [ngf.register_multilevel(d, opts_eq, r, t, u, stream) for d, r, t, u in zip(descs, R, T, Us)]
            es1.record(stream)
        stream.synchronize()
        eq_rows.append({"zc": zc_c, "batched_ms": a_.elapsed_time(b_), "sequential_ms": es0.elapsed_time(es1),
                        "same_u_as_sequential": all(torch.equal(x_, y_) for x_, y_ in zip(Ue, Us)),
                        "max_rel_J_diff_vs_sequential": max(abs(x_.J - y_.J) / abs(y_.J)
                                                            for x_, y_ in zip(reps_e, reps_s))})
    at_batch_zc = next(r_ for r_ in eq_rows if r_["zc"] == zc_batch)
    best = min(eq_rows, key=lambda r_: r_["sequential_ms"])
    # tile autotuner on the finest level, then per-pair parity with the oracle
    import oracle as O
    gen = torch.Generator(device="cpu").manual_seed(31)
    uu = [(0.5 * torch.randn(k, generator=gen)).to(dev) for k in nn]
    pp = [torch.randn(k, generator=gen).to(dev) for k in nn]
    qq = [torch.empty(k, device=dev) for k in nn]
    with torch.cuda.stream(stream), ngf.Batch(descs, 0, stream) as b:
        e0.record(stream)
        for _ in range(3):
            ngf.ngf_batch_hessvec(b.handle, R, T, uu, pp, qq)
        e1.record(stream)
        stream.synchronize()
        ms_default = e0.elapsed_time(e1) / 3
        zc, ms_tuned = ngf.ngf_batch_autotune(b.handle, R, T, uu, pp, qq)
        ngf.ngf_batch_hessvec(b.handle, R, T, uu, pp, qq)
        stream.synchronize()
    errs = []
    for k, (d, w) in enumerate(zip(descs, [p[2] for p in pairs])):
        L = O.level(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
        qo = O.hessvec(L, R[k].double().cpu().numpy(), T[k].double().cpu().numpy(), uu[k].double().cpu().numpy(),
                       pp[k].double().cpu().numpy())
        errs.append(float(np.linalg.norm(qq[k].double().cpu().numpy() - qo) / np.linalg.norm(qo)))
    total_vox = sum(w["m"][0] * w["m"][1] * w["m"][2] for _, _, w in pairs)
    line = {"workload": "batch_64: 64 blob pairs, cubic N ~ U{64..192} (seed 30), nodes N/2+1, 2 levels, "
                        f"{GN_ITERS} GN x {PCG_ITERS} PCG", "metric": METRIC,
            "value": voxels / (batch_ms / 1e3) / 1e9, "unit": "Gvoxel/s", "steps": args.steps,
            "warmup": args.warmup,
            "at_equal_NGF": {**at_batch_zc,
                             "speedup_vs_sequential": at_batch_zc["sequential_ms"] / at_batch_zc["batched_ms"],
                             "note": "both arms with the batch's z-chunk model, so every pair takes identical "
                                     "decisions (bitwise equal u); a single small pair fills few CTAs with "
                                     "long chunks, which is the cost the batched form removes"},
            "at_equal_NGF_sequential_best_zc": {
                **best, "speedup_vs_sequential": best["sequential_ms"] / best["batched_ms"],
                "note": "the common z-chunk that is best for the sequential arm among those timed"},
            "all_common_zc": eq_rows,
            "default_zc": {"batched_ms": batch_ms, "sequential_ms": seq_ms,
                           "speedup_vs_sequential": seq_ms / batch_ms, "same_u_as_sequential": same_u,
                           "max_rel_J_diff_vs_sequential": j_rel,
                           "note": "each arm with its own default z-chunk model: other tile depths round "
                                   "differently and the nonconvex problem can follow other trajectories"},
            "total_voxels": total_vox,
            "autotuned_registration_ms": auto_ms,
            "autotuned_max_rel_J_diff_vs_sequential": max(abs(a.J - b.J) / abs(b.J) for a, b in zip(reps_a, reps1)),
            "batched_hessvec_ms": {"default_zc": ms_default, "autotuned": ms_tuned, "zc": zc},
            "hessvec_rel_err_vs_oracle": {"max": max(errs), "median": statistics.median(errs)},
            "gpu_launches": int(launches), "clocks": clocks,
            "l2": "flushed before every step (256 MB write)", "dtype": "f32", "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_conv3d(args):
    """Tensor-core 3x3x3 convolution (learned-initializer building block) on
    the layer shapes of a 4-level encoder at 128^3 (16 -> 128 channels): per
    layer the median of `steps` single-launch CUDA-event timings, L2 flushed
    before each, and sampled outputs checked against the FP64 oracle."""
    import numpy as np
    import torch
    from paper_1804_10541_b300 import ngf
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import cnn_oracle as CO
    dev = torch.device("cuda", 0)
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peak = json.load(f)["bf16_tflops"]
    flush = torch.empty(64 * 1024 * 1024, device=dev, dtype=torch.float32)
    gen = torch.Generator().manual_seed(41)
    layers = []
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = ngf.ngf_launch_count()
    for (S, ci, co) in [(128, 16, 16), (64, 32, 32), (32, 64, 64), (16, 128, 128), (64, 32, 256)]:
        x = torch.randn(1, S, S, S, ci, generator=gen).to(torch.bfloat16)
        w = (torch.randn(co, 3, 3, 3, ci, generator=gen) / (27 * ci) ** 0.5).to(torch.bfloat16)
        xd, wd = x.to(dev), w.to(dev)
        y = torch.empty(1, S, S, S, co, device=dev)
        for _ in range(max(3, args.warmup)):
            ngf.ngf_conv3d_fwd(xd, wd, None, y)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record()
            ngf.ngf_conv3d_fwd(xd, wd, None, y)
            ev[k][1].record()
        torch.cuda.synchronize()
        assert ngf.ngf_conv3d_check() == 0
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        flop = 2.0 * S ** 3 * 27 * ci * co
        # sampled outputs against the oracle (3x3x3 neighbourhood crops)
        xp = np.pad(x.float().numpy()[0], ((1, 1), (1, 1), (1, 1), (0, 0)))
        wf = w.float().numpy()
        yc = y.cpu().numpy()[0]
        rng = np.random.default_rng(S + ci + co)
        worst = 0.0
        for _ in range(16):
            z, yy, xx = (int(v) for v in rng.integers(0, S, 3))
            crop = xp[z:z + 3, yy:yy + 3, xx:xx + 3][None]
            yo = CO.conv3d(crop, wf)[0, 1, 1, 1]
            scale = CO.conv3d_abs(crop, wf)[0, 1, 1, 1]
            worst = max(worst, float(np.max(np.abs(yc[z, yy, xx] - yo) / scale)))
        layers.append({"shape": f"{S}^3 {ci}->{co}", "ms": ms, "gflop": flop / 1e9, "tflops": flop / ms / 1e9,
                       "frac_of_measured_bf16": flop / ms / 1e9 / peak,
                       "max_err_over_abs_sum_sampled": worst})
    launches = ngf.ngf_launch_count() - launches0
    clocks = sampler.stop()
    total_flop = sum(l["gflop"] * 1e9 for l in layers)
    total_ms = sum(l["ms"] for l in layers)
    line = {"workload": "conv3d: 3x3x3 bf16 convolution layers of a 4-level encoder at 128^3, fp32 out",
            "metric": "conv3d TFLOP/s", "value": total_flop / total_ms / 1e9, "unit": "TFLOP/s",
            "steps": args.steps, "warmup": args.warmup, "layers": layers,
            "roofline": {"bound": "tensor", "achieved": total_flop / total_ms / 1e9, "peak": peak,
                         "unit": "TFLOP/s", "frac": total_flop / total_ms / 1e9 / peak,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)"},
            "gpu_launches": int(launches), "clocks": clocks, "l2": "flushed before every launch (256 MB write)",
            "dtype": "bf16 x bf16 -> f32", "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """Learned initializer (the encoder-decoder of ngf_cnn.h) end to end:
    `--learned-train` + `--learned-test` lung-CT-like pairs at 128^3
    (2 x 2 x 2.34 mm, 65^3 nodes, 4 levels) generated on the device, all
    registered by plain multilevel Gauss-Newton (batched, 10 GN x 20 PCG per
    level) for the training targets, training on the GPU (Adam, batch 8), and
    on the held-out pairs plain Gauss-Newton from zero against the network's
    start refined by Gauss-Newton, both to the same final objective (within
    0.1% of plain Gauss-Newton's full-schedule J)."""
    import numpy as np
    import torch
    from paper_1804_10541_b300 import learned as LR, ngf
    dev = torch.device("cuda", 0)
    s, ntr, nte = 128, args.learned_train, args.learned_test
    w = LR.workload(s)
    t0 = time.perf_counter()
    R, T = LR.make_pairs(s, 0, ntr + nte, dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    U0, Jb = LR.register_all(R, T, w)
    torch.cuda.synchronize()
    t_reg = time.perf_counter() - t0
    U1 = LR.level1_targets(U0, w["n"][0])
    del U0
    Rtr, Ttr, U1tr = R[:ntr], T[:ntr], U1[:ntr].contiguous()
    Rte, Tte, U1te = R[ntr:], T[ntr:], U1[ntr:].contiguous()
    batch = 8
    d = ngf.net_desc(s, batch, LR.IN_SHIFT, LR.IN_SCALE, LR.OUT_SCALE)
    launches0 = ngf.ngf_launch_count()
    with ngf.Net(d) as net:
        ngf.ngf_net_set_params(net.handle, torch.from_numpy(LR.init_params(7)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = LR.train(net, Rtr, Ttr, U1tr, epochs=args.learned_epochs, batch=batch, lr0=1e-3,
                          log=lambda m: print(m, file=sys.stderr, flush=True))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        assert ngf.ngf_conv3d_check() == 0
        pred = LR.predict(net, Rte, Tte, batch)
        mse_net = float(((pred - U1te) ** 2).mean())
        mse_zero = float((U1te ** 2).mean())
        rows = LR.compare(net, Rte, Tte, w, k1=args.learned_k1, finest_cap=30)
    launches = ngf.ngf_launch_count() - launches0
    # training throughput in tensor-core FLOP: forward over all layers, data
    # gradient of all but the first, weight gradient of all
    vol = [s ** 3, (s // 2) ** 3, (s // 4) ** 3, (s // 8) ** 3, (s // 4) ** 3, (s // 4) ** 3, (s // 4) ** 3]
    fwd = [2.0 * 27 * v * ci * co for v, (ci, co) in zip(vol, LR.LAYERS)]
    step_flop = batch * (2 * sum(fwd) + sum(fwd[1:]))
    steps = args.learned_epochs * ((ntr + batch - 1) // batch)
    reached = [r for r in rows if r["learned_reached"]]
    line = {"workload": f"learned initializer: {ntr} training + {nte} held-out lung-CT-like pairs at {s}^3 "
                        f"(2x2x2.34 mm, 65^3 nodes, 4 levels, 10 GN x 20 PCG); 4-level encoder-decoder 16..128 "
                        f"channels, bf16 activations, FP32 accumulation; Adam batch {batch}, "
                        f"{args.learned_epochs} epochs",
            "metric": "full-registration seconds at equal NGF", "unit": "s", "higher_is_better": False,
            "value": float(np.mean([r["learned_s"] for r in reached])) if reached else None,
            "plain_gn_s_mean": float(np.mean([r["plain_s"] for r in rows])),
            "plain_gn_full_schedule_s_mean": float(np.mean([r["full_s"] for r in rows])),
            "learned_s_mean_over_reached": float(np.mean([r["learned_s"] for r in reached])) if reached else None,
            "plain_s_mean_over_reached": float(np.mean([r["plain_s"] for r in reached])) if reached else None,
            "speedup_at_equal_J": (float(np.mean([r["plain_s"] for r in reached]) /
                                         np.mean([r["learned_s"] for r in reached])) if reached else None),
            "gn_steps_plain_mean": float(np.mean([r["plain_gn"] for r in rows])),
            "gn_steps_learned_mean_over_reached": float(np.mean([r["learned_gn"] for r in reached])) if reached else None,
            "held_out_reached_J_within_0.1pct": len(reached), "held_out": len(rows),
            "learned_J_rel_to_ref_median": float(np.median([(r["learned_J"] - r["J_ref"]) / r["J_ref"] for r in rows])),
            "held_out_mse_mm2": {"network": mse_net, "zero_start": mse_zero},
            "train_loss_first_last_epoch": [losses[0], losses[-1]],
            "seconds": {"generate": t_gen, "register_targets": t_reg, "train": t_train},
            "train_tflops": step_flop * steps / t_train / 1e12, "train_pairs_per_s": ntr * args.learned_epochs / t_train,
            "gpu_launches": int(launches), "dtype": "bf16 x bf16 -> f32 (network), f32 (registration)",
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


# The paper's 2-D GPU numbers (GeForce GTX 980, FP32, reductions FP64): the
# objective-gradient time per image and grid size (Sec. 6.4, table of 2-D
# gradient runtimes) and the 3-level L-BFGS registration time (Sec. 6.4,
# figure of 2-D registration runtimes), in milliseconds; context, not targets.
PAPER_2D_GRADIENT_MS = {(4096, 2049): 35.3, (4096, 1025): 33.5, (4096, 513): 32.3, (2048, 1025): 10.0,
                        (2048, 513): 9.38, (2048, 257): 9.32, (1024, 513): 3.66, (1024, 257): 3.53,
                        (1024, 129): 2.93, (512, 257): 2.29, (512, 129): 1.67, (512, 65): 1.67, (256, 129): 1.04,
                        (256, 65): 1.03, (256, 33): 1.07}
PAPER_2D_LBFGS_S = {4096: 1.51, 2048: 0.560, 1024: 0.267, 512: 0.143, 256: 0.0833}


def run_plane_2d(args):
    """The 2-D method (planar levels) on the paper's 2-D sizes: objective
    gradient (ngf_gradient_dev: the NGF gradient and D, S on the device) for
    m^2 images, m in 256..4096, with m/2+1, m/4+1 and m/8+1 nodes per axis
    (median of `steps` calls after warm-up, CUDA events), and the 3-level
    L-BFGS registration with nodes m/4+1 and 20 steps per level (median of
    3), on synthetic tissue-like pairs (the histology data is not available)."""
    import numpy as np
    import torch
    from paper_1804_10541_b300 import ngf, synth
    dev = torch.device("cuda", 0)
    sizes = [256, 512, 1024, 2048, 4096]
    grad_rows, reg_rows = [], []
    launches0 = ngf.ngf_launch_count()
    for M in sizes:
        R, T = synth.tissue_pair_2d((M, M), seed=60 + M, device=dev)
        for k in (2, 4, 8):
            nn = M // k + 1
            desc = ngf.level_desc((M, M, 1), (1.0, 1.0, 1.0), (nn, nn, 1), 1.0, 0.05, 0.05)
            N = nn * nn
            g = torch.Generator().manual_seed(M + k)
            u = torch.cat([0.5 * torch.randn(2 * N, generator=g), torch.zeros(N)]).to(dev)
            grad = torch.empty(3 * N, device=dev)
            ds = torch.empty(2, device=dev, dtype=torch.float64)
            with ngf.Plan(desc) as pl:
                for _ in range(max(3, args.warmup)):
                    ngf.ngf_gradient_dev(pl.handle, R, T, u, grad, ds)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(max(5, args.steps))]
                for a, b in ev:
                    a.record()
                    ngf.ngf_gradient_dev(pl.handle, R, T, u, grad, ds)
                    b.record()
                torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in ev)
            grad_rows.append({"m": M, "nodes": nn, "ms": ms, "gpixel_s": M * M / ms / 1e6,
                              "paper_gtx980_ms": PAPER_2D_GRADIENT_MS.get((M, nn))})
        nn = M // 4 + 1
        desc = ngf.level_desc((M, M, 1), (1.0, 1.0, 1.0), (nn, nn, 1), 1.0, 0.05, 0.05)
        opts = ngf.options(levels=3, gn_iters=20, method=ngf.NGF_METHOD_LBFGS, lbfgs_memory=5)
        u = torch.zeros(3 * nn * nn, device=dev)
        stream = torch.cuda.Stream(device=dev)
        times, rep = [], None
        with torch.cuda.stream(stream):
            ngf.register_multilevel(desc, opts, R, T, u, stream)
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep = ngf.register_multilevel(desc, opts, R, T, u, stream)
                e1.record(stream)
                stream.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
        reg_rows.append({"m": M, "nodes": nn, "seconds": statistics.median(times), "steps": rep.gn_done,
                         "ls_trials": rep.ls_trials, "J": rep.J, "paper_gtx980_s": PAPER_2D_LBFGS_S.get(M)})
        del R, T
    line = {"workload": "plane_2d: 2-D method (one image plane, one node plane) on synthetic tissue-like m^2 pairs "
                        "(unit spacing, alpha 1, tau = rho = 0.05)", "metric": "2-D objective gradient ms",
            "unit": "ms", "gradient": grad_rows, "lbfgs_registration_3_levels_20_steps": reg_rows,
            "gpu_launches": int(ngf.ngf_launch_count() - launches0),
            "note": "paper numbers: GeForce GTX 980, histology pairs; context, not a like-for-like target",
            "dtype": "f32", "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def _meminfo_gb(key="MemAvailable"):
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith(key + ":"):
                    return int(line.split()[1]) / 1024 ** 2
    except OSError:
        pass
    return None


def _oracle_leg(threads):
    """One leg of the oracle timing at a fixed OpenMP thread count (this
    process was started with OMP_NUM_THREADS = threads)."""
    import numpy as np
    import torch
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    from paper_1804_10541_b300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    out = {"threads": threads, "hessvec": {}, "registration": {}}

    def hv(L, Rh, Th, calls):
        N = L.n[0] * L.n[1] * L.n[2]
        u, p = synth.random_fields(N, 5, amp=0.5 * min(L.h[0], L.h[1], L.h[2]))
        uh, ph = u.double().numpy(), p.double().numpy()
        O.hessvec(L, Rh, Th, uh, ph)
        ts = []
        for _ in range(calls):
            t0 = time.perf_counter()
            O.hessvec(L, Rh, Th, uh, ph)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts), len(ts)

    for name in ("blobs_32", "lung_ct", "thorax_abd"):
        R, T, _, w = synth.make(name, device=dev)
        m, h, n = w["m"], w["h"], w["n"]
        M = m[0] * m[1] * m[2]
        rec = {}
        if name == "thorax_abd":
            # the full grid only when the host has room for the oracle's
            # staged arrays (about 200 bytes per voxel) and all cores run it
            avail = _meminfo_gb()
            if threads > 1 and avail is not None and avail > 80:
                L = O.level(m, h, n, w["alpha"], w["tau"], w["rho"])
                t, k = hv(L, R.double().cpu().numpy(), T.double().cpu().numpy(), 1)
                rec["full_grid"] = {"s": t, "calls": k, "mvoxel_s": M / t / 1e6}
            planes = 64 if threads > 1 else 16
            ms, hs, ns, Rh, Th, desc = oracle_sample(name, R, T, w, planes=planes)
            L = O.level(ms, hs, ns, w["alpha"], w["tau"], w["rho"])
            t, k = hv(L, Rh, Th, 5 if threads > 1 else 3)
            Ms = ms[0] * ms[1] * ms[2]
            rec["slab"] = {"sample": desc, "s": t, "calls": k, "mvoxel_s": Ms / t / 1e6,
                           "full_grid_s_extrapolated": t * M / Ms}
            if threads > 1:
                # one Gauss-Newton step (gradient, diagonal, 20 PCG, Armijo) on
                # the slab, extrapolated per voxel to the 5-level registration
                uh0 = np.zeros(3 * ns[0] * ns[1] * ns[2])
                t0 = time.perf_counter()
                O.gn_level(L, Rh, Th, uh0, O.gn_options(gn_iters=1, pcg_iters=PCG_ITERS))
                t_gn = time.perf_counter() - t0
                vox_levels = 0
                mm = list(m)
                for _ in range(w["levels"]):
                    vox_levels += mm[0] * mm[1] * mm[2]
                    mm = [(a + 1) // 2 for a in mm]
                rec["registration_extrapolated_s"] = t_gn / Ms * vox_levels * GN_ITERS
                rec["registration_extrapolation"] = (
                    f"one oracle GN step ({PCG_ITERS} PCG) on the slab took {t_gn:.1f} s; x {GN_ITERS} steps x "
                    f"the voxels of all {w['levels']} levels / slab voxels (labelled extrapolation, not a run)")
        else:
            L = O.level(m, h, n, w["alpha"], w["tau"], w["rho"])
            Rh, Th = R.double().cpu().numpy(), T.double().cpu().numpy()
            t, k = hv(L, Rh, Th, 5 if (threads > 1 or name == "blobs_32") else 3)
            rec = {"s": t, "calls": k, "mvoxel_s": M / t / 1e6}
            if threads > 1 or name == "blobs_32":
                t0 = time.perf_counter()
                _, rep = O.register_multilevel(L, w["levels"], O.gn_options(gn_iters=GN_ITERS, pcg_iters=PCG_ITERS),
                                               Rh, Th)
                out["registration"][name] = {"s": time.perf_counter() - t0, "J": rep.J, "gn_done": rep.gn_done,
                                             "pcg_total": rep.pcg_total, "levels": w["levels"]}
        out["hessvec"][name] = rec
        del R, T
    return out


def run_oracle_timing(args):
    """The FP64 oracle timed on the host cores: gn_hessvec (median of 5) on
    the 32^3, lung-CT and thorax-abdomen workloads, full registrations of the
    first two, and a labelled extrapolation for the 512x512x900 registration;
    once with all cores and once with one (each leg in its own process, so
    that OpenMP starts with that thread count)."""
    if args.threads > 0:
        print(json.dumps(_oracle_leg(args.threads)), flush=True)
        return 0
    nproc = os.cpu_count() or 1
    legs = []
    for t in (nproc, 1):
        env = dict(os.environ, OMP_NUM_THREADS=str(t))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", "oracle_timing", "--threads",
                            str(t)], env=env, capture_output=True, text=True)
        if r.returncode != 0:
            print(r.stderr[-2000:], file=sys.stderr)
            return r.returncode
        legs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    line = {"workload": "oracle_timing", "kind": "FP64 oracle (oracle/ngf_oracle.c) as it stands, OpenMP over z",
            "nproc": nproc, "cpu_model": cpu_model(), "host_mem_total_gb": _meminfo_gb("MemTotal"),
            "legs": legs}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-case", default=None, help="profile driver: gn_hessvec only on this workload")
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--slab", type=int, default=0, help="--kernel-case: central z-slab of this many planes")
    ap.add_argument("--distance", default="ngf", choices=["ngf", "ssd"], help="distance of --kernel-case")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[*REG_WORKLOADS, "batch_64", "conv3d", "oracle_timing", "learned", "plane_2d"],
                    help="thorax_abd (default) / lung_ct: full registrations; batch_64: the batched form on 64 "
                         "uneven pairs; conv3d: the tensor-core convolution layers; oracle_timing: the FP64 "
                         "oracle on the host cores (each of the last three prints its own JSON line)")
    ap.add_argument("--threads", type=int, default=0, help="oracle_timing: OpenMP threads of one leg")
    ap.add_argument("--learned-train", type=int, default=4000)
    ap.add_argument("--learned-test", type=int, default=500)
    ap.add_argument("--learned-epochs", type=int, default=8)
    ap.add_argument("--learned-k1", type=int, default=3, help="learned: Gauss-Newton steps on level 1")
    args = ap.parse_args()
    if args.kernel_case:
        return run_kernel_case(args)
    if args.workload == "batch_64":
        ws, rank = _dist()
        return run_batch_sharded(args, ws, rank) if ws > 1 else run_batch(args)
    if args.workload == "oracle_timing":
        return run_oracle_timing(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "plane_2d":
        return run_plane_2d(args)
    if args.workload == "conv3d":
        return run_conv3d(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
