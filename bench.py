"""Benchmark of the WSBM / HSS entry generator on GB300.

Metric: kernel entries/s of the HSS build at N = 2^18 (star r = 1 + 0.3 cos 5t, 15 nodes per
exterior wavelength, n = 1.5), i.e. complex matrix entries written by the entry kernels
(dense leaf blocks, near-field blocks, proxy-circle blocks) divided by the summed device time
of those kernels.  One step = one HSS leaf-level build through the C ABI: wsbm_create, then
wsbm_factor with max_levels = 1 (entries, interpolative decompositions, leaf LU and the
compressed leaf factors).  The line also reports the step time (build + factor seconds of
the level), the mixed-precision path, full HSS runs where they fit, the CPU oracle timed on
a bounded sample, an end-to-end figure through host buffers, clocks and a roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

Under torchrun every rank runs an independent replica of the workload (the single-curve build
does not shard without a skeleton exchange between ranks); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HSS build+factor s and kernel entries/s at N=2^18, FP64 vs mixed, at stated error"
UNIT = "entries/s"

# Per-pair FP64 operation counts and DRAM bytes of the entry kernels, read from ncu counters
# for the kernel sources with the recorded hash; when the sources change the traffic figure is
# withheld until re-measured.
KERNEL_COUNTS = {
    "src_sha": "39971b7a6cb47b86",
    # 16384-node star, leaf level (bench.py --profile-case), tiles of 16 x 8 node pairs (the
    # autotuned shape; the proxy kernel's per-pair count includes its proxy-point set-up, which
    # depends on the tile width): 4.16 M / 4.24 M pairs
    "k_proxy": {"tf": 16, "fp64_flops_per_pair": 244.5, "dram_bytes_per_pair": 50.1},
    "k_pairs": {"tf": 16, "fp64_flops_per_pair": 323.9, "dram_bytes_per_pair": 50.8},
    # DRAM traffic of the column-pivoted QR per ID matrix of this workload, keyed by the hash of
    # its dense.cu section and the matrix rows it was measured on (1024 sketches of 128 rows,
    # 65536-node star)
    "k_cpqr": {"src_sha": "efa00c1011a862ff", "rows": 128, "dram_bytes_per_matrix": 6.30e7},
    # DRAM traffic of the two fused LU + solve launches of a leaf level (box LU with D^-1 L of
    # 256 unknowns, and Dhat), per factored matrix: 25.71 GB over the 1024 matrices of the
    # 512 leaf boxes of the same star at N = 65536 (boxes of the same size and ranks)
    "k_lu_solve_fused": {"src_sha": "f6983435ab7b8259", "dram_bytes_per_matrix": 25.711e9 / 1024},
}
# FP64 peak from the unit counts: 152 SMs x 4 FP64 flops/clk/SM (2 DFMA) x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# A DFMA microbenchmark (every SM, dependent chains, CUDA events) reached 1.013 TFLOP/s at an
# SM clock of 2.0 GHz; it scales with the clock.
FP64_DFMA_MEASURED = (1.013, 2000.0)


def measured_peaks():
    """Measured peaks of this GPU model (HBM copy, cuBLAS BF16) from MEASURED_PEAKS.json, when present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def add_fracs(roof, clk):
    """frac against the unit-count FP64 peak (roof['frac']) and against the measured DFMA rate
    scaled to the median SM clock sampled during the timed region."""
    if not roof or roof.get("achieved") is None:
        return roof
    mhz = (clk or {}).get("sm_mhz") or FP64_DFMA_MEASURED[1]
    peak_m = FP64_DFMA_MEASURED[0] * mhz / FP64_DFMA_MEASURED[1]
    roof["peak_measured_dfma"] = peak_m
    roof["frac_of_measured_dfma"] = roof["achieved"] / peak_m
    return roof


def _dense_section(begin, end):
    with open(os.path.join(ROOT, "paper_2607_00790_gb300", "csrc", "dense.cu"), "rb") as fh:
        src = fh.read()
    a = src.index(begin.encode())
    return src[a:src.index(end.encode(), a)]


def cpqr_src_sha():
    """Hash of the column-pivoted QR kernel's source section of dense.cu."""
    sec = _dense_section("// ------------------------------------------------- column-pivoted Householder QR ----",
                         "// ------------------------------------------------------------------ host drivers ----")
    return hashlib.sha256(sec).hexdigest()[:16]


def lu_src_sha():
    """Hash of the fused LU + solve kernel's source section of dense.cu."""
    sec = _dense_section("// --------------------------------------------------------- fused LU + solve ----",
                         "// ------------------------------------------------- column-pivoted Householder QR ----")
    return hashlib.sha256(sec).hexdigest()[:16]


def kernel_src_sha():
    h = hashlib.sha256()
    for f in ("entries.cu", "entry_blocks.cuh", "hankel.cuh", "hankel_coeffs.inc"):
        with open(os.path.join(ROOT, "paper_2607_00790_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def workload():
    from paper_2607_00790_gb300 import inputs
    N = 262144
    c = inputs.star(N)
    cfg = dict(workload="star r=1+0.3cos(5t), N=262144, 15 nodes/wavelength, n=1.5, leaf 128, "
                        "128 proxy points (grown per box), ID tol 1e-8; step = HSS leaf-level "
                        "build (entries + ID + leaf factor)",
               N=N, k0=float(inputs.k0_for_density(c)), n=1.5, leaf=128, nproxy=128, tol=1e-8,
               l2="step writes > 10 GB (ID matrices, factors), far above the 129 MB L2")
    return c, cfg


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(ws, v, op, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(ws, v, device="cuda"):
    """Largest value over the ranks (timings: the slowest rank sets the job time)."""
    import torch.distributed as dist
    return v if ws == 1 else _reduce(ws, v, dist.ReduceOp.MAX, device)


def sum_over_ranks(ws, v, device="cuda"):
    """Sum over the ranks (work: entries generated by all replicas)."""
    import torch.distributed as dist
    return v if ws == 1 else _reduce(ws, v, dist.ReduceOp.SUM, device)


def job_throughput(ws, entries, ms_kernel, device="cuda"):
    """Whole-job entries/s: entries of every rank over the slowest rank's kernel time."""
    return sum_over_ranks(ws, entries, device) / (max_over_ranks(ws, ms_kernel, device) * 1e-3)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- ours ----
def run_ours(args, ws, rank, local):
    import torch
    from paper_2607_00790_gb300 import binding

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    curve, cfg = workload()
    g, keep = binding.make_geom(curve, device=dev)

    def params(precision=binding.WSBM_FP64, tol=cfg["tol"], max_levels=1):
        return binding.make_params(cfg["k0"], cfg["n"], leaf=cfg["leaf"], nproxy=cfg["nproxy"],
                                   id_tol=tol, precision=precision, max_levels=max_levels)

    def step(p):
        s = binding.Solver(g, p, device=dev)
        s.factor()
        st = s.stats()
        s.close()
        return st

    p64 = params()
    # launch shapes before the warm-up: the tensor-core paths timed on synthetic data of this
    # workload's sizes (leaf boxes of 2 x leaf unknowns, N / leaf of them, 128 right-hand sides
    # each), the entry-kernel tiles / grids and QR block size on leaf-level builds of it
    tuning = None
    if args.set_tuning:
        # fixed shapes (e.g. the choice of an earlier autotuned run, for a profiler capture)
        apply_tuning(args.set_tuning)
    elif not args.no_autotune:
        choice, tms = binding.wsbm_autotune(n_box=2 * cfg["leaf"], nbox=cfg["N"] // cfg["leaf"],
                                            nrhs_box=128, n_root=4096, device=dev)
        bchoice, bms = binding.wsbm_autotune_build(g, p64, device=dev)
        cand = [f"{tf}x{128 // tf}@{c}" for tf in (16, 32, 64) for c in (8, 16, 32)]
        tuning = {"choice": {**choice, **bchoice}, "candidate_ms": {
            "tc_group_4_8_16": tms[0:3], "box_nb_32_64": tms[3:5], "root_nb_128_256_at_4096": tms[5:7],
            "cpqr_cb_2_4_8": tms[7:10],
            "k_pairs_tile@ctas_per_sm": dict(zip(cand, bms[0:9])),
            "k_proxy_tile@ctas_per_sm": dict(zip(cand, bms[9:18])),
            "id_phase_cpqr_threads_128_256": bms[18:20]}}
    for _ in range(args.warmup):
        step(p64)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    stats = [step(p64) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms_region = e0.elapsed_time(e1)
    entries = sum(s["entries_generated"] for s in stats)
    ms_kern = sum(s["ms_entries"] for s in stats)
    value = job_throughput(ws, entries, ms_kern)
    ms_region_max = max_over_ranks(ws, ms_region)
    launches = int(sum(s["launches"] for s in stats))
    if rank != 0:
        return None
    s0 = stats[-1]
    # roofline of the step's dominant kernel, the column-pivoted QR of the ID matrices (device
    # time of its launch from the library's events; flops per matrix from the ncu counters)
    kq = KERNEL_COUNTS["k_cpqr"]
    qfresh = kq["src_sha"] == cpqr_src_sha()
    # algorithmic flops of the launch (16 per element per reflection step, from the ranks)
    q_ach = s0["cpqr_flops"] / (s0["ms_cpqr"] * 1e-3) / 1e12
    roof_q = {"bound": "alu", "achieved": q_ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
              "frac": q_ach / FP64_PEAK_TFLOPS,
              "traffic": (kq["dram_bytes_per_matrix"] * s0["cpqr_matrices"])
                         if (qfresh and kq["dram_bytes_per_matrix"]) else None,
              "kernel": "k_cpqr", "matrices_per_launch": s0["cpqr_matrices"],
              "flops_per_launch": s0["cpqr_flops"], "ms_per_launch": s0["ms_cpqr"],
              "peak_note": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (unit counts); a DFMA "
                           "microbenchmark reached 1.013 TFLOP/s",
              "counts_fresh": qfresh}
    # the fused LU + solve launches of the factor (box LU with D^-1 L, and Dhat = M^-1)
    kl = KERNEL_COUNTS.get("k_lu_solve_fused", {})
    lfresh = kl.get("src_sha") == lu_src_sha()
    roof_l = None
    if s0["ms_lu"] > 0 and s0.get("lu_tc_matrices", 0) > 0:
        # the box factors on the tensor cores: FP64 panels + batched tensor-core products; the
        # FP64-equivalent rate has no single-pipe peak (the products' roofline is the
        # tensor-core GEMM's, in the extras)
        l_ach = s0["lu_flops"] / (s0["ms_lu"] * 1e-3) / 1e12
        roof_l = {"bound": "tensor", "achieved": l_ach, "peak": None, "unit": "TFLOP/s (FP64-equivalent)",
                  "frac": None, "traffic": None,
                  "kernel": "batched box LU + solve (k_lu_panel FP64 panels, k_zgemm_tc products)",
                  "matrices_per_step": s0["lu_matrices"], "flops_per_step": s0["lu_flops"],
                  "ms_per_step": s0["ms_lu"],
                  "peak_note": "FP64-equivalent algorithmic flops of LU + solve over the device time of "
                               "the whole sequence (panels, inverses, digit splits, products)"}
    elif s0["ms_lu"] > 0:
        l_ach = s0["lu_flops"] / (s0["ms_lu"] * 1e-3) / 1e12
        roof_l = {"bound": "alu", "achieved": l_ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": l_ach / FP64_PEAK_TFLOPS,
                  "traffic": (kl["dram_bytes_per_matrix"] * s0["lu_matrices"])
                             if (lfresh and kl.get("dram_bytes_per_matrix")) else None,
                  "kernel": "k_lu_solve_fused", "matrices_per_step": s0["lu_matrices"],
                  "launches_per_step": 2, "flops_per_step": s0["lu_flops"], "ms_per_step": s0["ms_lu"],
                  "peak_note": roof_q["peak_note"], "counts_fresh": lfresh}
    # the headline roofline is the kernel with the larger device time per step
    roof_main, roof_other = roof_q, roof_l
    if roof_l is not None and roof_l["frac"] is not None and s0["ms_lu"] > s0["ms_cpqr"]:
        roof_main, roof_other = roof_l, roof_q
    # roofline of the dominant entry kernel (the metric's entries/s)
    dom = "k_proxy" if s0["ms_proxy"] >= s0["ms_pairs"] else "k_pairs"
    pairs = s0["pairs_proxy"] if dom == "k_proxy" else s0["pairs_pairs"]
    ms_dom = s0["ms_proxy"] if dom == "k_proxy" else s0["ms_pairs"]
    kc = KERNEL_COUNTS[dom]
    tf_now = binding.wsbm_tuning()["pair_tf" if dom == "k_pairs" else "proxy_tf"]
    fresh = KERNEL_COUNTS["src_sha"] == kernel_src_sha() and kc["tf"] == tf_now
    fl = kc["fp64_flops_per_pair"] if fresh else None
    achieved = (pairs * fl / (ms_dom * 1e-3) / 1e12) if fl else None
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
            "traffic": (kc["dram_bytes_per_pair"] * pairs) if (fresh and kc["dram_bytes_per_pair"]) else None,
            "kernel": dom, "pairs_per_launch": pairs, "ms_per_launch": ms_dom,
            "entries_per_s_kernel": (s0["entries_proxy"] if dom == "k_proxy" else s0["entries_pairs"]) / (ms_dom * 1e-3),
            "peak_note": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (unit counts); a DFMA "
                         "microbenchmark reached 1.013 TFLOP/s",
            "counts_fresh": fresh}
    for r in (roof_main, roof_other, roof):
        add_fracs(r, clk)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_region_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {k: cfg[k] for k in ("workload", "N", "k0", "n", "leaf", "nproxy", "tol", "l2")},
           "gpu_launches": launches, "clocks": clk, "roofline": roof_main,
           "roofline_" + ("lu" if roof_other is roof_l else "cpqr") + "_kernel": roof_other,
           "roofline_entry_kernel": roof,
           "tuning": tuning if tuning is not None else binding.wsbm_tuning(),
           "step": {"entries_per_step": entries / args.steps,
                    "build_factor_s_leaf_level": ms_region / args.steps / 1e3,
                    "ms_entries": ms_kern / args.steps,
                    "ms_id": sum(s["ms_id"] for s in stats) / args.steps,
                    "ms_factor": sum(s["ms_factor"] for s in stats) / args.steps,
                    "leaf_rank_max": s0["rank_per_level"][-1] if s0["rank_per_level"] else None,
                    "sketched_id_matrices": s0["sketch_matrices"],
                    "sketch_fallbacks": s0["sketch_fallbacks"], "ms_sketch": s0["ms_sketch"],
                    "ms_cpqr": s0["ms_cpqr"], "ms_lu_fused": s0["ms_lu"]}}
    if args.step_only:
        return out
    out["e2e"] = run_e2e(args, curve, cfg, dev, params)
    if ws == 1:
        out["cpu_baseline"] = run_cpu_baseline(curve, cfg, budget_s=12.0)
    if not args.no_extras:
        # the extras are context for the line above: a failure there must not cost the line
        try:
            out["extras"] = run_extras(curve, cfg, dev, params)
        except Exception as exc:  # noqa: BLE001
            out["extras"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    return out


def run_e2e(args, curve, cfg, dev, params):
    """Same metric through the C ABI with the curve in pinned host memory: every step copies
    the geometry host -> device, builds the leaf level and reads its result (the ranks and the
    QR permutations that give the skeletons, which wsbm_factor reads back to the host; then the
    skeleton lists through wsbm_box_skeletons).  Beside it, the user pipeline of the full HSS on
    the 16384-node star: geometry and angles in, create, factor, plane-wave right-hand sides,
    solve, far field, far field out."""
    import torch
    from paper_2607_00790_gb300 import binding, inputs

    host = {k: torch.as_tensor(curve[k], dtype=torch.float64).pin_memory()
            for k in ("x", "y", "nx", "ny", "w", "kappa")}
    devt = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    g = binding.Geom(curve["x"].size, *[devt[k].data_ptr() for k in ("x", "y", "nx", "ny", "w", "kappa")])
    p = params()
    steps = max(1, min(args.steps, 3))
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    entries, d2h = 0, 0
    e0.record(stream)
    for _ in range(steps):
        for k in host:
            devt[k].copy_(host[k], non_blocking=True)
        s = binding.Solver(g, p, device=dev)
        s.factor()
        st = s.stats()
        entries += st["entries_generated"]
        L, nb = st["levels"], st["nboxes_leaf"]
        ks = 0
        for b in range(nb):
            jr, jc = s.skeletons(L, b, cap=512)
            ks += jr.size
        s.close()
        # read back inside wsbm_factor: QR state (4 int32 per box) and the row and column
        # permutations of every box's candidates (2 x 2N int32)
        d2h += 16 * nb + 2 * 2 * curve["x"].size * 4
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d = sum(v.numel() * 8 for v in host.values())
    out = {"value": entries / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h // steps, "steps": steps,
           "note": "H2D of the curve from pinned memory, create, leaf-level build incl. ID and factor, "
                   "D2H of the ranks and QR permutations (skeletons, read by wsbm_factor) and the "
                   "skeleton lists through wsbm_box_skeletons; the factors stay resident in HBM"}
    # the user pipeline on the star workload (full HSS): in -> factor -> solve -> far field -> out
    c16 = inputs.star(16384)
    h16 = {k: torch.as_tensor(c16[k], dtype=torch.float64).pin_memory()
           for k in ("x", "y", "nx", "ny", "w", "kappa")}
    d16 = {k: torch.empty_like(v, device=dev) for k, v in h16.items()}
    g16 = binding.Geom(16384, *[d16[k].data_ptr() for k in ("x", "y", "nx", "ny", "w", "kappa")])
    p16 = binding.make_params(float(inputs.k0_for_density(c16)), 1.5, leaf=128, nproxy=128, id_tol=1e-8)
    ang_h = torch.tensor(2 * np.pi * np.arange(8) / 8, dtype=torch.float64).pin_memory()
    obs_h = torch.tensor(2 * np.pi * np.arange(360) / 360, dtype=torch.float64).pin_memory()
    ff_h = torch.empty((360, 8), dtype=torch.complex128).pin_memory()

    def pipeline():
        for k in h16:
            d16[k].copy_(h16[k], non_blocking=True)
        ang = ang_h.to(dev, non_blocking=True)
        obs = obs_h.to(dev, non_blocking=True)
        s = binding.Solver(g16, p16, device=dev)
        s.factor()
        n_ent = s.stats()["entries_generated"]
        u, q = s.solve(s.rhs_planewave(ang))
        ff_h.copy_(s.farfield(u, q, obs), non_blocking=True)
        torch.cuda.synchronize()
        s.close()
        return n_ent

    pipeline()  # warm-up
    t = time.time()
    n_ent = pipeline()
    wall = time.time() - t
    out["pipeline_star16384_full"] = {
        "seconds": wall, "entries_per_s": n_ent / wall,
        "h2d_bytes": sum(v.numel() * 8 for v in h16.values()) + (8 + 360) * 8,
        "d2h_bytes": ff_h.numel() * 16,
        "steps": "H2D curve and angles, wsbm_create, wsbm_factor (full HSS), wsbm_rhs_planewave, "
                 "wsbm_solve (8 plane waves), wsbm_farfield (360 angles), D2H far field"}
    return out


# --------------------------------------------------------------------- CPU oracle ----
def oracle_sample(curve, cfg, budget_s):
    """The oracle computing the entries of whole leaf boxes of the same build (diagonal block,
    near blocks with the nodes inside the proxy circle, proxy row and column blocks) until the
    budget is spent."""
    import oracle

    N = cfg["N"]
    ph = oracle.Physics(cfg["k0"], n=cfg["n"])
    L = 0
    while (N >> L) > cfg["leaf"]:
        L += 1
    nb = 1 << L
    rng = np.random.default_rng(11)
    entries, boxes = 0, 0
    t0 = time.time()
    cut = cfg["tol"] / (4.0 * np.sqrt(nb))  # the library's QR cutoff for 2^L leaf boxes
    while True:
        b = int(rng.integers(0, nb))
        lo, hi = b * N // nb, (b + 1) * N // nb
        nodes = np.arange(lo, hi)
        unk = np.concatenate([nodes, nodes + N])
        cx, cy, rho = oracle.proxy_circle(curve, nodes)
        P = int(np.ceil(ph.k1 * rho + np.log(1 / cut) / np.log(1.5)))
        P = max(P, cfg["nproxy"])
        P = (P + 7) // 8 * 8
        D = oracle.wsbm_entries(curve, ph, unk, unk)
        entries += D.size
        # near unknowns: every node of the other boxes inside the proxy circle
        d = np.hypot(curve["x"] - cx, curve["y"] - cy)
        inside = np.nonzero(d < rho)[0]
        inside = inside[(inside < lo) | (inside >= hi)]
        su = np.concatenate([inside, inside + N])
        entries += oracle.wsbm_entries(curve, ph, unk, su).size
        entries += oracle.wsbm_entries(curve, ph, su, unk).size
        entries += oracle.proxy_row_block(curve, ph, unk, (cx, cy, rho), P).size
        entries += oracle.proxy_col_block(curve, ph, unk, (cx, cy, rho), P).size
        boxes += 1
        if time.time() - t0 >= budget_s:
            break
    el = time.time() - t0
    return entries, el, boxes


def cpu_model():
    """CPU model of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cores():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count()


def run_cpu_baseline(curve, cfg, budget_s):
    entries, el, boxes = oracle_sample(curve, cfg, budget_s)
    return {"value": entries / el, "unit": UNIT, "cores": cores(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{boxes} random leaf boxes of the N=262144 build: diagonal, near and proxy "
                      f"blocks ({entries} entries, {el:.1f} s; long-double libstdc++ Hankel, OpenMP)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    curve, cfg = workload()
    oracle_sample(curve, cfg, 0.0)  # load / build the oracle outside the timed steps
    for _ in range(args.warmup):
        oracle_sample(curve, cfg, 0.0)
    tot_e, tot_t, tot_b = 0, 0.0, 0
    for _ in range(args.steps):
        e, t, b = oracle_sample(curve, cfg, 0.0)
        tot_e += e
        tot_t += t
        tot_b += b
    v = tot_e / tot_t
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {k: cfg[k] for k in ("workload", "N", "k0", "n", "leaf", "nproxy", "tol")},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores(), "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": f"one random leaf box of the build per step ({tot_b} boxes)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------------- extras ----
def run_extras(curve, cfg, dev, params):
    """Untimed-by-contract measurements: mixed path, full HSS where the root fits."""
    import torch
    from paper_2607_00790_gb300 import binding, inputs

    out = {}
    # the whole build + factor at N = 2^18 (the metric's build+factor seconds), first
    out["full_2p18_fp64_tol1e-8"] = run_full_2p18(dev)
    out["roofline_tc_gemm"] = run_tc_gemm(dev)
    g, keep = binding.make_geom(curve, device=dev)

    def build(gg, p):
        s = binding.Solver(gg, p, device=dev)
        t = time.time()
        s.factor()
        torch.cuda.synchronize()
        st = s.stats()
        st["wall_s"] = time.time() - t
        return s, st

    # mixed precision leaf-level build at N = 2^18 (ID tol 1e-6), against FP64 at the same tol
    res = {}
    for name, prec in (("fp64", binding.WSBM_FP64), ("mixed", binding.WSBM_MIXED),
                       ("mixed_fine", binding.WSBM_MIXED_FINE)):
        build(g, params(prec, 1e-6))
        s, st = build(g, params(prec, 1e-6))
        res[name] = {"entries_per_s": st["entries_generated"] / (st["ms_entries"] * 1e-3),
                     "proxy_entries_per_s": st["entries_proxy"] / (st["ms_proxy"] * 1e-3),
                     "build_factor_s": st["ms_total_factor"] / 1e3}
        s.close()
    res["proxy_kernel_speedup"] = res["mixed"]["proxy_entries_per_s"] / res["fp64"]["proxy_entries_per_s"]
    res["proxy_kernel_speedup_fine"] = (res["mixed_fine"]["proxy_entries_per_s"] /
                                        res["fp64"]["proxy_entries_per_s"])
    out["mixed_vs_fp64_2p18_leaf_level_tol1e-6"] = res

    # full HSS on the 16384-node star (the largest 15 nodes/wavelength case whose root fits):
    # FP64 and mixed, far field of the mixed path against the FP64 path
    c16 = inputs.star(16384)
    g16, k16 = binding.make_geom(c16, device=dev)
    ang = torch.tensor(2 * np.pi * np.arange(8) / 8, device=dev)
    obs = torch.tensor(2 * np.pi * np.arange(360) / 360, device=dev)
    ffs = {}
    for name, prec, tol in (("fp64_tol1e-8", binding.WSBM_FP64, 1e-8), ("fp64_tol1e-6", binding.WSBM_FP64, 1e-6),
                            ("mixed_tol1e-6", binding.WSBM_MIXED, 1e-6), ("fp64_tol1e-7", binding.WSBM_FP64, 1e-7),
                            ("mixed_fine_tol1e-7", binding.WSBM_MIXED_FINE, 1e-7)):
        p = binding.make_params(float(inputs.k0_for_density(c16)), 1.5, leaf=128, nproxy=128,
                                id_tol=tol, precision=prec)
        s, st = build(g16, p)
        t = time.time()
        rhs = s.rhs_planewave(ang)
        u, q = s.solve(rhs)
        ff = s.farfield(u, q, obs)
        torch.cuda.synchronize()
        ffs[name] = ff.cpu().numpy()
        out[f"star16384_full_{name}"] = {"build_factor_s": st["ms_total_factor"] / 1e3,
                                         "solve_farfield_s": time.time() - t,
                                         "ms_entries": st["ms_entries"], "ms_id": st["ms_id"],
                                         "ms_factor": st["ms_factor"], "root_size": st["root_size"],
                                         "rank_per_level": st["rank_per_level"]}
        s.close()
    ref = ffs["fp64_tol1e-8"]
    for name in ("fp64_tol1e-6", "mixed_tol1e-6", "fp64_tol1e-7", "mixed_fine_tol1e-7"):
        out[f"star16384_full_{name}"]["farfield_rel_err_vs_fp64_tol1e-8"] = float(
            np.linalg.norm(ffs[name] - ref) / np.linalg.norm(ref))

    # batched scatterers: 64 seeded ellipses / stars (N in [2048, 32768], 15 nodes/wavelength,
    # n in [1.2, 2.0]); leaf-level builds in one batch (shared launches per phase) against the
    # same builds one curve at a time
    man = inputs.batched_manifest(0)
    curves, prms = [], []
    for m in man:
        c = (inputs.ellipse(m["N"], m["geo"]["a"], m["geo"]["b"]) if m["kind"] == "ellipse"
             else inputs.star(m["N"], m["geo"]["a"], m["geo"]["m"]))
        curves.append(c)
        prms.append(binding.make_params(float(inputs.k0_for_density(c)), m["n"], leaf=128,
                                        nproxy=128, id_tol=1e-8, max_levels=1))
    geoms = [binding.make_geom(c, device=dev) for c in curves]
    bt = binding.Batch([g for g, _ in geoms], prms, device=dev)
    bt.factor()
    torch.cuda.synchronize()
    t = time.time()
    bt.factor()
    torch.cuda.synchronize()
    t_batch = time.time() - t
    bst = bt.stats()
    bt.close()
    t = time.time()
    ent = 0
    for (g2, _), p2 in zip(geoms, prms):
        s = binding.Solver(g2, p2, device=dev)
        s.factor()
        ent += s.stats()["entries_generated"]
        s.close()
    torch.cuda.synchronize()
    t_seq = time.time() - t
    out["batched_64_scatterers_leaf_level"] = {
        "nodes_total": int(sum(m["N"] for m in man)), "launches_batch": bst["launches"],
        "build_factor_s_batch": t_batch, "build_factor_s_one_by_one": t_seq,
        "speedup": t_seq / t_batch, "entries": bst["entries_generated"],
        "entries_per_s_kernel": bst["entries_generated"] / (bst["ms_entries"] * 1e-3),
        "ms_entries": bst["ms_entries"], "ms_id": bst["ms_id"], "ms_factor": bst["ms_factor"]}

    # full HSS at N = 2^18 with the paper's Table para physics (eps1 = 5, omega = 10)
    p = binding.make_params(10.0, float(np.sqrt(5.0)), eps1=5.0, leaf=128, nproxy=128, id_tol=1e-8)
    s, st = build(g, p)
    t = time.time()
    rhs = s.rhs_planewave(ang)
    u, q = s.solve(rhs)
    s.farfield(u, q, obs)
    torch.cuda.synchronize()
    out["paper_table_2p18_full_fp64"] = {"build_factor_s": st["ms_total_factor"] / 1e3,
                                         "solve_farfield_s": time.time() - t,
                                         "entries_per_s": st["entries_generated"] / (st["ms_entries"] * 1e-3),
                                         "root_size": st["root_size"], "rank_per_level": st["rank_per_level"]}
    # field off the curve from that solution: 4096 points inside (half radius) and 4096 outside
    # (1.5 radius) of the star, 8 right-hand sides
    tt = 2 * np.pi * (np.arange(8192) + 0.5) / 8192
    rr = (1.0 + 0.3 * np.cos(5 * tt)) * np.where(np.arange(8192) < 4096, 0.5, 1.5)
    tx = torch.tensor(rr * np.cos(tt), device=dev)
    ty = torch.tensor(rr * np.sin(tt), device=dev)
    binding.field(g, p, u, q, tx, ty)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, ins = binding.field(g, p, u, q, tx, ty)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["field_2p18_8192_points_8_rhs"] = {
        "ms": ms, "pairs_per_s": 8192 * curve["x"].size / (ms * 1e-3),
        "inside_points": int(ins.sum().item()), "note": "one Hankel evaluation per pair shared by 8 RHS"}
    s.close()
    out["adjoint_fourier_32768"] = run_adjoint(dev, fd=("a8", "n"))
    out["batched_solve_16_scatterers_256_rhs"] = run_batched_solve(dev)
    return out


_FULL_TUNING = {}


def run_full_2p18(dev, precision=0, tol=1e-8, rows=256, refine=True, ff_ref=None):
    """The whole HSS build + factor at the bench workload (N = 2^18, 15 nodes per wavelength):
    every level compressed while the one-CTA QR takes its boxes, then the dense root factored by
    the LU whose trailing updates run on the tensor cores.  Accuracy: the relative residual on
    `rows` random equations (entries from wsbm_entries, which matches the oracle to 1e-12), and
    the far-field change under one step of iterative refinement with the dense matrix-free
    product (the far-field error of the HSS solution, to within the refined error)."""
    import torch
    from paper_2607_00790_gb300 import binding, inputs
    curve, cfg = workload()
    N = cfg["N"]
    g, keep = binding.make_geom(curve, device=dev)
    p = binding.make_params(cfg["k0"], cfg["n"], leaf=cfg["leaf"], nproxy=cfg["nproxy"], id_tol=tol,
                            precision=precision, root_cap=200000)
    # the tensor-core shapes timed once per process, before the build; the root panel width is
    # timed on a 4096-unknown matrix (its class below 12288 unknowns), so the large class keeps
    # its width (256): a timing at 16384 unknowns does not carry over to a root of ~1e5
    if not _FULL_TUNING:
        choice, tms = binding.wsbm_autotune(n_box=2 * cfg["leaf"], nbox=N // cfg["leaf"], nrhs_box=128,
                                            n_root=4096, device=dev)
        _FULL_TUNING.update(choice=choice, candidate_ms={
            "tc_group_4_8_16": tms[0:3], "box_nb_32_64": tms[3:5], "root_nb_128_256_at_4096": tms[5:7],
            "cpqr_cb_2_4_8": tms[7:10]})
    tuning = dict(_FULL_TUNING)
    binding.trim_memory()
    s = binding.Solver(g, p, device=dev)
    t = time.time()
    s.factor()
    torch.cuda.synchronize()
    wall = time.time() - t
    st = s.stats()
    ang = torch.tensor(2 * np.pi * np.arange(8) / 8, device=dev)
    obs = torch.tensor(2 * np.pi * np.arange(360) / 360, device=dev)
    t = time.time()
    rhs = s.rhs_planewave(ang)
    u, q = s.solve(rhs)
    ff = s.farfield(u, q, obs)
    torch.cuda.synchronize()
    t_solve = time.time() - t
    # residual on random equations
    rng = np.random.default_rng(17)
    ridx = torch.tensor(np.sort(rng.choice(2 * N, rows, replace=False)), device=dev)
    cols = torch.arange(2 * N, device=dev)
    x = torch.cat([u, q], dim=0)
    Arows = s.entries(ridx, cols)
    r = Arows @ x - rhs[ridx]
    res_rows = (torch.linalg.norm(r) / torch.linalg.norm(rhs[ridx])).item()
    if not refine:
        out = {"build_factor_s": st["ms_total_factor"] / 1e3, "ms_entries": st["ms_entries"],
               "ms_id": st["ms_id"], "ms_factor": st["ms_factor"], "root_size": st["root_size"],
               "rank_per_level": st["rank_per_level"], "id_tol": tol, "precision": precision,
               "solve_8rhs_farfield_s": t_solve, "residual_rel_sampled_rows": res_rows,
               "tuning": tuning}
        if ff_ref is not None:
            out["farfield_rel_err_vs_fp64_tol1e-8"] = float(
                np.linalg.norm(ff.cpu().numpy() - ff_ref) / np.linalg.norm(ff_ref))
        s.close()
        binding.trim_memory()
        return out, ff.cpu().numpy()
    # one refinement step for the first plane wave: r = b - A x (matrix-free, O(N^2)),
    # x1 = x + HSS^-1 r
    t = time.time()
    b0, x0 = rhs[:, :1].contiguous(), x[:, :1].contiguous()
    rfull = b0 - binding.wsbm_matvec(g, p, x0)
    res_full = (torch.linalg.norm(rfull) / torch.linalg.norm(b0)).item()
    du, dq = s.solve(rfull)
    ff1 = s.farfield(u[:, :1] + du, q[:, :1] + dq, obs)
    torch.cuda.synchronize()
    t_ref = time.time() - t
    ff_err = (torch.linalg.norm(ff[:, :1] - ff1) / torch.linalg.norm(ff1)).item()
    u_err = (torch.linalg.norm(du) / torch.linalg.norm(u[:, :1] + du)).item()
    out = {"build_factor_s": st["ms_total_factor"] / 1e3, "wall_s": wall,
           "ms_entries": st["ms_entries"], "ms_id": st["ms_id"], "ms_factor": st["ms_factor"],
           "root_size": st["root_size"], "rank_per_level": st["rank_per_level"],
           "factor_bytes": st["factor_bytes"], "entries": st["entries_generated"],
           "entries_per_s": st["entries_generated"] / (st["ms_entries"] * 1e-3),
           "solve_8rhs_farfield_s": t_solve, "id_tol": tol, "precision": precision,
           "residual_rel_full_angle0": res_full, "residual_rel_sampled_rows": res_rows,
           "farfield_rel_err_vs_one_refinement_step_angle0": ff_err,
           "density_rel_correction_angle0": u_err,
           "refinement_step_s": t_ref, "tuning": tuning}
    s.close()
    binding.trim_memory()
    return out


def run_tc_gemm(dev, m=16384, n=16384, k=128, reps=5):
    """Roofline of the tensor-core complex GEMM (the trailing update of the root LU): device
    time on its stream over `reps` calls; executed tensor work 272 flops per complex
    multiply-add (34 digit pairs x 4 real products x 2), against the measured BF16 peak."""
    import ctypes

    import torch
    from paper_2607_00790_gb300 import binding
    A = torch.randn(k, m, dtype=torch.complex128, device=dev)  # column-major m x k
    B = torch.randn(n, k, dtype=torch.complex128, device=dev)  # column-major k x n
    C = torch.zeros(n, m, dtype=torch.complex128, device=dev)
    al = (ctypes.c_double * 2)(-1.0, 0.0)
    be = (ctypes.c_double * 2)(1.0, 0.0)
    L = binding.lib()
    st = torch.cuda.current_stream(dev)

    def call():
        rc = L.wsbm_zgemm(m, n, k, al, ctypes.c_void_p(A.data_ptr()), m, ctypes.c_void_p(B.data_ptr()), k,
                          be, ctypes.c_void_p(C.data_ptr()), m, ctypes.c_void_p(st.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"wsbm_zgemm: {rc}")

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        call()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    peaks = measured_peaks()
    pk = peaks.get("bf16_tflops") or 1900.0
    tflops = 272.0 * m * n * k / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": tflops, "peak": pk, "unit": "TFLOP/s",
            "frac": tflops / pk, "traffic": None, "kernel": "k_zgemm_tc (+ digit split kernels)",
            "shape": [m, n, k], "ms_per_call": ms,
            "fp64_equivalent_tflops": 8.0 * m * n * k / (ms * 1e-3) / 1e12,
            "peak_note": "of measured" if peaks.get("bf16_tflops") else "of fallback",
            "work_note": "executed BF16 tensor flops of the digit products (34 digit pairs per "
                         "real product, 4 real products per complex); the call time includes "
                         "the digit-split kernels"}


def run_tc_sweep(dev):
    """The tensor-core complex GEMM at the shapes of the root LU's trailing updates, and the
    LU of dense complex matrices (wsbm_lu_dense) at 16384 and 32768 unknowns (complex LU:
    n^3 / 3 complex multiply-adds = 8/3 n^3 real flops)."""
    import torch
    from paper_2607_00790_gb300 import binding
    out = {"gemm": [run_tc_gemm(dev, m, n, k) for m, n, k in
                    ((4096, 4096, 128), (16384, 16384, 128), (16384, 16384, 256), (8192, 8192, 512),
                     (32768, 32768, 256))]}
    torch.cuda.empty_cache()
    lu = []
    for n in (16384, 32768):
        g = torch.Generator(device=dev).manual_seed(n)
        A = torch.randn(n, n, dtype=torch.complex128, device=dev, generator=g)
        A.diagonal().add_(4.0 * n ** 0.5)
        binding.wsbm_lu_dense(A.clone())  # warm-up (work space, opt-ins)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        LU, piv = binding.wsbm_lu_dense(A)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        lu.append({"n": n, "ms": ms, "fp64_equivalent_tflops": 8.0 / 3.0 * n ** 3 / (ms * 1e-3) / 1e12})
        del A, LU, piv
        torch.cuda.empty_cache()
    out["lu_dense"] = lu
    out["tuning"] = binding.wsbm_tuning()
    return out


def run_formulations(dev, N=262144, tol=1e-8):
    """Leaf-level build (entries, IDs, leaf factors) of the star at N for the three
    formulations of Sec. II: eq. (weakly_bm), eq. (bm) and eq. (pmchwt).  The paper reports the
    standard Burton-Miller solver 10-20 % faster than the weakly singular one and PMCHWT about
    equal; here the two comparison formulations run on plain (untuned) entry kernels."""
    import torch
    from paper_2607_00790_gb300 import binding, inputs
    c = inputs.star(N)
    k0 = float(inputs.k0_for_density(c))
    g, keep = binding.make_geom(c, device=dev)
    out = {}
    for name, form in (("wsbm", 0), ("bm", 1), ("pmchwt", 2)):
        p = binding.make_params(k0, 1.5, leaf=128, nproxy=128, id_tol=tol, max_levels=1,
                                formulation=form)
        for rep in range(2):  # the first build warms up
            s = binding.Solver(g, p, device=dev)
            s.factor()
            torch.cuda.synchronize()
            st = s.stats()
            s.close()
        out[name] = {"build_factor_s": st["ms_total_factor"] / 1e3, "ms_entries": st["ms_entries"],
                     "ms_id": st["ms_id"], "ms_factor": st["ms_factor"],
                     "entries_per_s": st["entries_generated"] / (st["ms_entries"] * 1e-3),
                     "leaf_rank_max": st["max_rank"]}
    return {"N": N, "id_tol": tol, **out}


def run_batched_solve(dev, count=16, nmax=16384, nrhs=256, tol=1e-8):
    """Full HSS of the first `count` scatterers of the batched manifest with N <= nmax (batched
    factor), then `nrhs` plane waves each: one batched solve plan (shared launches per tree
    step, CUDA graph) against per-curve solves (each its own graph).  Both are warmed up once;
    the timed calls are graph replays plus the copies in and out."""
    import torch
    from paper_2607_00790_gb300 import binding, inputs

    man = [m for m in inputs.batched_manifest(0) if m["N"] <= nmax][:count]
    curves, prms = [], []
    for m in man:
        c = (inputs.ellipse(m["N"], m["geo"]["a"], m["geo"]["b"]) if m["kind"] == "ellipse"
             else inputs.star(m["N"], m["geo"]["a"], m["geo"]["m"]))
        curves.append(c)
        prms.append(binding.make_params(float(inputs.k0_for_density(c)), m["n"], leaf=128,
                                        nproxy=128, id_tol=tol))
    geoms = [binding.make_geom(c, device=dev) for c in curves]
    bt = binding.Batch([g for g, _ in geoms], prms, device=dev)
    torch.cuda.synchronize()
    t = time.time()
    bt.factor()
    torch.cuda.synchronize()
    t_factor = time.time() - t
    binding.trim_memory()  # the build's cached work space back to the device
    bst = bt.stats()
    free_b, total_b = torch.cuda.mem_get_info(dev)
    ang = torch.tensor(2 * np.pi * np.arange(nrhs) / nrhs, device=dev)
    rhs = [bt.solver(i).rhs_planewave(ang) for i in range(len(man))]
    out = {"scatterers": len(man), "nodes_total": int(sum(m["N"] for m in man)), "nrhs": nrhs,
           "id_tol": tol, "batch_factor_s": t_factor, "factor_bytes": bst["factor_bytes"],
           "largest_root": bst["root_size"], "device_free_bytes_after_factor": free_b,
           "rhs_bytes": int(sum(r.numel() * 16 for r in rhs))}

    def timed(f, reps=3):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.time()
            f()
            torch.cuda.synchronize()
            ts.append(time.time() - t0)
        return min(ts)

    # all right-hand sides in one plan when they fit, else in column chunks (each plan holds its
    # own copies of the right-hand sides and solutions)
    chunk = nrhs
    while True:
        try:
            parts = [[r[:, c:c + chunk].contiguous() for r in rhs] for c in range(0, nrhs, chunk)]
            out["batched_solve_s"] = timed(lambda: [bt.solve(pr) for pr in parts])
            break
        except binding.WsbmError as exc:
            if exc.code != -2 or chunk <= 8:
                raise
            parts = None
            chunk //= 2
            torch.cuda.empty_cache()
            binding.trim_memory()
    out["rhs_per_plan"] = chunk
    # per-curve solves, one curve at a time (each handle caches its own plan: after timing it is
    # replaced by a one-column plan so that only one large plan exists at a time; the batch's
    # own plan likewise first)
    one = [torch.zeros((r.shape[0], 1), dtype=r.dtype, device=dev) for r in rhs]
    bt.solve(one)
    binding.trim_memory()
    tot = 0.0
    for i in range(len(man)):
        sv = bt.solver(i)
        tot += timed(lambda: [sv.solve(pr[i]) for pr in parts])
        sv.solve(one[i])
    out["per_curve_solves_s"] = tot
    out["speedup"] = out["per_curve_solves_s"] / out["batched_solve_s"]
    out["rhs_per_s_batched"] = len(man) * nrhs / out["batched_solve_s"]
    bt.close()
    return out


def run_adjoint(dev, N=32768, fd=("a1", "a8", "a16", "b3", "b12", "n"), tol=1e-8, h=1e-6,
                refine=2):
    """Shape / refractive-index gradient of the far-field intensity misfit on the Fourier
    curve (coefficients ~ N(0, 0.02^2), seed 1; target shape seed 2; k0 for 15 nodes per
    wavelength of the initial shape; n = 1.5; one plane wave at 0; 64 far-field angles).
    The gradient runs the library calls that autograd.FarField makes: HSS factor, solve,
    far field; far-field reverse map, transposed HSS solve, right-hand-side reverse map,
    pairwise backward kernel, curve reverse map; solution and multipliers refined `refine`
    times against the dense matrix-free products.  The check is a central difference (step h)
    of the loss with each perturbed system solved to rounding level by refinement (HSS factor
    at the unperturbed shape as preconditioner)."""
    import torch
    from paper_2607_00790_gb300 import autograd as ag
    from paper_2607_00790_gb300 import binding, inputs

    a, b = inputs.shape_coefficients(1)
    at, bt = inputs.shape_coefficients(2)
    k0 = float(inputs.k0_for_density(inputs.fourier(N, a, b)))
    n = 1.5
    T = lambda v: torch.as_tensor(np.asarray(v, dtype=np.float64), device=dev)
    inc, obs = T([0.0]), T(2 * np.pi * np.arange(64) / 64)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def sync_time(f):
        torch.cuda.synchronize()
        t = time.time()
        r = f()
        torch.cuda.synchronize()
        return r, time.time() - t

    with torch.no_grad():
        Ft = ag.farfield(ag.fourier_curve(T(at), T(bt), N), T(n), k0, inc, obs, leaf=128,
                         nproxy=128, tol=tol, refine=refine)
        target = Ft[:, 0].abs() ** 2
    out = {"N": N, "k0": k0, "n": n, "id_tol": tol, "nobs": 64, "refine_steps": refine}
    ta, tb = T(a), T(b)
    cur = binding.curve_fourier(ta, tb, N)
    geom, keep = binding.geom_from_tensors(*[cur[k] for k in range(6)])
    prm = binding.make_params(k0, n, leaf=128, nproxy=128, id_tol=tol)
    s = binding.Solver(geom, prm, device=dev)

    def forward():
        s.factor()
        rhs = s.rhs_planewave(inc)
        u, q = s.solve(rhs)
        u, q, res = s.refine(geom, prm, rhs, u, q, iters=refine)
        F = s.farfield(u, q, obs)
        return rhs, u, q, res, F

    (rhs, u, q, res, F), t_fwd = sync_time(forward)
    L = torch.sum((F[:, 0].abs() ** 2 - target) ** 2)
    e0, e1 = ev(), ev()

    def backward(u, q, F, nref):
        gF = (4.0 * (F.abs() ** 2 - target[:, None]) * F).contiguous()
        v, g_ff = binding.farfield_vjp(geom, prm, u, q, obs, gF)
        l1, l2 = s.solve_transposed(v)
        l1, l2, lres = s.refine(geom, prm, v, l1, l2, iters=nref, trans=True)
        lam = torch.cat([l1, l2])
        g_rhs = binding.rhs_planewave_vjp(geom, prm, inc, lam)
        e0.record()
        g_a, gph = binding.entries_vjp(geom, prm, lam[:, 0].contiguous(),
                                       torch.cat([u, q])[:, 0].contiguous())
        e1.record()
        g = g_ff + g_rhs - g_a
        gc = binding.curve_fourier_vjp(ta, tb, N, g)
        gn = -(gph[0] * k0 + gph[1] * 2.0 * n)
        return torch.cat([gc, gn.reshape(1)]), lres

    (gvec, lres), t_bwd = sync_time(lambda: backward(u, q, F, refine))
    grad = gvec.cpu().numpy()
    # the same gradient from the HSS solutions alone (no refinement)
    u0, q0 = s.solve(rhs)
    g_hss = backward(u0, q0, s.farfield(u0, q0, obs), 0)[0].cpu().numpy()
    out["hss_only_grad_max_rel_diff"] = float(np.max(np.abs(g_hss - grad) / np.abs(grad)))
    st = s.stats()
    e2, e3 = ev(), ev()
    xs = torch.cat([u, q])
    e2.record()
    binding.wsbm_matvec(geom, prm, xs)
    e3.record()
    torch.cuda.synchronize()
    ms_vjp, ms_mv = e0.elapsed_time(e1), e2.elapsed_time(e3)
    out.update(loss=L.item(), forward_s=t_fwd, backward_s=t_bwd,
               factor_s=st["ms_total_factor"] / 1e3, root_size=st["root_size"],
               rank_per_level=st["rank_per_level"], hss_residual=res[0], refined_residual=res[-1],
               adjoint_hss_residual=lres[0], adjoint_refined_residual=lres[-1],
               vjp_kernel_ms=ms_vjp, vjp_pairs_per_s=N * (N - 1) / (ms_vjp * 1e-3),
               matvec_ms=ms_mv, matvec_pairs_per_s=N * N / (ms_mv * 1e-3))

    def loss_at(aa, bb, nn):
        c2 = binding.curve_fourier(T(aa), T(bb), N)
        g2, k2 = binding.geom_from_tensors(*[c2[k] for k in range(6)])
        p2 = binding.make_params(k0, nn, leaf=128, nproxy=128, id_tol=tol)
        s2 = binding.Solver(g2, p2, device=dev)  # geometry and tree only (not factored)
        b2 = s2.rhs_planewave(inc)
        x = torch.cat([u, q])
        for _ in range(6):
            r = b2 - binding.wsbm_matvec(g2, p2, x)
            if torch.linalg.norm(r).item() <= 1e-14 * torch.linalg.norm(b2).item():
                break
            du, dq = s.solve(r)
            x = x + torch.cat([du, dq])
        F2 = s2.farfield(x[:N], x[N:], obs)
        s2.close()
        return torch.sum((F2[:, 0].abs() ** 2 - target) ** 2).item()

    def central(name, idx, step):
        vals = []
        for sgn in (1.0, -1.0):
            aa, bb, nn = a.copy(), b.copy(), n
            if name == "n":
                nn += sgn * step
            elif name[0] == "a":
                aa[idx] += sgn * step
            else:
                bb[idx - 16] += sgn * step
            vals.append(loss_at(aa, bb, nn))
        return (vals[0] - vals[1]) / (2 * step)

    # central differences with step h (the stated check) and h/2; their Richardson
    # combination removes the O(h^2) truncation term, which at k0 ~ 1.8e3 is the larger error
    fdres = {}
    t0 = time.time()
    for name in fd:
        idx = 32 if name == "n" else (int(name[1:]) - 1 + (16 if name[0] == "b" else 0))
        d1 = central(name, idx, h)
        d2 = central(name, idx, h / 2)
        rich = (4.0 * d2 - d1) / 3.0
        ga = float(grad[idx])
        fdres[name] = {"adjoint": ga, "central_h": d1, "central_h_half": d2, "richardson": rich,
                       "rel_err_vs_central_h": abs(ga - d1) / abs(d1),
                       "truncation_est_central_h": abs(d1 - rich) / abs(rich),
                       "rel_err_vs_richardson": abs(ga - rich) / abs(rich)}
    out["fd_s"] = time.time() - t0
    out["fd_step"] = h
    out["fd_check"] = fdres
    out["max_rel_err_vs_central_h"] = max(v["rel_err_vs_central_h"] for v in fdres.values())
    out["max_rel_err_vs_richardson"] = max(v["rel_err_vs_richardson"] for v in fdres.values())
    out["grad_norm"] = float(np.linalg.norm(grad))
    s.close()
    return out


def apply_tuning(spec):
    """Launch shapes of the current device from "key=value,..." (keys of binding.wsbm_tuning())."""
    from paper_2607_00790_gb300 import binding
    binding.wsbm_tuning_set(**{k: int(v) for k, v in (kv.split("=") for kv in spec.split(","))})


def profile_case(N=16384):
    import torch
    from paper_2607_00790_gb300 import binding, inputs
    c = inputs.star(N)
    g, keep = binding.make_geom(c)
    for prec in (binding.WSBM_FP64, binding.WSBM_MIXED, binding.WSBM_MIXED_FINE):
        p = binding.make_params(float(inputs.k0_for_density(c)), 1.5, leaf=128, nproxy=128,
                                id_tol=1e-8, precision=prec, max_levels=1)
        s = binding.Solver(g, p)
        s.factor()
        torch.cuda.synchronize()
        print(json.dumps({"precision": prec, **{k: v for k, v in s.stats().items() if k != "rank_per_level"}}))
        s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--profile-tc-shape", default="4096,4096,128",
                    help="m,n,k of the --profile-tc product")
    ap.add_argument("--tc-sweep", action="store_true",
                    help="tensor-core GEMM at several shapes and the dense LU at 16384 / 32768 unknowns")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of timing the candidates")
    ap.add_argument("--set-tuning", default="",
                    help="launch shapes to use instead of the autotuners, as key=value,... with the "
                         "keys of binding.wsbm_tuning() (e.g. pair_tf=32,pair_ctas=16)")
    ap.add_argument("--step-only", action="store_true",
                    help="only the warm-up and timed steps (no e2e, CPU baseline or extras): "
                         "the launch list of a step for ncu")
    ap.add_argument("--adjoint", action="store_true",
                    help="only the shape-gradient measurement (N = 32768 Fourier curve)")
    ap.add_argument("--adjoint-n", type=int, default=32768)
    ap.add_argument("--formulations", action="store_true",
                    help="only the leaf-level builds of the three formulations at N = 2^18")
    ap.add_argument("--batched-solve", action="store_true",
                    help="only the batched-solve measurement (16 scatterers, 256 right-hand sides)")
    ap.add_argument("--batch-count", type=int, default=16, help="scatterers of --batched-solve")
    ap.add_argument("--batch-nmax", type=int, default=16384, help="largest N of --batched-solve")
    ap.add_argument("--profile-case", action="store_true",
                    help="one leaf-level build of the star (small case for ncu) per precision mode")
    ap.add_argument("--profile-n", type=int, default=16384, help="nodes of the --profile-case star")
    ap.add_argument("--profile-tc", action="store_true",
                    help="two tensor-core GEMM calls, 4096 x 4096 x 128 (small case for ncu)")
    ap.add_argument("--full-2p18", action="store_true",
                    help="only the whole build + factor at N = 2^18 (FP64, and WSBM_MIXED_FINE "
                         "with --mixed-tol)")
    ap.add_argument("--mixed-tol", type=float, default=0.0)
    args = ap.parse_args()
    if args.set_tuning and (args.profile_case or args.profile_tc or args.full_2p18 or args.adjoint
                            or args.batched_solve or args.formulations or args.tc_sweep):
        apply_tuning(args.set_tuning)  # the single-GPU modes below run on device 0
    if args.profile_case:
        profile_case(args.profile_n)
        return
    if args.tc_sweep:
        print(json.dumps({"tc_sweep": run_tc_sweep("cuda")}), flush=True)
        return
    if args.profile_tc:
        m, n, k = (int(v) for v in args.profile_tc_shape.split(","))
        print(json.dumps(run_tc_gemm("cuda", m, n, k, reps=1)), flush=True)
        return
    if args.full_2p18:
        if args.mixed_tol > 0:
            # the mixed workload: far fields of FP64 and WSBM_MIXED_FINE builds at the given ID
            # tolerance against the FP64 build at tol 1e-8 (8 plane waves, 360 angles)
            r64, ff_ref = run_full_2p18("cuda", 0, 1e-8, refine=False)
            out = {"fp64_tol1e-8": r64}
            for name, prec in (("fp64", 0), ("mixed_fine", 2)):
                out[f"{name}_tol{args.mixed_tol:g}"], _ = run_full_2p18(
                    "cuda", prec, args.mixed_tol, refine=False, ff_ref=ff_ref)
        else:
            out = {"fp64": run_full_2p18("cuda")}
        print(json.dumps(out), flush=True)
        return
    if args.adjoint:
        print(json.dumps({"adjoint": run_adjoint("cuda", N=args.adjoint_n)}), flush=True)
        return
    if args.batched_solve:
        print(json.dumps({"batched_solve": run_batched_solve("cuda", count=args.batch_count,
                                                            nmax=args.batch_nmax)}), flush=True)
        return
    if args.formulations:
        print(json.dumps({"formulations": run_formulations("cuda")}), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_init()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
