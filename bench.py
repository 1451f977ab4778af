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
# (profiles/entry_kernels_ncu.md) for the kernel sources with the recorded hash; when the
# sources change the traffic figure is withheld until re-measured.
KERNEL_COUNTS = {
    "src_sha": None,
    "k_proxy": {"fp64_flops_per_pair": None, "dram_bytes_per_pair": None},
    "k_pairs": {"fp64_flops_per_pair": None, "dram_bytes_per_pair": None},
}
# FP64 peak from the unit counts: 152 SMs x 4 FP64 flops/clk/SM (2 DFMA) x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def kernel_src_sha():
    h = hashlib.sha256()
    for f in ("entries.cu", "hankel.cuh", "hankel_coeffs.inc"):
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


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


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
    tot_entries = sum_over_ranks(ws, entries)
    ms_kern_max = max_over_ranks(ws, ms_kern)
    ms_region_max = max_over_ranks(ws, ms_region)
    value = tot_entries / (ms_kern_max * 1e-3)
    launches = int(sum(s["launches"] for s in stats))
    if rank != 0:
        return None
    s0 = stats[-1]
    # roofline of the dominant entry kernel (device time per launch from the library's events)
    dom = "k_proxy" if s0["ms_proxy"] >= s0["ms_pairs"] else "k_pairs"
    pairs = s0["pairs_proxy"] if dom == "k_proxy" else s0["pairs_pairs"]
    ms_dom = s0["ms_proxy"] if dom == "k_proxy" else s0["ms_pairs"]
    kc = KERNEL_COUNTS[dom]
    fresh = KERNEL_COUNTS["src_sha"] == kernel_src_sha()
    fl = kc["fp64_flops_per_pair"]
    achieved = (pairs * fl / (ms_dom * 1e-3) / 1e12) if fl else None
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
            "traffic": (kc["dram_bytes_per_pair"] * pairs) if (fresh and kc["dram_bytes_per_pair"]) else None,
            "kernel": dom, "pairs_per_launch": pairs, "ms_per_launch": ms_dom,
            "entries_per_s_kernel": (s0["entries_proxy"] if dom == "k_proxy" else s0["entries_pairs"]) / (ms_dom * 1e-3),
            "peak_note": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (unit counts); a DFMA "
                         "microbenchmark reached 1.013 TFLOP/s",
            "counts_fresh": fresh}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_region_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {k: cfg[k] for k in ("workload", "N", "k0", "n", "leaf", "nproxy", "tol", "l2")},
           "gpu_launches": launches, "clocks": clk, "roofline": roof,
           "step": {"entries_per_step": entries / args.steps,
                    "build_factor_s_leaf_level": ms_region / args.steps / 1e3,
                    "ms_entries": ms_kern / args.steps,
                    "ms_id": sum(s["ms_id"] for s in stats) / args.steps,
                    "ms_factor": sum(s["ms_factor"] for s in stats) / args.steps,
                    "leaf_rank_max": s0["rank_per_level"][-1] if s0["rank_per_level"] else None}}
    out["e2e"] = run_e2e(args, curve, cfg, dev, params)
    if ws == 1:
        out["cpu_baseline"] = run_cpu_baseline(curve, cfg, budget_s=12.0)
    if not args.no_extras:
        out["extras"] = run_extras(curve, cfg, dev, params)
    return out


def run_e2e(args, curve, cfg, dev, params):
    """Same metric through the C ABI with the curve in pinned host memory: every step copies
    the geometry host -> device, builds, and reads the counters back."""
    import torch
    from paper_2607_00790_gb300 import binding

    host = {k: torch.as_tensor(curve[k], dtype=torch.float64).pin_memory()
            for k in ("x", "y", "nx", "ny", "w", "kappa")}
    devt = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    g = binding.Geom(curve["x"].size, *[devt[k].data_ptr() for k in ("x", "y", "nx", "ny", "w", "kappa")])
    p = params()
    steps = max(1, min(args.steps, 3))
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    entries = 0
    e0.record(stream)
    for _ in range(steps):
        for k in host:
            devt[k].copy_(host[k], non_blocking=True)
        s = binding.Solver(g, p, device=dev)
        s.factor()
        entries += s.stats()["entries_generated"]
        s.close()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d = sum(v.numel() * 8 for v in host.values())
    return {"value": entries / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 0, "steps": steps,
            "note": "H2D of the curve from pinned memory, create, leaf-level build incl. ID and "
                    "factor; the factors stay resident in HBM, counters are host-side"}


# --------------------------------------------------------------------- CPU oracle ----
def oracle_sample(curve, cfg, budget_s):
    """The oracle computing the entries of whole leaf boxes of the same build (diagonal block,
    near blocks with both neighbours, proxy row and column blocks) until the budget is spent."""
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
    cut = cfg["tol"] / 4.0
    while True:
        b = int(rng.integers(0, nb))
        lo, hi = b * N // nb, (b + 1) * N // nb
        nodes = np.arange(lo, hi)
        unk = np.concatenate([nodes, nodes + N])
        cx, cy, rho = oracle.proxy_circle(curve, nodes)
        P = int(np.ceil(2 * (ph.k1 * rho + np.log(1 / cut) / np.log(1.5))))
        P = max(P, cfg["nproxy"])
        P = (P + 7) // 8 * 8
        D = oracle.wsbm_entries(curve, ph, unk, unk)
        entries += D.size
        for s in ((b + 1) % nb, (b - 1) % nb):
            sl, sh = s * N // nb, (s + 1) * N // nb
            su = np.concatenate([np.arange(sl, sh), np.arange(sl, sh) + N])
            entries += oracle.wsbm_entries(curve, ph, unk, su).size
            entries += oracle.wsbm_entries(curve, ph, su, unk).size
        entries += oracle.proxy_row_block(curve, ph, unk, (cx, cy, rho), P).size
        entries += oracle.proxy_col_block(curve, ph, unk, (cx, cy, rho), P).size
        boxes += 1
        if time.time() - t0 >= budget_s:
            break
    el = time.time() - t0
    return entries, el, boxes


def cores():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count()


def run_cpu_baseline(curve, cfg, budget_s):
    entries, el, boxes = oracle_sample(curve, cfg, budget_s)
    return {"value": entries / el, "unit": UNIT, "cores": cores(), "kind": "oracle",
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
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores(), "kind": "oracle",
                             "sample": f"one random leaf box of the build per step ({tot_b} boxes)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------------- extras ----
def run_extras(curve, cfg, dev, params):
    """Untimed-by-contract measurements: mixed path, full HSS where the root fits."""
    import torch
    from paper_2607_00790_gb300 import binding, inputs

    out = {}
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
    for name, prec in (("fp64", binding.WSBM_FP64), ("mixed", binding.WSBM_MIXED)):
        build(g, params(prec, 1e-6))
        s, st = build(g, params(prec, 1e-6))
        res[name] = {"entries_per_s": st["entries_generated"] / (st["ms_entries"] * 1e-3),
                     "proxy_entries_per_s": st["entries_proxy"] / (st["ms_proxy"] * 1e-3),
                     "build_factor_s": st["ms_total_factor"] / 1e3}
        s.close()
    res["proxy_kernel_speedup"] = res["mixed"]["proxy_entries_per_s"] / res["fp64"]["proxy_entries_per_s"]
    out["mixed_vs_fp64_2p18_leaf_level_tol1e-6"] = res

    # full HSS on the 16384-node star (the largest 15 nodes/wavelength case whose root fits):
    # FP64 and mixed, far field of the mixed path against the FP64 path
    c16 = inputs.star(16384)
    g16, k16 = binding.make_geom(c16, device=dev)
    ang = torch.tensor(2 * np.pi * np.arange(8) / 8, device=dev)
    obs = torch.tensor(2 * np.pi * np.arange(360) / 360, device=dev)
    ffs = {}
    for name, prec, tol in (("fp64_tol1e-8", binding.WSBM_FP64, 1e-8), ("fp64_tol1e-6", binding.WSBM_FP64, 1e-6),
                            ("mixed_tol1e-6", binding.WSBM_MIXED, 1e-6)):
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
    for name in ("fp64_tol1e-6", "mixed_tol1e-6"):
        out[f"star16384_full_{name}"]["farfield_rel_err_vs_fp64_tol1e-8"] = float(
            np.linalg.norm(ffs[name] - ref) / np.linalg.norm(ref))

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
    s.close()
    return out


def profile_case():
    import torch
    from paper_2607_00790_gb300 import binding, inputs
    c = inputs.star(16384)
    g, keep = binding.make_geom(c)
    for prec in (binding.WSBM_FP64, binding.WSBM_MIXED):
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
    ap.add_argument("--profile-case", action="store_true",
                    help="one leaf-level build of the 16384-node star (small case for ncu)")
    args = ap.parse_args()
    if args.profile_case:
        profile_case()
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
