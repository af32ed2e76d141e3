#!/usr/bin/env python3
"""Benchmark: time to solution of mixed-precision iterative refinement on GB300.

Workload (one system per step, inputs resident in HBM): the Green's-function
system of the paper's Sec. 2 at N = 4096, A = I - 800 G (midpoint rule),
x_true = sin(pi x), b = A x_true; TW = binary64, TF = binary32 (tensor-core
TF32 trailing update reported beside it), TR = binary64.  A step is the whole
hot path: rounded copy of A, blocked LU with partial pivoting, and the
refinement loop (correction solves, x += d, binary64 residual) until the
termination rule of Sec. 5.1 holds.

Metric: milliseconds per solved system (lower is better).  With N GPUs
(torchrun, one process per GPU) every rank solves its own copy of the system
("replicas only": one system does not shard); the value is the slowest
rank's step time divided by the number of systems solved per step.

Besides the headline it reports: the plain binary64 LU solve (cuSOLVER via
torch.linalg) on the same system, the LU rate in TFLOP/s, a roofline line for
the kernel that takes the most time, an end-to-end number through the
host-buffer entry point, and the CPU oracle timed on the host cores.

The batched workload (2000 systems, N uniform in [32, 512], A = I - alpha G
+ 1e-3 E with alpha uniform in [1, 800], b = 1; TW = binary64, TF = binary16
scaled and bfloat16, one persistent launch per batch) is reported in the same
line under "batched": solves per second, accuracy against binary64 LU
solutions, and the binary64 LU solve of the same systems (cuSOLVER through
torch.linalg, systems of equal N stacked) for comparison.

`--impl reference` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 4096
ALPHA = 800.0
L2_FLUSH_BYTES = 512 * 1024 * 1024

# Algorithmic work per launcher call (for the roofline line).
#   panel:     the N x nb rank-1 updates of a panel, 2 * sum_k (M - k)(nb - k) flops
#   gemm_*:    2 m^2 nb flops (trailing update of an m x m block, K = nb)
#   residual:  N^2 * sizeof(TW) bytes of A read once
#   trsv_pair: N^2 * 4 bytes of factors read once (L and U)


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the binary64 cuSOLVER comparators (e.g. under a profiler)")
    ap.add_argument("--batch-count", type=int, default=2000)
    ap.add_argument("--no-gmres", action="store_true", help="skip the GMRES-IR / BiCGSTAB-IR lines")
    return ap.parse_args()


# DRAM bytes (read + written) of one k_panel launch from the ncu capture summarised
# in profiles/k_panel_green_N4096.md (the 21st panel of N = 4096: 2816 rows), and
# the SHA-256 of the kernel source it was taken on; the traffic is reported only
# while the source is unchanged, scaled to the average launch by its rows (the
# panel reads each of its rows once).
PANEL_TRAFFIC = {"sha256": "a99d0a37d965bbb824be2b60acf53b80c644ea8400fed5db6cf1279e84823ee6",
                 "bytes": 755968.0, "rows": 2816}


def panel_traffic_per_launch(n, nb=64):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2311_14616_gb300", "csrc", "k_panel.cu")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != PANEL_TRAFFIC["sha256"]:
        return None
    rows = [n - j for j in range(0, n, nb)]
    return PANEL_TRAFFIC["bytes"] * (sum(rows) / len(rows)) / PANEL_TRAFFIC["rows"]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained"), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    """One process per GPU (torchrun env): NCCL on the GPU machine. The replicas
    exchange nothing but the barrier and the max of the step times; without a
    GPU (the host-side tests) the same calls run over gloo."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(n):
    import irgen
    A, b, xt = irgen.case_green_sine(n, ALPHA)
    return A, b, xt


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def oracle_sample_time(n_full, sample_n):
    """Oracle IR (binary32 factorization, binary64 residual) on the host cores for
    the same workload at N = sample_n; time scaled by (n_full / sample_n)^3 (the
    LU's N^3 term dominates)."""
    import oracle as O
    A, b, _ = make_inputs(sample_n)
    t0 = time.perf_counter()
    res = O.ir_solve(A, b, O.F32, nb=64)
    dt = time.perf_counter() - t0
    scale = (n_full / sample_n) ** 3
    return dt * scale * 1e3, res, dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = cpu_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    sample_n = min(args.n, 2048)
    times = []
    for i in range(args.warmup + args.steps):
        ms, _, _ = oracle_sample_time(args.n, sample_n)
        if i >= args.warmup:
            times.append(ms)
    v = statistics.mean(times)
    sample = (f"oracle IR (binary32 LU, binary64 residual) at N={sample_n} of the same workload, "
              f"time x (N/{sample_n})^3")
    out = {
        "impl": "reference", "metric": "ir_solve_ms", "value": v, "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": f"green_sine_N{args.n}_alpha800_TWf64_TFf32_TRf64", "n": args.n,
                   "alpha": ALPHA},
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------

BATCH_SEED = 1005


def run_batched(args, ctx, dev, stream, flush, ws, rank):
    """2000 uneven systems per step, one persistent launch (ir_batch_run)."""
    import numpy as np
    import torch

    import irgen
    from paper_2311_14616_gb300 import ir

    count = args.batch_count
    ns, alphas, As, bs = irgen.case_batch(count, BATCH_SEED)
    Ad = [torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t() for A in As]
    bd = [torch.from_numpy(b).to(dev) for b in bs]
    flops = float(sum(2.0 * int(n) ** 3 / 3.0 for n in ns))
    # binary64 LU solves of the same systems (cuSOLVER via torch.linalg), equal sizes stacked
    groups = {}
    for i, n in enumerate(ns):
        groups.setdefault(int(n), []).append(i)
    stacks = [(idx, torch.stack([torch.from_numpy(As[i]).to(dev) for i in idx]),
               torch.stack([bd[i] for i in idx]).unsqueeze(2)) for idx in groups.values()]

    def fp64_step():
        return [torch.linalg.lu_solve(*torch.linalg.lu_factor(S), B) for _, S, B in stacks]

    # the same systems padded to one [count, nmax, nmax] batch (identity on the padding)
    nmax = int(max(ns))

    def fp64_padded():
        P = torch.zeros(count, nmax, nmax, dtype=torch.float64, device=dev)
        Pb = torch.zeros(count, nmax, 1, dtype=torch.float64, device=dev)
        for i, n in enumerate(ns):
            n = int(n)
            P[i, :n, :n] = Ad[i]
            P[i, n:, n:] = torch.eye(nmax - n, dtype=torch.float64, device=dev)
            Pb[i, :n, 0] = bd[i]
        return P, Pb

    def fp64_padded_step():
        return torch.linalg.lu_solve(*torch.linalg.lu_factor(P), Pb)

    def time_ref(fn):
        for _ in range(2):
            r = fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(max(2, args.steps // 2)):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.mean(t), r

    if args.no_fp64:
        t_grouped = t_padded = float("nan")
        xref = [np.linalg.solve(A, b) for A, b in zip(As, bs)]
    else:
        t_grouped, x64 = time_ref(fp64_step)
        P, Pb = fp64_padded()
        t_padded, _ = time_ref(fp64_padded_step)
        del P, Pb
        xref = [None] * count
        for (idx, _, _), X in zip(stacks, x64):
            for k, i in enumerate(idx):
                xref[i] = X[k, :, 0].cpu().numpy()
    t64 = min(t_grouped, t_padded)
    # binary64 floor: the batch's LU flops at the rate of a large binary64 GEMM on this GPU
    G = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(G, G)
    torch.cuda.synchronize()
    t_g = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(G, G)
        e1.record(stream)
        torch.cuda.synchronize()
        t_g.append(e0.elapsed_time(e1))
    del G
    dgemm_tflops = 2 * 4096 ** 3 / (min(t_g) * 1e-3) / 1e12
    floor64 = flops / (dgemm_tflops * 1e12) * 1e3
    out = {"workload": f"batch_{count}_N32-512_green_alpha1-800_E1e-3_TWf64", "count": count,
           "seed": BATCH_SEED, "fp64_lu_solve_ms": t64,
           "fp64_lu_solve": "binary64 LU solve with torch.linalg.lu_factor + lu_solve (cuSOLVER): the "
                            "faster of one batch padded to N=512 with identity blocks "
                            f"({t_padded:.1f} ms) and systems of equal N stacked ({t_grouped:.1f} ms)",
           "lu_flops_per_batch": flops, "fp64_gemm_tflops": dgemm_tflops,
           "fp64_lu_floor_ms": floor64,
           "fp64_lu_floor": "the batch's 2N^3/3 LU flops at the measured binary64 GEMM rate "
                            "(torch.matmul 4096^3): no binary64 LU of these systems can be faster"}
    for tf in ("f16", "bf16"):
        plan = ctx.batch(Ad, bd, tf=tf, autotune=True)      # the plan times its schedule candidates
        for _ in range(max(3, args.warmup)):
            plan.run()
        torch.cuda.synchronize()
        barrier(ws)
        ms = []
        l0 = ir.kernel_launches()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        launches = ir.kernel_launches() - l0
        t = max_over_ranks(statistics.mean(ms), ws)
        res = plan.results()
        errs = np.array([np.max(np.abs(x.cpu().numpy() - xr)) / np.max(np.abs(xr))
                         for x, xr in zip(plan.xs, xref)])
        st = {}
        for r in res:
            st[r["status"]] = st.get(r["status"], 0) + 1
        grid, tcm = plan.schedule()
        out[tf] = {"ms": t, "solves_per_s": ws * count / (t * 1e-3), "speedup_vs_fp64_lu": t64 / t,
                   "schedule": {"grid": grid, "tc_min_trail": tcm, "autotuned": True},
                   "speedup_vs_fp64_floor": floor64 / t,
                   "gpu_launches_per_step": launches / args.steps,
                   "status": st, "mean_iters": float(np.mean([r["iters"] for r in res])),
                   "rel_err_vs_fp64_lu": {"median": float(np.median(errs)), "max": float(np.max(errs)),
                                          "frac_le_1e-12": float(np.mean(errs <= 1e-12))}}
        if tf == "f16":
            # precision escalation: members that stop above 1e-10 ||b|| are solved again
            # with binary32 factors in a second device pass (ir_batch_run_escalate)
            ms_e = []
            for _ in range(2):
                plan.run_escalate("f32", 1e-10)
            torch.cuda.synchronize()
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.run_escalate("f32", 1e-10)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_e.append(e0.elapsed_time(e1))
            te = max_over_ranks(statistics.mean(ms_e), ws)
            res_e = plan.results()
            errs_e = np.array([np.max(np.abs(x.cpu().numpy() - xr)) / np.max(np.abs(xr))
                               for x, xr in zip(plan.xs, xref)])
            out[tf]["escalated_to_f32"] = {
                "ms": te, "solves_per_s": ws * count / (te * 1e-3), "rtol": 1e-10,
                "members_escalated": int(sum(1 for r in res_e if r["tf"] == ir.F32)),
                "rel_err_vs_fp64_lu": {"median": float(np.median(errs_e)), "max": float(np.max(errs_e)),
                                       "frac_le_1e-12": float(np.mean(errs_e <= 1e-12))}}
        plan.destroy()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle as O
        sample = list(range(0, count, max(1, count // 20)))[:20]
        t0 = time.perf_counter()
        for i in sample:
            O.ir_solve(As[i], bs[i], O.F16, nb=64)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(sample) / dt, "unit": "solves/s", "cores": cpu_cores(),
                               "kind": "oracle",
                               "sample": f"oracle IR (binary16 factors) on {len(sample)} of the systems "
                                         f"({dt:.2f} s)"}
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_setup(args)
    import numpy as np
    import torch

    from paper_2311_14616_gb300 import ir

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    A, b, xt = make_inputs(n)
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()        # column-major
    b_d = torch.from_numpy(b).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = ir.Context(local)
    stream = torch.cuda.current_stream(dev)

    def timed_steps(step_fn, steps, warmup, profile=False):
        for _ in range(warmup):
            step_fn()
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        launches0 = ir.kernel_launches()
        if profile:
            ir.profile_start()
        out = None
        for e0, e1 in ev:
            flush.fill_(1.0)                    # evict A from L2 between steps
            e0.record(stream)
            out = step_fn()
            e1.record(stream)
        torch.cuda.synchronize()
        prof = ir.profile_stop() if profile else None
        launches = ir.kernel_launches() - launches0
        barrier(ws)
        ms = [a.elapsed_time(z) for a, z in ev]
        return ms, out, prof, launches

    # --- headline: TF = binary32 (bit-exact FP32 LU), default termination
    fact32 = ctx.factor(A_d, tf="f32", autotune=True)     # schedule timed on this A before the run
    x32 = torch.empty_like(b_d)
    term = ir.default_term()

    def step32():
        fact32.refactor(A_d)
        return fact32.solve(b_d, x32, term)[1]

    clocks = ClockSampler(local)
    clocks.start()
    ms32, rep32, prof32, _ = timed_steps(step32, args.steps, args.warmup, profile=True)
    # unprofiled repeat: the headline number carries no event overhead (and runs the
    # lookahead schedule, which per-launcher profiling turns off); its launches are
    # the ones reported
    ms32_plain, rep32, _, launches = timed_steps(step32, args.steps, 1)
    clk = clocks.stop()
    t32 = max_over_ranks(statistics.mean(ms32_plain), ws)

    # --- tensor-core arm: TF = TF32, litmax raised so IR reaches its limiting accuracy
    fact_tc = ctx.factor(A_d, tf="tf32", autotune=True)
    xtc = torch.empty_like(b_d)
    term_tc = ir.default_term(litmax=30)

    def step_tc():
        fact_tc.refactor(A_d)
        return fact_tc.solve(b_d, xtc, term_tc)[1]

    ms_tc, rep_tc, prof_tc, _ = timed_steps(step_tc, max(3, args.steps // 2), 1, profile=True)
    t_tc = max_over_ranks(statistics.mean(ms_tc), ws)

    # --- binary64 LU solve (cuSOLVER through torch.linalg) on the same system
    A_row = torch.from_numpy(np.ascontiguousarray(A)).to(dev)

    def step64():
        LU, piv = torch.linalg.lu_factor(A_row)
        return torch.linalg.lu_solve(LU, piv, b_d.unsqueeze(1))

    if args.no_fp64:
        t64, x64 = None, None
    else:
        ms64, x64, _, _ = timed_steps(step64, max(3, args.steps // 2), 1)
        t64 = max_over_ranks(statistics.mean(ms64), ws)

    # --- accuracy against the closed form and the binary64 LU solution
    xg = x32.double().cpu().numpy()
    err_true = float(np.max(np.abs(xg - xt)) / np.max(np.abs(xt)))
    err_vs_lu64 = None
    if x64 is not None:
        x64h = x64.squeeze(1).cpu().numpy()
        err_vs_lu64 = float(np.max(np.abs(xg - x64h)) / np.max(np.abs(x64h)))
    err_tc_true = float(np.max(np.abs(xtc.double().cpu().numpy() - xt)) / np.max(np.abs(xt)))

    # --- roofline of the kernel kind with the largest share of the profiled step
    peaks = load_peaks()
    total_prof = sum(v[0] for v in prof32.values())
    dom = max(prof32, key=lambda k: prof32[k][0])
    nb = 64
    dom_ms, dom_calls = prof32[dom]
    avg_ms = dom_ms / dom_calls
    sm_mhz = clk.get("sm_mhz") or 2070.0
    fp32_peak_tflops = 152 * 128 * 2 * 2070e6 / 1e12   # SMs x FP32 lanes x FMA x max clock
    if dom == "panel":
        flops = sum(2 * sum((n - j - k) * (min(nb, n - j) - k) for k in range(min(nb, n - j)))
                    for j in range(0, n, nb)) / dom_calls
        roof = {"bound": "alu", "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "kernel": "k_panel"}
    elif dom in ("gemm_simt", "gemm_tc"):
        flops = sum(2 * (n - j - nb) ** 2 * nb for j in range(0, n - nb, nb)) / dom_calls
        peak = fp32_peak_tflops if dom == "gemm_simt" else peaks["bf16_tflops"] * 1.1 / 2.25
        roof = {"bound": "alu" if dom == "gemm_simt" else "tensor",
                "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "kernel": "k_" + dom}
    elif dom == "residual":
        roof = {"bound": "hbm", "achieved": n * n * 8 / (avg_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "kernel": "k_resid_partial+k_resid_final"}
    else:
        roof = {"bound": "hbm", "achieved": n * n * 4 / (avg_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "kernel": "k_" + dom}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = panel_traffic_per_launch(n) if dom == "panel" else None   # bytes per launch
    roof["peak_source"] = peaks["source"] if roof["bound"] != "alu" else "unit counts x 2070 MHz"
    roof["share_of_step"] = dom_ms / total_prof
    roof["avg_launch_ms"] = avg_ms

    # --- a roofline line for every kernel kind of the step (the dominant one is the latency-bound panel)
    def dgemm_rate():
        G = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        torch.matmul(G, G)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.matmul(G, G)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ = e0.elapsed_time(e1)
            best = t_ if best is None else min(best, t_)
        return 2 * 4096 ** 3 / (best * 1e-3) / 1e12

    fp64_tflops = dgemm_rate()
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25
    n_iter = rep32.iters
    kr = {}

    def line(kind, prof, steps, bound, work, peak, unit, note):
        if kind not in prof:
            return
        ms_, calls = prof[kind]
        rate = work / (ms_ / steps * 1e-3) / (1e12 if unit == "TFLOP/s" else 1e9)
        kr[kind] = {"bound": bound, "achieved": rate, "peak": peak, "unit": unit, "frac": rate / peak,
                    "ms_per_step": ms_ / steps, "calls_per_step": calls / steps, "work": note}

    gemm_flops = sum(2 * (n - j - nb) ** 2 * nb for j in range(0, n - nb, nb))
    line("gemm_simt", prof32, args.steps, "alu", gemm_flops, fp32_peak_tflops, "TFLOP/s",
         "2 m^2 nb flops per block step, binary32 FMA pipe (unit counts x 2070 MHz)")
    tc_steps = max(3, args.steps // 2)
    line("gemm_tc", prof_tc, tc_steps, "tensor", gemm_flops, tf32_peak, "TFLOP/s",
         "2 m^2 nb flops per block step, TF32 peak = measured bf16 x 1.1/2.25")
    line("residual", prof32, args.steps, "alu", 2.0 * n * n * n_iter, fp64_tflops, "TFLOP/s",
         "2 N^2 flops per residual on the binary64 pipe; peak = measured binary64 GEMM rate")
    line("trsv_pair", prof32, args.steps, "hbm", 4.0 * n * n * n_iter, peaks["hbm_gbs"], "GB/s",
         "N^2 x 4 B of factors (L and U) per correction solve")
    line("cast", prof32, args.steps, "hbm", 12.0 * n * n, peaks["hbm_gbs"], "GB/s",
         "N^2 x (8 B read + 4 B written)")

    # --- LU rate of the headline path (2 N^3 / 3 flops over factor time = cast + LU kernels)
    lu_kinds = ("cast", "iota", "panel", "laswp", "trsm", "gemm_simt", "diag_inv")
    lu_ms = sum(prof32[k][0] for k in lu_kinds if k in prof32) / args.steps
    lu_tflops = (2.0 * n ** 3 / 3.0) / (lu_ms * 1e-3) / 1e12
    lu_tc_ms = sum(prof_tc[k][0] for k in ("cast", "iota", "panel", "laswp", "trsm", "gemm_tc", "diag_inv")
                   if k in prof_tc) / max(3, args.steps // 2)

    # --- end to end through the host-buffer entry point (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        A_h = torch.from_numpy(np.ascontiguousarray(A.T)).t().pin_memory()
        b_h = torch.from_numpy(b).pin_memory()
        for _ in range(2):
            ctx.solve_host(A_h, b_h, tf="f32")
        torch.cuda.synchronize()
        barrier(ws)
        t_e = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.solve_host(A_h, b_h, tf="f32")
            t_e.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": max_over_ranks(statistics.mean(t_e), ws) / ws, "unit": "ms",
               "h2d_bytes_per_step": int(n * n * 8 + n * 8), "d2h_bytes_per_step": int(n * 8),
               "api": "ir_solve_host (pinned host A, b: copies in, factor, refine, copy back; the context keeps "
                      "its device buffers and factorization across calls of the same shape)"}

    # --- CPU oracle on the host cores (rank 0, one GPU only)
    cpu = None
    acc_oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        sample_n = min(n, 2048)
        ms_cpu, res, dt = oracle_sample_time(n, sample_n)
        cpu = {"value": ms_cpu, "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": f"one oracle IR solve of the same workload at N={sample_n} "
                         f"({dt:.2f} s), scaled by (N/{sample_n})^3"}

    batched = None if args.no_batch else run_batched(args, ctx, dev, stream, flush, ws, rank)

    # --- GMRES-IR (Sec. 4.3) with binary16 factors on the same system, where plain IR
    # with the same factors does not converge
    gmres = None
    if not args.no_gmres:
        fact16 = ctx.factor(A_d, tf="f16")
        fact16.gmres_reserve(10)
        xg16 = torch.empty_like(b_d)
        x16 = torch.empty_like(b_d)
        kopts = ir.krylov_opts()

        def step_gm():
            fact16.refactor(A_d)
            return fact16.solve_gmres(b_d, xg16, term, kopts)[1]

        gsteps = max(3, args.steps // 2)
        _, _, prof_gm, l_gm = timed_steps(step_gm, gsteps, 1, profile=True)
        ms_gm, rep_gm, _, _ = timed_steps(step_gm, gsteps, 1)
        _, rep_ir16 = fact16.solve(b_d, x16, term)
        rel = lambda v: float(np.max(np.abs(v.double().cpu().numpy() - xt)) / np.max(np.abs(xt)))
        gm_kinds = {k: v[0] / gsteps for k, v in sorted(prof_gm.items())}

        # BiCGSTAB-IR (Sec. 2.3, 4.2) on the same factors and system
        fact16.bicgstab_reserve()
        xb16 = torch.empty_like(b_d)

        def step_bi():
            fact16.refactor(A_d)
            return fact16.solve_bicgstab(b_d, xb16, term, kopts)[1]

        _, _, prof_bi, l_bi = timed_steps(step_bi, gsteps, 1, profile=True)
        ms_bi, rep_bi, _, _ = timed_steps(step_bi, gsteps, 1)
        bicgstab = {
            "ms": max_over_ranks(statistics.mean(ms_bi), ws), "unit": "ms (refactor + BiCGSTAB-IR solve)",
            "iters": rep_bi.iters, "status": rep_bi.status, "khist": rep_bi.khist,
            "rel_err_vs_closed_form": rel(xb16),
            "kernel_ms_per_step": {k: v[0] / gsteps for k, v in sorted(prof_bi.items())},
            "gpu_launches_per_step": l_bi / gsteps,
        }
        gmres = {
            "workload": f"green_sine_N{n}_alpha800_TWf64_TFf16_TRf64_basis10",
            "ms": max_over_ranks(statistics.mean(ms_gm), ws), "unit": "ms (refactor + GMRES-IR solve)",
            "iters": rep_gm.iters, "status": rep_gm.status, "khist": rep_gm.khist,
            "rhist": rep_gm.rhist, "rel_err_vs_closed_form": rel(xg16),
            "ir_same_factors": {"iters": rep_ir16.iters, "status": rep_ir16.status,
                                "rel_err_vs_closed_form": rel(x16)},
            "kernel_ms_per_step": gm_kinds,
            "gpu_launches_per_step": l_gm / gsteps,
            "bicgstab_ir": bicgstab,
        }

    value = t32 / ws if ws > 1 else t32
    out = {
        "metric": "ir_solve_ms", "value": value, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t32, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": f"green_sine_N{n}_alpha800_TWf64_TFf32_TRf64", "n": n, "alpha": ALPHA,
                   "TW": "f64", "TF": "f32", "TR": "f64", "rhs": "b = A sin(pi x)",
                   "l2": "flushed by a 512 MiB write before every timed step",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "schedule": {"nb": fact32.schedule()[0], "panel_reserve_sms": fact32.schedule()[1],
                                "autotuned": True}},
        "iters": rep32.iters, "status": rep32.status,
        "rel_err_vs_closed_form": err_true, "rel_err_vs_fp64_lu": err_vs_lu64,
        "fp64_lu_solve_ms": t64, "speedup_vs_fp64_lu": (t64 / t32) if t64 else None,
        "lu_ms": lu_ms, "lu_tflops": lu_tflops,
        "tf32_tensor_core": {"ms": t_tc, "iters": rep_tc.iters, "status": rep_tc.status,
                             "lu_ms": lu_tc_ms, "rel_err_vs_closed_form": err_tc_true,
                             "litmax": 30,
                             "kernel_ms_per_step": {k: v[0] / max(3, args.steps // 2)
                                                    for k, v in sorted(prof_tc.items())}},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof32.items())},
        "roofline": roof,
        "kernel_rooflines": kr,
        "fp64_gemm_tflops": fp64_tflops,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps,
        "clocks": clk,
        "batched": batched,
        "gmres_ir": gmres,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
