#!/usr/bin/env python3
"""Benchmark: time to solution of mixed-precision iterative refinement on GB300.

Headline workload (one system per step, inputs resident in HBM): N = 8192,
A = N(0,1) entries + 2 sqrt(N) I (seed 1002), b ~ N(0,1); TW = binary64,
TF = binary16 with A scaled by s = 2^10 / max|a_ij| before the cast (binary32
accumulation on the tensor cores), TR = binary64.  A step is the whole hot
path: rounded copy of A, blocked LU with partial pivoting, and the refinement
loop (correction solves, x += d, binary64 residual) until the termination
rule of Sec. 5.1 holds.

Metric: milliseconds per solved system (lower is better).  With N GPUs
(torchrun, one process per GPU) every rank solves its own copy of the system
("replicas only": one system does not shard); the value is the slowest
rank's step time divided by the number of systems solved per step.

Beside the headline the line reports: the same system with bfloat16 factors;
the plain binary64 LU solve (cuSOLVER via torch.linalg) and the binary32
cuSOLVER LU solve on the same system; the LU rate in TFLOP/s; the roofline of
the tensor-core trailing update against the dtype's measured tensor peak; the
panel's share of the factorization; accuracy against the oracle's binary64
solution x_ref and the oracle's own refinement; an end-to-end number through
the host-buffer entry point; the CPU oracle timed on the host cores; and
lines for the other workloads:
  * N = 256 Green's system I - G (b = 1, ||r|| <= 1e-13 ||b||), binary32
    factors, in microseconds (launch and latency bound);
  * N = 4096 Green's system I - 800 G, x_true = sin(pi x), binary32 factors
    (SIMT update, bitwise the unblocked LU) and TF32 tensor-core factors;
  * N = 8192 A = U diag(s) V^T, s geometric from 1 to 1e-6, TW = TF = binary32,
    TR = binary64 (the promoted problem);
  * the batch of 2000 systems, N uniform in [32, 512], A = I - alpha G
    + 1e-3 E (alpha uniform in [1, 800]), b = 1, binary16 (scaled) and
    bfloat16 factors, one persistent launch per batch;
  * GMRES-IR and BiCGSTAB-IR with binary16 factors on the N = 4096 Green's
    system, where plain IR with the same factors does not converge.

`--impl reference` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 8192
SEED_GAUSS = 1002          # seed of the headline system
SEED_SVD = 1003
ALPHA = 800.0
NB = 64
L2_FLUSH_BYTES = 512 * 1024 * 1024
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--order", dest="n", type=int, default=N_DEFAULT, help="order N of the headline system")
    ap.add_argument("--group", type=int, default=0,
                    help="fixed group size of the tensor-core LU for the headline (0: autotuned schedule)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the cuSOLVER comparators (e.g. under a profiler)")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle's reference solutions (accuracy fields become null)")
    ap.add_argument("--no-extra", action="store_true", help="skip the N = 256 / 4096 / kappa = 1e6 lines")
    ap.add_argument("--batch-count", type=int, default=2000)
    ap.add_argument("--no-gmres", action="store_true", help="skip the GMRES-IR / BiCGSTAB-IR lines")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the headline system's variants (mixed precision solves, 2-byte factors, 4 right-hand sides)")
    return ap.parse_args()


# Algorithmic work per unit (the roofline's numerators):
#   trailing update:  2 m^2 nb flops per block step (m = trailing order, K = nb),
#                     summed over the factorization: ~2 N^3 / 3
#   panel:            2 sum_k (M - k)(nb - k) flops per panel (latency bound: reported
#                     as a share of the factorization, not as a roofline)
#   residual:         N^2 sizeof(TW) bytes of A (and 2 N^2 binary64 flops)
#   correction solve: N^2 x 4 bytes of binary32 factors (L and U)
#   cast:             N^2 (sizeof(TW) + 4) bytes

def trailing_update_flops(n, nb=NB):
    return float(sum(2.0 * (n - j - nb) ** 2 * nb for j in range(0, n - nb, nb)))


def group_update_flops(n, group, nb=NB):
    """Flops of the tensor-core factorization's group updates (k_gemm_tc with all
    of a group's slots): for every group of `group` block steps with far columns,
    the rows below the group times the far columns times K = nb * group."""
    W, f = nb * group, 0.0
    for c0 in range(0, n, W):
        c1 = min(c0 + W, n)
        near_end = min(c1 + nb, n)
        if near_end < n:
            f += 2.0 * (n - c1) * (n - near_end) * (c1 - c0)
    return f


def lu_flops(n):
    return 2.0 * n ** 3 / 3.0


def traffic_per_launch(kernel):
    """DRAM bytes (read + written) per launch of `kernel` from the committed ncu
    summary record, while the kernel's source is the one it was captured on."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if digest != rec.get("sha256"):
        return None
    return float(rec["bytes_per_launch"])


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


def headline_inputs(n):
    import irgen
    return irgen.case_gaussian(n, SEED_GAUSS)


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_solve_ms(A, b, tf):
    """One oracle IR solve (emulated-TF LU, binary32 solves, binary64 residual) on
    the host cores: (milliseconds, result)."""
    import oracle as O
    t0 = time.perf_counter()
    res = O.ir_solve(A, b, tf, nb=NB)
    return (time.perf_counter() - t0) * 1e3, res


def run_reference(args):
    """The oracle on the headline workload: every timed step is one complete
    oracle solve of the N x N system (no sampling, no scaling); the warm-up
    steps solve an N/8 instance of the same recipe (they only start the
    OpenMP pool and page the library in)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    cores = cpu_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    n = args.n
    A, b = headline_inputs(n)
    Aw, bw = headline_inputs(max(1, n // 8))
    for _ in range(args.warmup):
        oracle_solve_ms(Aw, bw, O.F16)
    times = [oracle_solve_ms(A, b, O.F16)[0] for _ in range(args.steps)]
    v = statistics.mean(times)
    sample = (f"one complete oracle IR solve of the N={n} system per timed step (binary16 factors emulated: "
              f"binary32 panel and U12, TF-rounded update operands, exact products summed in binary64; "
              f"binary32 solves; binary64 residual); warm-up steps solve an N={max(1, n // 8)} instance")
    out = {
        "impl": "reference", "metric": "ir_solve_ms", "value": v, "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16/f32/f64", "data": "synthetic",
        "config": headline_config(n),
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def headline_config(n):
    return {"workload": f"gauss_shift_N{n}_seed{SEED_GAUSS}_TWf64_TFf16scaled_TRf64", "n": n,
            "A": "N(0,1) entries + 2 sqrt(N) I", "b": "N(0,1)", "TW": "f64", "TF": "f16 (s = 2^10/max|a|)",
            "TR": "f64", "l2": "flushed by a 512 MiB write before every timed step"}


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
    A, b = headline_inputs(n)
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()        # column-major
    b_d = torch.from_numpy(b).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = ir.Context(local)
    stream = torch.cuda.current_stream(dev)
    peaks = load_peaks()

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

    def rel(x, ref):
        if ref is None:
            return None
        x = x.double().cpu().numpy() if hasattr(x, "cpu") else np.asarray(x, dtype=np.float64)
        return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))

    oracle_ok = rank == 0 and ws == 1 and not args.no_oracle
    if oracle_ok:
        import oracle as O
        os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))

    # --- headline: TF = binary16 (scaled), tensor-core trailing update
    tune = args.group == 0
    fact = ctx.factor(A_d, tf="f16", autotune=tune, group=args.group)   # schedule timed on this A before the run
    sched16 = fact.schedule()
    x16 = torch.empty_like(b_d)
    term = ir.default_term()

    def step16():
        fact.refactor(A_d)
        return fact.solve(b_d, x16, term)[1]

    clocks = ClockSampler(local)
    clocks.start()
    ms16, rep16, _, launches = timed_steps(step16, args.steps, args.warmup)
    clk = clocks.stop()
    t16 = max_over_ranks(statistics.mean(ms16), ws)
    # the factorization alone (graph replay of the lookahead schedule)
    ms_fac, _, _, _ = timed_steps(lambda: fact.refactor(A_d), args.steps, 1)
    t_fac = max_over_ranks(statistics.mean(ms_fac), ws)
    # per-launcher CUDA events (kernels issued one after another, no lookahead):
    # the per-kernel breakdown and the roofline's launch times
    _, _, prof16, _ = timed_steps(step16, args.steps, 1, profile=True)
    kms = {k: v[0] / args.steps for k, v in sorted(prof16.items())}
    kcalls = {k: v[1] / args.steps for k, v in sorted(prof16.items())}
    x16h = x16.double().cpu().numpy()

    # --- the same system with bfloat16 factors (unscaled)
    factb = ctx.factor(A_d, tf="bf16", autotune=tune, group=args.group)
    xb = torch.empty_like(b_d)

    def stepb():
        factb.refactor(A_d)
        return factb.solve(b_d, xb, term)[1]

    msb, repb, _, _ = timed_steps(stepb, max(3, args.steps // 2), 1)
    tb = max_over_ranks(statistics.mean(msb), ws)
    factb.destroy()

    # --- cuSOLVER LU solves of the same system (torch.linalg): binary64, and binary32 as a yardstick
    A_row = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    t64 = t32 = t32f = None
    x64h = None
    if not args.no_fp64:
        def step64():
            LU, piv = torch.linalg.lu_factor(A_row)
            return torch.linalg.lu_solve(LU, piv, b_d.unsqueeze(1))
        ms64, x64, _, _ = timed_steps(step64, max(3, args.steps // 4), 1)
        t64 = max_over_ranks(statistics.mean(ms64), ws)
        x64h = x64.squeeze(1).cpu().numpy()
        A32 = A_row.float()
        b32 = b_d.float().unsqueeze(1)
        ms32, _, _, _ = timed_steps(lambda: torch.linalg.lu_solve(*torch.linalg.lu_factor(A32), b32),
                                    max(3, args.steps // 2), 1)
        t32 = max_over_ranks(statistics.mean(ms32), ws)
        ms32f, _, _, _ = timed_steps(lambda: torch.linalg.lu_factor(A32), max(3, args.steps // 2), 1)
        t32f = max_over_ranks(statistics.mean(ms32f), ws)
        del A32, b32

    # --- the oracle: x_ref (binary64 LU solve refined with extended residuals) and
    # its own binary16 refinement, timed on the host cores (the CPU baseline)
    xr = None
    cpu = None
    acc = {"rel_err_vs_x_ref": None, "rel_err_vs_oracle_ir": None, "rel_err_vs_fp64_lu": rel(x16h, x64h)}
    if oracle_ok:
        xr = O.reference_solution(A, b)
        kappa = float(np.linalg.cond(A, np.inf))
        bar = max(1e-12, 10.0 * kappa * 2.0 ** -52)
        if not args.no_cpu_baseline:
            ms_cpu, ores = oracle_solve_ms(A, b, O.F16)
            cpu = {"value": ms_cpu, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"one complete oracle IR solve of the same N={n} system (binary16 factors emulated; "
                             f"{ores.iters} iterations, status {O.STATUS_NAMES[ores.status]})"}
            acc["rel_err_vs_oracle_ir"] = rel(x16h, ores.x)
            acc["oracle_ir"] = {"iters": ores.iters, "status": O.STATUS_NAMES[ores.status],
                                "rel_err_vs_x_ref": rel(ores.x, xr)}
        e = rel(x16h, xr)
        acc.update({"rel_err_vs_x_ref": e, "kappa_inf": kappa, "parity_bar": bar,
                    "parity_bar_met": e <= bar, "literal_1e-12_met": e <= 1e-12,
                    "bf16_rel_err_vs_x_ref": rel(xb, xr)})

    # --- roofline: the tensor-core trailing update at the binary16 tensor peak
    roof = tensor_roofline(prof16, args.steps, n, peaks, sched16[2])

    # --- a line for every other kernel kind of the step
    fp64_tflops = dgemm_rate(torch, dev, stream)
    iters = rep16.iters
    kr = {}

    def line(kind, bound, work, peak, unit, note):
        if kind not in prof16:
            return
        ms_ = prof16[kind][0] / args.steps
        rate = work / (ms_ * 1e-3) / (1e12 if unit == "TFLOP/s" else 1e9)
        kr[kind] = {"bound": bound, "achieved": rate, "peak": peak, "unit": unit, "frac": rate / peak,
                    "ms_per_step": ms_, "calls_per_step": kcalls[kind], "work": note}

    gflops = group_update_flops(n, sched16[2]) if "gemm_tc_group" in prof16 else 0.0
    line("gemm_tc", "tensor", trailing_update_flops(n) - gflops, peaks["bf16_tflops"], "TFLOP/s",
         "single block steps (K = 64): the near columns and the group's own rows; 2 m_rows m_cols 64 flops each")
    line("residual", "alu", 2.0 * n * n * iters, fp64_tflops, "TFLOP/s",
         "2 N^2 flops per residual on the binary64 pipe; peak = measured binary64 GEMM rate")
    line("trsv_pair", "hbm", 4.0 * n * n * iters, peaks["hbm_gbs"], "GB/s",
         "N^2 x 4 B of binary32 factors (L and U) per correction solve")
    line("cast", "hbm", 12.0 * n * n, peaks["hbm_gbs"], "GB/s", "N^2 x (8 B read + 4 B written)")
    lu_kinds = ("maxabs", "cast", "iota", "panel", "laswp", "trsm", "gemm_tc", "diag_inv")
    lu_prof_ms = sum(kms.get(k, 0.0) for k in lu_kinds)
    panel_share = {"panel_ms_per_factorization": kms.get("panel"),
                   "share_of_factorization_serial": (kms.get("panel", 0.0) / lu_prof_ms) if lu_prof_ms else None,
                   "note": "latency bound (one cluster-wide pivot search per column); with lookahead the "
                           "trailing update runs beside it"}

    # --- end to end through the host-buffer entry point (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        A_h = torch.from_numpy(np.ascontiguousarray(A.T)).t().pin_memory()
        b_h = torch.from_numpy(b).pin_memory()
        for _ in range(2):
            ctx.solve_host(A_h, b_h, tf="f16")
        torch.cuda.synchronize()
        barrier(ws)
        t_e = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.solve_host(A_h, b_h, tf="f16")
            t_e.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": max_over_ranks(statistics.mean(t_e), ws) / ws, "unit": "ms",
               "h2d_bytes_per_step": int(n * n * 8 + n * 8), "d2h_bytes_per_step": int(n * 8),
               "api": "ir_solve_host (pinned host A, b: copies in, factor, refine, copy back; the context keeps "
                      "its device buffers and factorization across calls of the same shape)"}
        del A_h, b_h

    variants = None if args.no_variants else run_variants(args, ctx, A_d, b_d, timed_steps, rel, xr, x16h)
    fact.destroy()
    del A_row
    extra = None if args.no_extra else run_extra(args, ctx, dev, stream, flush, ws, rank, timed_steps, rel,
                                                 oracle_ok)
    batched = None if args.no_batch else run_batched(args, ctx, dev, stream, flush, ws, rank)
    gmres = None if args.no_gmres else run_krylov(args, ctx, dev, ws, timed_steps)

    value = t16 / ws if ws > 1 else t16
    cfg = headline_config(n)
    cfg.update({"parallelism": "replicas" if ws > 1 else "single",
                "schedule": {"nb": sched16[0], "panel_reserve_sms": sched16[1], "group": sched16[2],
                             "autotuned": tune}})
    out = {
        "metric": "ir_solve_ms", "value": value, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t16, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16/f32/f64", "data": "synthetic",
        "config": cfg,
        "iters": rep16.iters, "status": rep16.status, "rhist": rep16.rhist,
        "accuracy": acc,
        "fp64_lu_solve_ms": t64, "speedup_vs_fp64_lu": (t64 / t16) if t64 else None,
        "fp32_lu_solve_ms": t32, "fp32_lu_factor_ms": t32f,
        "lu_ms": t_fac, "lu_tflops": lu_flops(n) / (t_fac * 1e-3) / 1e12,
        "lu_tflops_note": "2 N^3 / 3 over the factorization (cast + LU + diagonal-block inverses, lookahead "
                          "schedule replayed from its graph)",
        "bf16": {"ms": tb, "iters": repb.iters, "status": repb.status},
        "variants": variants,
        "kernel_ms_per_step": kms,
        "roofline": roof,
        "panel": panel_share,
        "kernel_rooflines": kr,
        "fp64_gemm_tflops": fp64_tflops,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps,
        "clocks": clk,
        "workloads": extra,
        "batched": batched,
        "krylov_ir": gmres,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tensor_roofline(prof, steps, n, peaks, group):
    """The contract's roofline object for the tensor-core trailing update's group
    kernel (k_gemm_tc applying a group of block steps to the far trailing
    columns, the launches that carry most of the update's flops): their
    algorithmic flops over their summed launch time in one step (per-launcher
    CUDA events), against the measured dense bf16 tensor peak (binary16 has the
    same rate).  The single-step launches (K = 64) get their own line.
    prof: {kind: (total ms, calls)} over `steps` steps."""
    kind = "gemm_tc_group" if "gemm_tc_group" in prof else "gemm_tc"
    if kind not in prof:
        return None
    g_ms, g_calls = prof[kind][0] / steps, prof[kind][1] / steps
    flops = group_update_flops(n, group) if kind == "gemm_tc_group" else trailing_update_flops(n)
    achieved = flops / (g_ms * 1e-3) / 1e12
    peak = peaks["bf16_tflops"]
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic_per_launch("k_gemm_tc"),
            "kernel": f"k_gemm_tc ({kind}: binary16 operands, binary32 accumulators in TMEM)",
            "peak_source": f"{peaks['source']} bf16 dense burst (binary16 has the same tensor rate); "
                           "the kernel is timed alone (per-launcher events)",
            "work": "2 m_rows m_cols K flops per launch (K = 64 x group), summed over the factorization",
            "flops_per_step": flops, "flops_per_launch": flops / g_calls, "avg_launch_ms": g_ms / g_calls,
            "launches_per_step": g_calls, "ms_per_step": g_ms, "group": group}


def dgemm_rate(torch, dev, stream):
    """Measured binary64 GEMM rate (torch.matmul 4096^3, best of 3): the binary64 pipe's ceiling."""
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


def run_extra(args, ctx, dev, stream, flush, ws, rank, timed_steps, rel, oracle_ok):
    """The other single-system workloads: N = 256 (microseconds), N = 4096 Green's
    system (binary32 and TF32 factors), N = 8192 promoted problem (kappa = 1e6)."""
    import numpy as np
    import torch

    import irgen
    from paper_2311_14616_gb300 import ir
    steps = max(3, args.steps // 2)
    out = {}

    def one(A, b, tf, term, steps_):
        Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()
        bd = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
        f = ctx.factor(Ad, tf=tf, autotune=True)
        x = torch.empty_like(bd)

        def step():
            f.refactor(Ad)
            return f.solve(bd, x, term)[1]
        ms, rep, _, _ = timed_steps(step, steps_, 1)
        msf, _, _, _ = timed_steps(lambda: f.refactor(Ad), steps_, 1)
        f.destroy()
        return max_over_ranks(statistics.mean(ms), ws), max_over_ranks(statistics.mean(msf), ws), rep, x

    # N = 256, I - G, b = 1, ||r|| <= 1e-13 ||b||
    A1, b1 = irgen.case_green(256, 1.0)
    t1, tf1, rep1, x1 = one(A1, b1, "f32", ir.default_term(abs_rel_tol=1e-13), args.steps)
    out["green_N256_alpha1_TFf32"] = {
        "us": t1 * 1e3, "lu_us": tf1 * 1e3, "iters": rep1.iters, "status": rep1.status,
        "rel_err_vs_x_ref": rel(x1, O_ref(A1, b1)) if oracle_ok else None,
        "note": "L2-resident and launch/latency bound: absolute microseconds, no roofline fraction"}
    # N = 4096, I - 800 G, x_true = sin(pi x)
    A2, b2, xt2 = irgen.case_green_sine(4096, ALPHA)
    xr2 = O_ref(A2, b2) if oracle_ok else None
    for tf, litmax in (("f32", 10), ("tf32", 30)):
        t2, tf2, rep2, x2 = one(A2, b2, tf, ir.default_term(litmax=litmax), steps)
        e = rel(x2, xr2)
        out[f"green_sine_N4096_alpha800_TF{tf}"] = {
            "ms": t2, "lu_ms": tf2, "lu_tflops": lu_flops(4096) / (tf2 * 1e-3) / 1e12,
            "iters": rep2.iters, "status": rep2.status, "litmax": litmax,
            "rel_err_vs_closed_form": rel(x2, xt2), "rel_err_vs_x_ref": e,
            "literal_1e-12_met": (e <= 1e-12) if e is not None else None}
    # N = 8192, U diag(s) V^T, kappa = 1e6, TW = TF = binary32, TR = binary64
    A4, b4 = irgen.case_svd(8192, SEED_SVD)
    t4, tf4, rep4, x4 = one(A4, b4, "f32", ir.default_term(litmax=30), steps)
    d = {"ms": t4, "lu_ms": tf4, "iters": rep4.iters, "status": rep4.status, "litmax": 30,
         "TW": "f32", "TF": "f32", "TR": "f64"}
    if oracle_ok:
        xr4 = O_ref(A4, b4)
        k4 = float(np.linalg.cond(A4.astype(np.float64), np.inf))
        d.update({"rel_err_vs_promoted_x_ref": rel(x4, xr4), "kappa_inf": k4,
                  "bound_thm_irterm": 4 * (8192 + 1) * k4 * 2.0 ** -52 + 2.0 ** -23})
    out["svd_N8192_kappa1e6_TWf32_TFf32_TRf64"] = d
    return out


def run_variants(args, ctx, A_d, b_d, timed_steps, rel, xr, x16h):
    """The headline system with the paper's other solve arrangements: mixed
    precision solves (binary64 triangular solves on the promoted binary16
    factors, mplu(A; onthefly = true), Sec. 5.3), the factors kept in 2 bytes
    (Sec. 1, 2.5), and four right-hand sides refined together on one
    factorization (per column)."""
    import numpy as np
    import torch

    from paper_2311_14616_gb300 import ir
    out = {}
    steps = max(3, args.steps // 2)
    term = ir.default_term()
    for name, kw in (("mps_binary64_solves", dict(onthefly=True)), ("factors_in_2_bytes", dict(store_tf=True))):
        f = ctx.factor(A_d, tf="f16", autotune=True, **kw)
        x = torch.empty_like(b_d)

        def step():
            f.refactor(A_d)
            return f.solve(b_d, x, term)[1]
        ms, rep, prof, _ = timed_steps(step, steps, 1, profile=True)
        ms2, rep, _, _ = timed_steps(step, steps, 1)
        solve_kind = "trsv_pair_f64" if kw.get("onthefly") else "trsv_pair"
        out[name] = {"ms": max_over_ranks(statistics.mean(ms2), ws_of()), "iters": rep.iters, "status": rep.status,
                     "solve_ms_per_step": prof[solve_kind][0] / steps if solve_kind in prof else None,
                     "rel_err_vs_x_ref": rel(x, xr)}
        f.destroy()
    # four right-hand sides on one factorization: ms per right-hand side of the refinement
    f = ctx.factor(A_d, tf="f16", autotune=True)
    g = np.random.Generator(np.random.PCG64(7))
    B = torch.from_numpy(g.standard_normal((A_d.shape[0], 4))).to(A_d.device)
    B[:, 0] = b_d
    _, rep1 = f.solve(b_d, term=term)
    ms1, _, _, _ = timed_steps(lambda: f.solve(b_d, term=term)[1], steps, 1)
    ms4, out4, _, _ = timed_steps(lambda: f.solve_many(B, term=term), steps, 1)
    X, reps = f.solve_many(B, term=term)
    out["four_rhs"] = {"refine_ms_per_rhs": statistics.mean(ms4) / 4, "refine_ms_single_rhs": statistics.mean(ms1),
                       "iters": [r.iters for r in reps], "status": [r.status for r in reps],
                       "column0_bitwise_single": bool(np.array_equal(X[:, 0].cpu().numpy(), x16h)),
                       "note": "refinement only (the factorization is shared); solves apply each factor tile to "
                               "all four columns, the residual reads A once for all of them"}
    f.destroy()
    return out


def ws_of():
    return int(os.environ.get("WORLD_SIZE", "1"))


def O_ref(A, b):
    import oracle as O
    return O.reference_solution(A, b)


def run_krylov(args, ctx, dev, ws, timed_steps):
    """GMRES-IR (Sec. 4.3) and BiCGSTAB-IR (Sec. 2.3, 4.2) with binary16 factors on the
    N = 4096 Green's system, where plain IR with the same factors does not converge."""
    import numpy as np
    import torch

    import irgen
    from paper_2311_14616_gb300 import ir
    A, b, xt = irgen.case_green_sine(4096, ALPHA)
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()
    b_d = torch.from_numpy(b).to(dev)
    term = ir.default_term()
    fact16 = ctx.factor(A_d, tf="f16")
    fact16.gmres_reserve(10)
    xg16 = torch.empty_like(b_d)
    x16 = torch.empty_like(b_d)
    kopts = ir.krylov_opts()
    rel = lambda v: float(np.max(np.abs(v.double().cpu().numpy() - xt)) / np.max(np.abs(xt)))

    def step_gm():
        fact16.refactor(A_d)
        return fact16.solve_gmres(b_d, xg16, term, kopts)[1]

    gsteps = max(3, args.steps // 2)
    _, _, prof_gm, l_gm = timed_steps(step_gm, gsteps, 1, profile=True)
    ms_gm, rep_gm, _, _ = timed_steps(step_gm, gsteps, 1)
    _, rep_ir16 = fact16.solve(b_d, x16, term)
    fact16.bicgstab_reserve()
    xb16 = torch.empty_like(b_d)

    def step_bi():
        fact16.refactor(A_d)
        return fact16.solve_bicgstab(b_d, xb16, term, kopts)[1]

    _, _, prof_bi, l_bi = timed_steps(step_bi, gsteps, 1, profile=True)
    ms_bi, rep_bi, _, _ = timed_steps(step_bi, gsteps, 1)
    fact16.destroy()
    return {
        "workload": "green_sine_N4096_alpha800_TWf64_TFf16_TRf64_basis10",
        "gmres_ir": {"ms": max_over_ranks(statistics.mean(ms_gm), ws), "unit": "ms (refactor + GMRES-IR solve)",
                     "iters": rep_gm.iters, "status": rep_gm.status, "khist": rep_gm.khist,
                     "rel_err_vs_closed_form": rel(xg16),
                     "kernel_ms_per_step": {k: v[0] / gsteps for k, v in sorted(prof_gm.items())},
                     "gpu_launches_per_step": l_gm / gsteps},
        "bicgstab_ir": {"ms": max_over_ranks(statistics.mean(ms_bi), ws),
                        "unit": "ms (refactor + BiCGSTAB-IR solve)", "iters": rep_bi.iters,
                        "status": rep_bi.status, "khist": rep_bi.khist, "rel_err_vs_closed_form": rel(xb16),
                        "kernel_ms_per_step": {k: v[0] / gsteps for k, v in sorted(prof_bi.items())},
                        "gpu_launches_per_step": l_bi / gsteps},
        "ir_same_factors": {"iters": rep_ir16.iters, "status": rep_ir16.status, "rel_err_vs_closed_form": rel(x16)},
    }


if __name__ == "__main__":
    main()
