"""Benchmark of the inverse apply f = G-dot K-dot* u (the direct solver of the approximate FIO
inverse) on the 2D generalized Radon transform, n = 256 (N = 65536), complex64, 32 right-hand
sides per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

A step is one inverse apply of a batch of b seeded complex-Gaussian right-hand sides already
resident in HBM.  L2 (129 MB) is flushed by a 256 MB write before every timed step; the flush is
outside the per-step CUDA-event interval.  value = right-hand sides solved per second by the
whole job (sum over ranks / max time over ranks).  The factors are built once per operator on the
host before timing (cached on disk between runs of the same box).

Multi-GPU: replicas only (the right-hand sides are independent): every rank applies its own
batch with its own copy of the factors; no collective on the data path.

Before timing, every stage launch's kernel variant is picked by the autotuner (fio_autotune) for
the batches timed here (--no-autotune keeps the built-in shapes).  Beside the headline the JSON
line carries: roofline (FLOP/s of the stage launches against the FP32 CUDA-core peak, DRAM
traffic per apply from the committed ncu capture), e2e (host buffers through fio_apply_inv_host),
cpu_baseline (the oracle), the tensor-core variants and the full solve f = F^{-1} G K* u,
per-stage errors of every precision against the FP64 path, and solve latencies to residual
1e-10 (plain FP64 PCG one right-hand side at a time against iterative refinement on batches).
--kind / --n / --eps-bf / --eps-hif select another operator (e.g. Example 2: --kind ex2b --n
65536 --eps-bf 1e-7 --eps-hif 1e-4).

--impl reference times the oracle (oracle/factor_apply.py: the same factors multiplied out as
sparse matrices in FP64 on the host cores) on a bounded sample of the same workload.
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

HBM_FALLBACK_GBS = 6800.0
FP32_LANES = 128  # FP32 FMA lanes per SM (nominal; the roofline uses the measured rate)


# headline precision: name -> (fio precision, dtype string, description, stage kernel source)
PRECISIONS = {
    "fp32": ("FIO_P32", "f32", "FP32 arithmetic on the CUDA cores", "fio_kernels.cuh"),
    "split_tf32": ("FIO_PTF32X3", "tf32x3",
                   "split-TF32 tensor-core products (head x head + head x tail + tail x head, FP32 accumulation)",
                   "fio_tma.cuh"),
    "tf32": ("FIO_PTF32", "tf32", "TF32 tensor-core products, FP32 accumulation", "fio_tma.cuh"),
    "bf16": ("FIO_PBF16", "bf16", "BF16 tensor-core products, FP32 accumulation", "fio_tma.cuh"),
}


def measured_traffic(precision="fp32"):
    """DRAM bytes per apply of the stage kernels from the committed ncu summary, or None when the
    kernel source changed since the counters were taken (the summary records its hash)."""
    import hashlib
    name = "traffic_ex3_n256_b32.md" if precision == "fp32" else f"traffic_ex3_n256_b32_{precision}.md"
    prof = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_2105_02995_gb300", "csrc", PRECISIONS[precision][3])
    try:
        text = open(prof).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if f"kernel_source_sha256_16: {h}" not in text:
            return None
        for line in text.splitlines():
            if line.startswith("traffic_bytes_per_apply:"):
                return int(line.split(":")[1])
    except OSError:
        return None
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"fio_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi's start-up (driver queries) can stall the GPU for a moment: let it finish,
        # i.e. wait for the first sample, before the timed region begins
        t0 = time.time()
        while time.time() - t0 < 10.0 and self.proc.poll() is None:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def get_operator(a, rank, ws):
    """Rank 0 builds (or reuses the on-disk cache); the others read the cache after a barrier.
    The build's peeling probes run on the GPU when there is one."""
    import torch
    from paper_2105_02995_gb300.builder.__main__ import build_cached
    if rank == 0:
        buf, info = build_cached(a.kind, a.n, a.eps_bf, a.eps_hif, gpu=torch.cuda.is_available(), verbose=True)
    barrier(ws)
    if rank != 0:
        buf, info = build_cached(a.kind, a.n, a.eps_bf, a.eps_hif, gpu=False, verbose=False)
    return buf, info


OPERATORS = {"ex3": "2D generalized Radon transform (Example 3)", "ex1": "1D FIO (Example 1)",
             "ex2a": "1D FIO with variable amplitude, sigma^2 = 0.1 (Example 2)",
             "ex2b": "1D FIO with variable amplitude, sigma^2 = 0.05 (Example 2)"}


def grid_size(a):
    return a.n * a.n if a.kind == "ex3" else a.n


def metric_of(a):
    """The headline metric's name (2D n = 256 by default; other operators name themselves)."""
    if a.kind == "ex3":
        return f"inverse-apply RHS/s at 2D n={a.n}"
    return f"inverse-apply RHS/s at {a.kind} N={a.n}"


def config_of(a, info, l2):
    N = grid_size(a)
    size = f"n={a.n} (N={N})" if a.kind == "ex3" else f"N={N}"
    return {"workload": f"{OPERATORS.get(a.kind, a.kind)}, {size}, direct "
                        f"inverse apply f = G K* u, complex64 vectors ({PRECISIONS[a.precision][2]}), "
                        f"b={a.b} RHS per step",
            "precision": a.precision,
            "kind": a.kind, "n": a.n, "N": N, "b": a.b, "eps_bf": a.eps_bf, "eps_hif": a.eps_hif,
            "L": info.get("L"), "LH": info.get("LH"), "root": info.get("root"), "l2": l2,
            "parallelism": "replicas"}


def host_threads():
    return max(1, os.cpu_count() or 1)


def oracle_round(P, u_np, cols, nthreads):
    """The oracle's direct solve (oracle/factor_apply.py, unchanged) of the given right-hand sides,
    one per host thread at a time (scipy's sparse products release the GIL); returns seconds."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import factor_apply as fa
    s = time.perf_counter()
    with ThreadPoolExecutor(nthreads) as ex:
        list(ex.map(lambda j: fa.apply_inv(P, u_np[:, j:j + 1]), cols))
    return time.perf_counter() - s


def cpu_baseline(buf, a, u_np, budget_s=20.0):
    """The oracle's product of the packed factors (FP64, scipy sparse) on a bounded sample, on all
    host cores: rounds of one right-hand side per thread until the budget is spent."""
    from oracle import factor_apply as fa
    t0 = time.time()
    P = fa.PackedFactors(buf, verify=False)
    t_parse = time.time() - t0
    nth = host_threads()
    done, t = 0, 0.0
    while t < budget_s:
        cols = [(done + k) % u_np.shape[1] for k in range(nth)]
        t += oracle_round(P, u_np, cols, nth)
        done += nth
    return {"value": done / t, "unit": "RHS/s", "cores": nth, "kind": "oracle",
            "sample": f"{done} right-hand sides (columns of the {a.b}-RHS batch), one per host thread at a time "
                      f"on {nth} threads, FP64 sparse products of the same packed factors ({t:.1f} s; factor "
                      f"parse {t_parse:.1f} s untimed)"}


def run_reference(a, ws, rank):
    if rank != 0:
        return
    from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed
    buf, info = get_operator(a, 0, 1)
    u = complex_gaussian(grid_size(a), a.b, rhs_seed(2))
    from oracle import factor_apply as fa
    P = fa.PackedFactors(buf, verify=False)
    nth = host_threads()
    # a step: one right-hand side per host thread, all threads at once
    for k in range(a.warmup):
        oracle_round(P, u, [(k * nth + j) % a.b for j in range(nth)], nth)
    times = [oracle_round(P, u, [(k * nth + j) % a.b for j in range(nth)], nth) for k in range(a.steps)]
    ms = 1000 * statistics.mean(times)
    val = nth * 1000.0 / ms
    line = {"metric": metric_of(a), "value": val, "unit": "RHS/s", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_of(a, info, "host only"),
            "cpu_baseline": {"value": val, "unit": "RHS/s", "cores": nth, "kind": "oracle",
                             "sample": f"per step {nth} right-hand sides of the {a.b}-RHS batch, one per host "
                                       f"thread, the oracle's FP64 sparse products of the same factors"},
            "e2e": {"value": val, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def solve_converged(e):
    """Equal final residual: every right-hand side reported convergence, and the residual
    recomputed with the FP64 apply is at 1e-10 (5% margin for the recomputation's rounding)."""
    return bool(e.get("statuses_ok")) and e.get("relres_max", 1.0) <= 1e-10 and e.get("relres_fp64_check", 1.0) <= 1.05e-10


def solve_summary(solves):
    """The mixed, batched path with the highest RHS/s at residual 1e-10 against the plain FP64
    path (both held to solve_converged); an error entry when the plain path did not converge or no
    mixed path did."""
    try:
        plain = solves["plain_fp64_pcg_b1"]
        if not solve_converged(plain):
            raise RuntimeError("the plain FP64 path did not reach 1e-10")
        cands = [k for k in solves if (k.startswith("ir_") or k.startswith("gmres_")) and solve_converged(solves[k])]
        if not cands:
            raise RuntimeError("no mixed-precision path reached 1e-10")
        best_tag = max(cands, key=lambda k: solves[k]["rhs_per_s"])
        best = solves[best_tag]
        return {"plain": "plain_fp64_pcg_b1", "plain_p50_ms": plain["p50_ms"],
                "plain_p99_ms": plain["p99_ms"], "plain_rhs_per_s": plain["rhs_per_s"],
                "best": best_tag, "best_p50_ms": best["p50_ms"], "best_p99_ms": best["p99_ms"],
                "best_rhs_per_s": best["rhs_per_s"],
                "rhs_per_s_ratio": round(best["rhs_per_s"] / plain["rhs_per_s"], 2)}
    except Exception as exc:
        return {"error": str(exc)[:200]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--kind", default="ex3")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--b", type=int, default=32)
    ap.add_argument("--eps-bf", type=float, default=1e-4)
    ap.add_argument("--eps-hif", type=float, default=1e-3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in tile shapes")
    ap.add_argument("--tight-eps-bf", type=float, default=0.0,
                    help="also time refinement whose outer residual uses a butterfly built with this tolerance")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="arithmetic of the timed apply (complex64 vectors)")
    a = ap.parse_args()
    a.warmup = max(3, a.warmup)
    ws, rank, local = dist_init()
    if a.impl == "reference":
        run_reference(a, ws, rank)
        return

    import numpy as np
    import torch

    from paper_2105_02995_gb300 import binding, build as fbuild
    from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed
    from paper_2105_02995_gb300.packinfo import totals

    torch.cuda.set_device(local)
    if rank == 0:
        fbuild.build()
    barrier(ws)
    buf, info = get_operator(a, rank, ws)
    op = binding.Operator(buf)
    N, b = op.N, a.b
    u_np = complex_gaussian(N, b, rhs_seed(2, rank))
    u = binding.colmajor(torch.from_numpy(u_np.astype(np.complex64)).cuda())
    f = binding.colmajor(torch.empty_like(u))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    hp = getattr(binding, PRECISIONS[a.precision][0])  # the timed apply's precision

    # autotuner: every stage launch's tile shape picked by timing, for the batches timed below
    # (FP32 headline and inner corrections, double-float residuals, and the FP64 b = 1 plain path)
    tuned = {}
    if not a.no_autotune:
        t0 = time.perf_counter()
        for tb, tp, tag in ((b, binding.FIO_P32, f"fp32_b{b}"), (b, binding.FIO_PTF32, f"tf32_b{b}"),
                            (b, binding.FIO_PBF16, f"bf16_b{b}"), (b, binding.FIO_PTF32X3, f"split_tf32_b{b}"),
                            (b, binding.FIO_PDF, f"df_b{b}"), (16, binding.FIO_PTF32X3, "split_tf32_b16"),
                            (128, binding.FIO_PTF32X3, "split_tf32_b128"),
                            (1, binding.FIO_P64, "fp64_b1"), (1, binding.FIO_P32, "fp32_b1"),
                            (1, binding.FIO_PDF, "df_b1"), (16, binding.FIO_PDF, "df_b16"),
                            (128, binding.FIO_PDF, "df_b128")):
            ch = op.autotune(tb, tp)
            tuned[tag] = {str(v): ch.count(v) for v in sorted(set(ch))}
        tuned["seconds"] = round(time.perf_counter() - t0, 2)

    for _ in range(a.warmup):
        op.apply_inv(u, f, precision=hp)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    op.apply_inv(u, f, precision=hp)  # one more untimed step after the sampler has started
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("fio_timed")  # lets a profiler select exactly the timed launches
    for k in range(a.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        op.apply_inv(u, f, precision=hp)
        ev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(ws)
    ck = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    ms = allmax(ws, statistics.mean(step_ms))
    value = ws * b * 1000.0 / ms

    # per-stage times of the same apply (events after every launch group, same flush discipline)
    tot = totals(buf)
    st = tot["stages"]
    nbf = tot["n_bf"]
    groups = []  # (label, stage dict or None), in the order fio_apply_profiled marks them
    if b >= 5 and nbf > 1:
        groups.append(("layout", None))  # caller's column-major u -> row-major work array
    for s in reversed(range(nbf)):
        groups.append(("bf", st[s]))
    hif = st[nbf:]
    nh = len(hif) - 1 if hif and hif[-1]["role"] == "root" else len(hif)
    for s in range(nh):
        groups.append(("hif", hif[s]))
    if len(hif) > nh:
        groups.append(("root", hif[nh]))
    for s in reversed(range(nh)):
        groups.append(("hif", hif[s]))
    groups.append(("layout", None))
    prof = []
    for k in range(max(3, min(a.steps, 10))):
        flush.fill_(float(k))
        prof.append(op.apply_profiled("inv", u, f, precision=hp))
    per = [statistics.mean(p[i] for p in prof) for i in range(len(prof[0]))]
    es = 4 if a.precision == "bf16" else 8  # bytes per complex factor entry read by the kernels
    kern_time = kern_flops = kern_bytes = 0.0
    stage_rows = []
    for (lab, sd), t in zip(groups, per):
        if sd is None:
            continue
        flops = 8.0 * sd["nnz"] * b
        byt = es * sd["nnz"] + es * b * (sd["in_len"] + sd["out_len"] if lab == "bf" else 2 * sd["touched"])
        kern_time += t
        kern_flops += flops
        kern_bytes += byt
        stage_rows.append({"group": lab, "role": sd["role"], "level": sd["level"], "ms": round(t, 4),
                           "tflops": round(flops / t / 1e9, 2), "gbs": round(byt / t / 1e6, 1)})
    peaks, src = measured_peaks()
    # the FP32 FMA rate of this device, measured (fio_probe_fp32: independent FMA chains on every
    # SM, CUDA events), with the SM clock sampled around it
    pclk = Clocks(local)
    pclk.start()
    fp32_peak, fp32_probe_ms, nsm = binding.probe_fp32(1 << 20)
    pck = pclk.stop()
    nominal = nsm * FP32_LANES * 2 * (pck.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    achieved = kern_flops / (kern_time / 1e3) / 1e12
    hbm_peak = peaks.get("hbm_gbs") or HBM_FALLBACK_GBS
    achieved_gbs = kern_bytes / (kern_time / 1e3) / 1e9
    # the apply's HBM floor (factors read once, u read and f written once): s (P_K + 2 P_G) + 2 s N b
    floor_bytes = es * (tot["P_K"] + 2 * tot["P_G"]) + 2 * 8 * N * b
    alu_view = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4),
                "peak_source": f"measured: FFMA-chain kernel (fio_probe_fp32) on {nsm} SMs, {fp32_probe_ms:.2f} ms "
                               f"per launch, SM clock median {pck.get('sm_mhz')} MHz (max {pck.get('sm_max_mhz')}); "
                               f"nominal {nsm} SMs x {FP32_LANES} lanes x 2 flop x max clock = {nominal:.1f}"}
    hbm_view = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved_gbs / hbm_peak, 4), "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
    main_view = alu_view if a.precision == "fp32" else hbm_view
    roof = dict(main_view)
    roof.update({
        "traffic": measured_traffic(a.precision) if (a.n == 256 and b == 32 and a.kind == "ex3") else None,
        "traffic_unit": "DRAM bytes per apply (all stage launches), ncu",
        "kernel": ("stage kernels k_stage_mm_vt / k_stage_mm_pipe" if a.precision == "fp32" else
                   "stage kernels k_stage_tma (TMA-fed tcgen05) and k_stage_tc") +
                  f" (every stage launch of one apply, complex64 vectors, b={b}, autotuned variants)",
        "algorithmic_bytes_per_apply": int(kern_bytes),
        "algorithmic_bytes_definition": "per stage launch: factor entries read once + its input and output "
                                        "vectors (s nnz + s b (in_len + out_len))",
        "other_view": hbm_view if a.precision == "fp32" else alu_view,
        "apply_floor": {"bytes": int(floor_bytes), "definition": "s (P_K + 2 P_G) + 2 s N b",
                        "floor_ms": round(floor_bytes / hbm_peak / 1e6, 4),
                        "frac_of_step": round(floor_bytes / hbm_peak / 1e6 / ms, 4)},
        "stage_ms_sum": round(kern_time, 4), "step_ms": round(ms, 4)})

    # tensor-core stage products (tcgen05: TF32 / BF16 operands, and split TF32 at FP32 accuracy;
    # FP32 accumulation) and the FP32 CUDA cores, same timing; rel_diff_vs_headline =
    # ||f_variant - f_headline|| / ||f_headline||
    variants = {}
    f_head = f.clone()
    # the FP64 apply of the same (complex64-valued) right-hand sides: the reference for the error
    # of every complex64 result (the FP64 path agrees with the oracle's product of the same
    # factors to 1e-12 in the parity tests)
    f_ref = op.apply_inv(binding.colmajor(u.to(torch.complex128)))
    torch.cuda.synchronize()

    def err64(x):
        return float("%.3g" % float(torch.linalg.norm(x.to(torch.complex128) - f_ref) / torch.linalg.norm(f_ref)))

    head_err = err64(f_head)
    for name, prec in (("fp32_cuda_cores", binding.FIO_P32), ("tf32_tensor_core", binding.FIO_PTF32),
                       ("bf16_tensor_core", binding.FIO_PBF16), ("split_tf32_tensor_core", binding.FIO_PTF32X3)):
        if prec == hp:
            continue
        try:
            for _ in range(3):
                op.apply_inv(u, f, precision=prec)
            torch.cuda.synchronize()
            vdiff = float(torch.linalg.norm(f - f_head) / torch.linalg.norm(f_head))
            evv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(a.steps)]
            for k in range(a.steps):
                flush.fill_(float(k))
                evv[k][0].record(stream)
                op.apply_inv(u, f, precision=prec)
                evv[k][1].record(stream)
            torch.cuda.synchronize()
            vms = allmax(ws, statistics.mean(s_.elapsed_time(e_) for s_, e_ in evv))
            variants[name] = {"value": round(ws * b * 1000.0 / vms, 2), "unit": "RHS/s", "ms_per_step": round(vms, 4),
                              "rel_diff_vs_headline": float("%.3g" % vdiff), "rel_err_vs_fp64": err64(f)}
        except Exception as exc:  # reported, not hidden: the variant line says why it is missing
            variants[name] = {"error": str(exc)[:200]}

    # full solve of u = K F f (section 1): f = F^{-1} G K* u, complex64; and the inverse DFT alone
    # (two shared-memory FFT passes, each reading and writing the N x b vector: HBM-bound)
    try:
        fsol = binding.colmajor(torch.empty_like(u))
        for _ in range(3):
            op.apply_inv(u, f, precision=hp)
            op.apply_Finv(f, fsol)
        torch.cuda.synchronize()
        evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for k in range(a.steps):
            flush.fill_(float(k))
            evf[k][0].record(stream)
            op.apply_inv(u, f, precision=hp)
            evf[k][1].record(stream)
            op.apply_Finv(f, fsol)
            evf[k][2].record(stream)
        torch.cuda.synchronize()
        full_ms = allmax(ws, statistics.mean(e0.elapsed_time(e2) for e0, _, e2 in evf))
        finv_ms = statistics.mean(e1.elapsed_time(e2) for _, e1, e2 in evf)
        npass = 2 if (info.get("d", 2) == 2 or N > 2048) else 1
        finv_bytes = npass * 2 * 8 * N * b
        peak_hbm = measured_peaks()[0].get("hbm_gbs")
        variants["full_solve_u_eq_KFf"] = {
            "value": round(ws * b * 1000.0 / full_ms, 2), "unit": "RHS/s", "ms_per_step": round(full_ms, 4),
            "Finv_ms": round(finv_ms, 4), "Finv_gbs": round(finv_bytes / finv_ms / 1e6, 1),
            "Finv_frac_of_hbm": round(finv_bytes / finv_ms / 1e6 / peak_hbm, 3) if peak_hbm else None,
            "Finv_bytes_per_apply": finv_bytes}
    except Exception as exc:
        variants["full_solve_u_eq_KFf"] = {"error": str(exc)[:200]}

    # the tensor-core kernel variants stage by stage on this operator (every stage launch of the
    # apply pinned to one variant at a time; CUDA events per launch group): what the autotuner
    # weighs, for the headline's tensor-core precision
    variant_ms = {}
    if a.precision != "fp32":
        try:
            for var in (0, 20, 30, 31, 32, 33):
                op.set_variant(b, hp, var)
                for _ in range(2):
                    op.apply_profiled("inv", u, f, precision=hp)
                runs = []
                for k in range(3):
                    flush.fill_(float(k))
                    runs.append(op.apply_profiled("inv", u, f, precision=hp))
                variant_ms[str(var)] = [round(min(r[i] for r in runs), 4) for i in range(len(runs[0]))]
            variant_ms["groups"] = [lab if sd is None else f"{lab}:{sd['role']}:{sd['level']}" for lab, sd in groups]
        except Exception as exc:
            variant_ms["error"] = str(exc)[:200]
        finally:
            op.set_variant(b, hp, 0)
            if not a.no_autotune:
                op.autotune(b, hp)  # restore the tuned choices

    # per-stage error of every precision against the FP64 path (8 right-hand sides: the
    # tensor-core precisions need b >= 8), in application order of the inverse apply
    stage_err = {}
    try:
        u8 = binding.colmajor(torch.from_numpy(u_np[:, :8]).cuda())
        for tag, prec in (("fp32", binding.FIO_P32), ("tf32", binding.FIO_PTF32), ("bf16", binding.FIO_PBF16),
                          ("split_tf32", binding.FIO_PTF32X3), ("double_float", binding.FIO_PDF)):
            stage_err[tag] = [float("%.3g" % e) for e in op.stage_errors("inv", u8, prec)]
    except Exception as exc:
        stage_err["error"] = str(exc)[:200]

    # solve latency to ||u - K-dot f|| <= 1e-10 ||u||: the plain FP64 path (PCG on K*K with G, FP64
    # factors, one right-hand side per call) against FP64-residual iterative refinement whose
    # corrections run on the tensor cores, on batches of b right-hand sides
    solves = {}
    u128 = binding.colmajor(torch.from_numpy(u_np).cuda())

    def timed_solves(tag, make_u, reps, **kw):
        lat, its, rr = [], [], []
        for _ in range(reps):
            uu = make_u()
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            ff, infos = op.solve(uu, tol=1e-10, maxit=200, **kw)
            lat.append(1000 * (time.perf_counter() - s0))
            its += [i for i, _, _ in infos]
            rr += [r for _, r, _ in infos]
        nb = make_u().shape[1] if make_u().dim() == 2 else 1
        # the last solution's residual recomputed with the FP64 apply of the operator the solve
        # was held to (outside the timed region)
        rop = kw.get("residual_op") or op
        ru = uu - rop.apply_K(ff)
        rr64 = float((torch.linalg.norm(ru, dim=0) / torch.linalg.norm(uu, dim=0)).max())
        lat.sort()
        sts = [st for _, _, st in infos]
        solves[tag] = {"b": nb, "statuses_ok": all(st == 0 for st in sts), "p50_ms": round(statistics.median(lat), 3),
                       "p99_ms": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
                       "rhs_per_s": round(nb * 1000.0 / statistics.mean(lat), 2),
                       "iters_max": max(its), "relres_max": max(rr), "relres_fp64_check": float("%.3g" % rr64),
                       "solves": reps}

    try:
        cols = iter(range(10 ** 9))
        timed_solves("plain_fp64_pcg_b1", lambda: binding.colmajor(u128[:, next(cols) % b:][:, :1].contiguous()),
                     6, method=binding.FIO_PCG, inner=binding.FIO_P64)
        # iterative refinement, FP64 residuals (FP64 stage arithmetic)
        timed_solves(f"ir_fp32_inner_fp64res_b{b}", lambda: u128, 3, method=binding.FIO_IR, inner=binding.FIO_P32)
        # iterative refinement, double-float residuals, inner corrections in each precision
        for tag, inner in (("fp32", binding.FIO_P32), ("split_tf32", binding.FIO_PTF32X3),
                           ("tf32", binding.FIO_PTF32), ("bf16", binding.FIO_PBF16)):
            timed_solves(f"ir_{tag}_inner_dfres_b{b}", lambda: u128, 3, method=binding.FIO_IR, inner=inner,
                         outer=binding.FIO_PDF)
        # the right-hand-side batches of the mixed-precision configuration (1, 16, 128)
        u_more = complex_gaussian(N, 128, rhs_seed(3, rank))
        u_more = binding.colmajor(torch.from_numpy(u_more).cuda())
        for nb in (1, 16, 128):
            timed_solves(f"ir_split_tf32_inner_dfres_b{nb}", lambda: binding.colmajor(u_more[:, :nb].contiguous()),
                         3, method=binding.FIO_IR, inner=binding.FIO_PTF32X3, outer=binding.FIO_PDF)
        timed_solves(f"gmres_fp32_precond_b{b}", lambda: u128, 3, method=binding.FIO_GMRES, inner=binding.FIO_P32)
        if a.tight_eps_bf > 0:
            # the outer residual u - K-dot_tight f with a tighter butterfly of the same FIO (the
            # corrections still come from this operator's G-dot K-dot*)
            from paper_2105_02995_gb300.builder.__main__ import build_cached
            t0 = time.perf_counter()
            tbuf, tinfo = build_cached(a.kind, a.n, a.tight_eps_bf, a.eps_hif, verbose=rank == 0, butterfly_only=True)
            tight = binding.Operator(tbuf, binding.FIO_MASK_P64 | binding.FIO_MASK_DF)
            tight_build_s = time.perf_counter() - t0
            for nb in (1, 16, 128):
                timed_solves(f"ir_split_tf32_inner_dfres_tight_b{nb}",
                             lambda: binding.colmajor(u_more[:, :nb].contiguous()), 3, method=binding.FIO_IR,
                             inner=binding.FIO_PTF32X3, outer=binding.FIO_PDF, residual_op=tight)
                solves[f"ir_split_tf32_inner_dfres_tight_b{nb}"].update(
                    {"tight_eps_bf": a.tight_eps_bf, "tight_nnz": tinfo.get("nnz_bf"),
                     "tight_build_s": round(tight_build_s, 1)})
            tight.release()
    except Exception as exc:
        solves["error"] = str(exc)[:200]
    solves["summary"] = solve_summary(solves)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    uh = torch.from_numpy(u_np.astype(np.complex64)).t().contiguous().pin_memory()  # (b, N) rows = RHS
    fh = torch.empty_like(uh).pin_memory()
    uh_np, fh_np = uh.numpy().T, fh.numpy().T  # (N, b) Fortran views
    for _ in range(2):
        op.apply_inv_host(uh_np, fh_np, precision=hp)
    barrier(ws)
    s = time.perf_counter()
    for _ in range(a.steps):
        op.apply_inv_host(uh_np, fh_np, precision=hp)
    e2e_ms = allmax(ws, 1000 * (time.perf_counter() - s) / a.steps)
    e2e = {"value": ws * b * 1000.0 / e2e_ms, "unit": "RHS/s", "h2d_bytes_per_step": N * b * 8,
           "d2h_bytes_per_step": N * b * 8, "ms_per_step": e2e_ms}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(buf, a, u_np)
    launches = op.launches("inv", b) * a.steps
    if rank == 0:
        line = {"metric": metric_of(a), "value": round(value, 2), "unit": "RHS/s",
                "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": PRECISIONS[a.precision][1],
                "data": "synthetic", "config": config_of(a, info, "flushed before every step (256 MB write)"),
                "rhs_N_per_s": round(value * N, 1), "wall_ms_per_step": round(1000 * t_wall / a.steps, 4),
                "clocks": ck, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "stages": stage_rows, "variants": variants, "solve_latency": solves,
                "autotune": tuned, "variant_stage_ms": variant_ms, "rel_err_vs_fp64": head_err, "stage_errors_vs_fp64": stage_err,
                "factors": {"P_K": tot["P_K"], "P_G": tot["P_G"], "padded_K": tot["padded_K"],
                            "padded_G": tot["padded_G"], "bytes_c64": 8 * (tot["padded_K"] + tot["padded_G"]),
                            "build_s": {k: info.get(k) for k in ("t_bf", "t_peel", "t_hif", "t_total")}}}
        print(json.dumps(line), flush=True)
    op.release()


if __name__ == "__main__":
    main()
