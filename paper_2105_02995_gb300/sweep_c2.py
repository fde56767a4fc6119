"""Sweep of the 1D Example 1 workloads at large N (paper section 6, Example 1; Table for Example 1
sizes): the approximate inverse as a direct solver and as the preconditioner of GMRES.

    python -m paper_2105_02995_gb300.sweep_c2 [--n 16384,65536] [--eps 1e-6,1e-9] [--b 1,8,64]
                                             [--reps 10]

For every N and tolerance eps (eps_HIF = eps, eps_BF = eps / 10) the operator is built (or taken
from the on-disk cache) and uploaded; then, per right-hand-side count b:
  * direct solve f = G-dot K-dot* u: complex128 vectors in FP64 arithmetic and complex64 vectors in
    FP32 arithmetic (autotuned kernels), RHS/s and RHS*N/s from CUDA events (median of reps,
    inputs resident, L2 flushed by a 256 MB write before each), and p50 / p99 latency;
  * GMRES on K-dot f = u right-preconditioned with G-dot K-dot* to ||u - K-dot f|| <= 1e-10 ||u||
    (FP64 solution and residuals; preconditioner in FP64 and in FP32): p50 / p99 latency over
    reps solves, RHS/s, iterations, final residual recomputed with the FP64 apply.
The right-hand sides are seeded complex Gaussians (paper_2105_02995_gb300.inputs).  Prints one
JSON object per (N, eps) on stdout.  No oracle is involved: these are measurements of the library.
"""

from __future__ import annotations

import argparse
import json
import statistics
import time


def _pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(q * len(v)))]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", default="16384,65536")
    ap.add_argument("--eps", default="1e-6,1e-9")
    ap.add_argument("--b", default="1,8,64")
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    import numpy as np
    import torch

    from . import binding, build as fbuild
    from .builder.__main__ import build_cached
    from .inputs import complex_gaussian, rhs_seed

    fbuild.build()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for n in [int(v) for v in a.n.split(",")]:
        for eps in [float(v) for v in a.eps.split(",")]:
            t0 = time.perf_counter()
            buf, info = build_cached("ex1", n, eps / 10, eps, gpu=True, verbose=False)
            op = binding.Operator(buf)
            out = {"kind": "ex1", "N": n, "eps_hif": eps, "eps_bf": eps / 10, "root": info.get("root"),
                   "build_s": round(time.perf_counter() - t0, 1), "direct": {}, "gmres": {}}
            for b in [int(v) for v in a.b.split(",")]:
                u_np = complex_gaussian(n, b, rhs_seed(1, b))
                for tag, dt, prec in (("c128_fp64", torch.complex128, binding.FIO_P64),
                                      ("c64_fp32", torch.complex64, binding.FIO_P32)):
                    op.autotune(b, prec)
                    u = binding.colmajor(torch.from_numpy(u_np).to("cuda", dt))
                    f = binding.colmajor(torch.empty_like(u))
                    for _ in range(3):
                        op.apply_inv(u, f)
                    torch.cuda.synchronize()
                    ms = []
                    for k in range(a.reps):
                        flush.fill_(float(k))
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        op.apply_inv(u, f)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ms.append(e0.elapsed_time(e1))
                    med = statistics.median(ms)
                    out["direct"][f"{tag}_b{b}"] = {"rhs_per_s": round(b * 1000 / med, 1),
                                                    "rhs_N_per_s": round(b * n * 1000 / med, 1),
                                                    "p50_ms": round(med, 4), "p99_ms": round(_pct(ms, 0.99), 4)}
                u = binding.colmajor(torch.from_numpy(u_np).cuda())
                for tag, inner in (("fp64_precond", binding.FIO_P64), ("fp32_precond", binding.FIO_P32)):
                    lat, its, rr = [], [], []
                    ff = None
                    for _ in range(max(3, a.reps // 2)):
                        torch.cuda.synchronize()
                        s = time.perf_counter()
                        ff, infos = op.solve(u, method=binding.FIO_GMRES, inner=inner, tol=1e-10, maxit=100)
                        lat.append(1000 * (time.perf_counter() - s))
                        its += [i for i, _, _ in infos]
                        rr += [r for _, r, st in infos]
                    res = u - op.apply_K(ff)
                    chk = float((torch.linalg.norm(res, dim=0) / torch.linalg.norm(u, dim=0)).max())
                    out["gmres"][f"{tag}_b{b}"] = {"p50_ms": round(statistics.median(lat), 3),
                                                   "p99_ms": round(_pct(lat, 0.99), 3),
                                                   "rhs_per_s": round(b * 1000 / statistics.mean(lat), 2),
                                                   "iters_max": max(its), "relres_max": max(rr),
                                                   "relres_fp64_check": float("%.3g" % chk)}
            print(json.dumps(out), flush=True)
            op.release()


if __name__ == "__main__":
    main()
