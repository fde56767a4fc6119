"""Serving loop for inverse applies or solves of several resident operators, with continuous batching.

Requests (operator name, b complex64 right-hand sides, arrival time) arrive over time.  The loop:
  * admits a request when the device memory its batch needs fits the HBM budget (the factors of
    every operator are resident and counted once at start-up);
  * keeps one CUDA stream per operator; whenever an operator's stream is idle it gathers its
    waiting requests (up to max_batch right-hand sides) into ONE launch of fio_apply_inv, so
    requests that arrived while the previous batch was on the GPU join the next one;
  * batches of different operators run concurrently on their streams;
  * polls completion events without blocking; results go back to their requests, and the latency
    of a request is completion time minus arrival time.
mode="apply": a request is the direct solve f = G-dot K-dot* u (complex64, one fio_apply_inv per
batch).  mode="solve": a request is solved to a relative residual (fio_solve, iterative
refinement by default: FP64 solution, double-float residuals, corrections in the serving
precision); fio_solve synchronises its stream, so each operator gets one worker thread that runs
its batches (ctypes releases the interpreter lock during the call) and batches of different
operators still overlap on the device.
Every step runs in libfio's kernels through the C ABI; this module only schedules.
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    op: str
    u: np.ndarray          # (N, b) complex64, host
    t_arrival: float       # seconds after the start of the run
    t_done: float = -1.0
    f: np.ndarray = None   # (N, b) host result (complex64 applies, complex128 solves)
    info: list = None      # solve mode: (iterations, relative residual, status) per column


@dataclass
class _Batch:
    reqs: list
    event: object
    f_host: object
    cols: list
    nbytes: int


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    rhs: int = 0
    rhs_N: float = 0.0
    wall_s: float = 0.0
    launches: int = 0
    max_inflight_bytes: int = 0

    def summary(self):
        lat = np.sort(np.asarray(self.latencies_ms))
        if lat.size == 0:
            return {}
        return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "rhs": self.rhs,
                "rhs_per_s": self.rhs / self.wall_s, "rhs_N_per_s": self.rhs_N / self.wall_s,
                "launches": self.launches, "max_inflight_bytes": self.max_inflight_bytes,
                "wall_s": self.wall_s}


class Server:
    def __init__(self, ops: dict, max_batch: int = 64, hbm_budget: int | None = None,
                 precision: int | None = None, mode: str = "apply", solve_kw: dict | None = None):
        import torch
        from . import binding
        if mode not in ("apply", "solve"):
            raise ValueError("mode is 'apply' or 'solve'")
        self.torch = torch
        self.binding = binding
        self.ops = ops
        self.max_batch = max_batch
        self.precision = precision
        self.mode = mode
        self.solve_kw = dict(method=binding.FIO_IR, tol=1e-10, maxit=60, outer=binding.FIO_PDF,
                             inner=binding.FIO_P32 if precision is None else precision)
        self.solve_kw.update(solve_kw or {})
        self.workers = {}
        if mode == "solve":
            from concurrent.futures import ThreadPoolExecutor
            self.workers = {name: ThreadPoolExecutor(max_workers=1) for name in ops}
        self.streams = {name: torch.cuda.Stream() for name in ops}
        resident = sum(op.device_bytes() for op in ops.values())
        free, total = torch.cuda.mem_get_info()
        self.budget = hbm_budget if hbm_budget is not None else int(0.5 * free)
        self.resident = resident

    def close(self):
        """Stop the solve-mode worker threads (they are idle between runs)."""
        for ex in self.workers.values():
            ex.shutdown(wait=True)
        self.workers = {}

    def _batch_bytes(self, name, b):
        N = self.ops[name].N
        if self.mode == "solve":  # u, f in complex128 and the solver's work vectors
            return (8 + self.solve_kw.get("restart", 20)) * N * b * 16
        return 2 * N * b * 8  # device u and f of the batch (complex64)

    def _solve_batch(self, name, uh):
        """Runs in the operator's worker thread: one fio_solve of the batch on its stream."""
        torch = self.torch
        op = self.ops[name]
        with torch.cuda.stream(self.streams[name]):
            u = self.binding.colmajor(torch.from_numpy(uh.T.copy()).to("cuda", torch.complex128).t())
            f, infos = op.solve(u, **self.solve_kw)
            return f.t().contiguous().cpu().numpy().T, infos

    def warmup(self):
        """One launch per operator and batch width class, so scratch pools are sized up front."""
        torch = self.torch
        for name, op in self.ops.items():
            with torch.cuda.stream(self.streams[name]):
                for b in sorted({1, 2, 4, 8, 16, 32, self.max_batch}):
                    u = self.binding.colmajor(torch.zeros((op.N, b), dtype=torch.complex64, device="cuda"))
                    op.apply_inv(u, precision=self.precision)
                    if self.mode == "solve":
                        u1 = self.binding.colmajor(torch.ones((op.N, b), dtype=torch.complex128, device="cuda"))
                        op.solve(u1, **self.solve_kw)
        torch.cuda.synchronize()

    def run(self, requests: list, poll_sleep: float = 0.0) -> ServeStats:
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        waiting = collections.deque()                       # arrived, not yet admitted
        pending = {name: collections.deque() for name in self.ops}  # admitted, not launched
        inflight = {name: None for name in self.ops}
        st = ServeStats()
        inflight_bytes = 0
        reserved = {}                                         # rid -> bytes
        nxt = 0
        t0 = time.perf_counter()
        done = 0
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].t_arrival <= now:
                waiting.append(reqs[nxt])
                nxt += 1
            # admission by device memory
            while waiting:
                r = waiting[0]
                need = self._batch_bytes(r.op, r.u.shape[1])
                if inflight_bytes + need > self.budget and inflight_bytes > 0:
                    break
                waiting.popleft()
                inflight_bytes += need
                reserved[r.rid] = need
                pending[r.op].append(r)
                st.max_inflight_bytes = max(st.max_inflight_bytes, inflight_bytes)
            for name, op in self.ops.items():
                bt = inflight[name]
                if bt is not None and (bt.event.done() if self.mode == "solve" else bt.event.query()):
                    tnow = time.perf_counter() - t0
                    if self.mode == "solve":
                        fh, infos = bt.event.result()
                    else:
                        fh, infos = bt.f_host.numpy(), None
                    for r, (c0, c1) in zip(bt.reqs, bt.cols):
                        r.f = fh[:, c0:c1].copy()
                        if infos is not None:
                            r.info = infos[c0:c1]
                        r.t_done = tnow
                        st.latencies_ms.append(1000 * (tnow - r.t_arrival))
                        inflight_bytes -= reserved.pop(r.rid)
                        done += 1
                    inflight[name] = None
                if inflight[name] is None and pending[name]:
                    batch, cols, bsum = [], [], 0
                    while pending[name] and bsum + pending[name][0].u.shape[1] <= self.max_batch:
                        r = pending[name].popleft()
                        cols.append((bsum, bsum + r.u.shape[1]))
                        bsum += r.u.shape[1]
                        batch.append(r)
                    if not batch:  # a single request wider than max_batch goes alone
                        r = pending[name].popleft()
                        batch, cols, bsum = [r], [(0, r.u.shape[1])], r.u.shape[1]
                    uh = np.empty((op.N, bsum), dtype=np.complex64, order="F")
                    for r, (c0, c1) in zip(batch, cols):
                        uh[:, c0:c1] = r.u
                    st.launches += 1
                    st.rhs += bsum
                    st.rhs_N += bsum * op.N
                    if self.mode == "solve":
                        fut = self.workers[name].submit(self._solve_batch, name, uh)
                        inflight[name] = _Batch(batch, fut, None, cols, 0)
                        continue
                    s = self.streams[name]
                    with torch.cuda.stream(s):
                        ut = torch.from_numpy(uh.T.copy()).pin_memory().to("cuda", non_blocking=True).t()
                        fd = op.apply_inv(ut, precision=self.precision)
                        fh = torch.empty((bsum, op.N), dtype=torch.complex64, pin_memory=True)
                        fh.copy_(fd.t(), non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(s)
                    inflight[name] = _Batch(batch, ev, _T(fh), cols, 0)
            if poll_sleep:
                time.sleep(poll_sleep)
        st.wall_s = time.perf_counter() - t0
        return st


class _T:
    """Host result of a batch: (b, N) pinned tensor viewed as an (N, b) array."""

    def __init__(self, t):
        self.t = t

    def numpy(self):
        return self.t.numpy().T


def poisson_requests(ops: dict, n_requests: int, rate_per_s: float, seed: int, b_range=(1, 64)):
    """Seeded Poisson arrivals over the operators, 1-64 complex Gaussian right-hand sides each."""
    from .inputs import complex_gaussian
    rng = np.random.Generator(np.random.PCG64(seed))
    names = sorted(ops)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        name = names[rng.integers(len(names))]
        b = int(rng.integers(b_range[0], b_range[1] + 1))
        u = complex_gaussian(ops[name].N, b, seed + 1 + k, dtype=np.complex64)
        out.append(Request(k, name, u, t))
    return out


def main(argv=None):
    """Serving run over a mix of operators (built or reused from the on-disk cache)."""
    import argparse
    import json

    from . import binding, build as fbuild
    from .builder.__main__ import build_cached

    ap = argparse.ArgumentParser()
    ap.add_argument("--mix", default="ex1:4096:1e-7:1e-6,ex1:16384:1e-7:1e-6,ex3:64:1e-4:1e-3,ex3:128:1e-4:1e-3")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--load", type=float, default=0.7, help="offered load as a fraction of capacity")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--seed", type=int, default=2105_02995 + 4000)
    ap.add_argument("--mode", default="apply", choices=["apply", "solve"])
    a = ap.parse_args(argv)
    fbuild.build()
    prec = {"fp32": binding.FIO_P32, "tf32": binding.FIO_PTF32, "bf16": binding.FIO_PBF16,
            "tf32x3": binding.FIO_PTF32X3}[a.precision]
    ops = {}
    for spec in a.mix.split(","):
        kind, n, eb, eh = spec.split(":")
        buf, _ = build_cached(kind, int(n), float(eb), float(eh), gpu=True, verbose=False)
        ops[f"{kind}_{n}"] = binding.Operator(buf)
    srv = Server(ops, precision=prec, mode=a.mode)
    srv.warmup()
    # capacity probe: back-to-back batches of 32 on every operator
    probe = poisson_requests(ops, 4 * len(ops), 1e9, a.seed, b_range=(32, 32))
    cap = srv.run(probe).summary()["rhs_per_s"]
    rate = a.load * cap / 32.5  # requests per second (mean 32.5 right-hand sides each)
    reqs = poisson_requests(ops, a.requests, rate, a.seed)
    stats = srv.run(reqs)
    srv.close()
    out = {"mix": sorted(ops), "mode": a.mode, "precision": a.precision, "capacity_rhs_per_s": cap,
           "offered_requests_per_s": rate, **stats.summary()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
