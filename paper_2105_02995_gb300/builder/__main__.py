"""Command-line factor builder: builds one operator and writes its packed buffer to a file.

    python -m paper_2105_02995_gb300.builder --kind ex3 --n 256 --eps-bf 1e-4 --eps-hif 1e-3 \
        --out /tmp/op.fio [--gpu]

The builder's inner loops run on a thread pool with single-threaded BLAS (builder/blas.py); a
separate process keeps the bench process free of the build's memory and threads, and the result
is cached on disk (build_cached).
--gpu makes the peeling probes use libfio's butterfly apply on the current GPU.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)


def source_hash() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(HERE)):
        if name.endswith(".py"):
            with open(os.path.join(HERE, name), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def cache_dir() -> str:
    d = os.environ.get("FIO_CACHE", os.path.join("/tmp", "fio_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def build_cached(kind, n, eps_bf, eps_hif, gpu=False, threads=None, verbose=True, hif_rescale=False,
                 butterfly_only=False):
    """Build (or reuse) an operator in a subprocess with single-threaded BLAS; returns (bytes, info).
    butterfly_only: K-dot alone (no peeling, no HIF; e.g. the tight operator of a refinement's
    residual)."""
    key = (f"{kind}_{n}_{eps_bf:g}_{eps_hif:g}{'_resc' if hif_rescale else ''}{'_bf' if butterfly_only else ''}"
           f"_{source_hash()}")
    path = os.path.join(cache_dir(), key + ".fio")
    meta = path + ".json"
    if not (os.path.exists(path) and os.path.exists(meta)):
        env = dict(os.environ)
        env["FIO_BUILD_THREADS"] = str(threads or os.cpu_count() or 1)
        env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
        cmd = [sys.executable, "-m", "paper_2105_02995_gb300.builder", "--kind", kind, "--n", str(n),
               "--eps-bf", repr(eps_bf), "--eps-hif", repr(eps_hif), "--out", path]
        if gpu:
            cmd.append("--gpu")
        if hif_rescale:
            cmd.append("--hif-rescale")
        if butterfly_only:
            cmd.append("--butterfly-only")
        # the build's progress goes to stderr: stdout of the caller stays free for its own output
        out = sys.stderr if verbose else subprocess.PIPE
        r = subprocess.run(cmd, env=env, stdout=out, stderr=out, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"factor build failed ({r.returncode}): {r.stderr if not verbose else ''}")
    with open(path, "rb") as fh:
        buf = fh.read()
    with open(meta) as fh:
        info = json.load(fh)
    return buf, info


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", required=True)
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--eps-bf", type=float, required=True)
    ap.add_argument("--eps-hif", type=float, required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--gpu", action="store_true")
    ap.add_argument("--hif-rescale", action="store_true", help="Cholesky-rescaled HIF skeletonization")
    ap.add_argument("--butterfly-only", action="store_true", help="K-dot alone: no peeling, no HIF")
    a = ap.parse_args(argv)
    sys.path.insert(0, ROOT)
    from paper_2105_02995_gb300.builder import build_butterfly_only, build_operator
    if a.butterfly_only:
        t = time.time()
        buf, bf = build_butterfly_only(a.kind, a.n, a.eps_bf)
        info = {"kind": a.kind, "n": a.n, "t_bf": time.time() - t, "t_peel": 0.0, "t_hif": 0.0,
                "t_total": time.time() - t, "root": 0, "nnz_bf": int(sum(sum(M.size for M, _, _ in st.blocks) for st in bf)),
                "nnz_hif": 0, "nbytes": len(buf), "butterfly_only": True, "eps_bf": a.eps_bf}
        tmp = a.out + ".tmp"
        with open(tmp, "wb") as fh:
            fh.write(buf)
        with open(a.out + ".json", "w") as fh:
            json.dump(info, fh, default=str)
        os.replace(tmp, a.out)
        print(json.dumps(info), flush=True)
        return
    mv = None
    if a.gpu:
        from paper_2105_02995_gb300 import binding, build as fbuild
        fbuild.build()
        prec = binding.FIO_P32 if a.eps_hif >= 1e-4 else binding.FIO_P64
        mv = binding.NormalMatvecGPU(prec)
    t = time.time()
    buf, info = build_operator(a.kind, a.n, a.eps_bf, a.eps_hif, mv=mv, verbose=True, hif_rescale=a.hif_rescale)
    info["t_total"] = time.time() - t
    info["peel_on_gpu"] = bool(a.gpu)
    tmp = a.out + ".tmp"
    with open(tmp, "wb") as fh:
        fh.write(buf)
    with open(a.out + ".json", "w") as fh:
        json.dump({k: v for k, v in info.items()}, fh, default=str)
    os.replace(tmp, a.out)
    print(json.dumps({k: info[k] for k in ("kind", "n", "t_bf", "t_peel", "t_hif", "t_total", "root",
                                              "nnz_bf", "nnz_hif", "nbytes")}), flush=True)


if __name__ == "__main__":
    main()
