"""Synthetic one-stage benchmark of the stage kernels (for tuning and profiling them).

    python -m paper_2105_02995_gb300.stagebench [--nblk 1024] [--rows 512] [--cols 512]
        [--b 8,32,64] [--prec fp32,tf32,bf16] [--variants 0] [--reps 5]

Builds a packed operator whose first butterfly-type stage holds nblk random dense complex blocks
of rows x cols with random gather and scatter permutations (a second stage of 16 x 16 identity
blocks closes the chain), uploads it through the C ABI and times that first stage of apply_K
with fio_apply_profiled (CUDA events around the launch), for each precision, batch width and kernel variant (fio_set_variant; 0 = the built-in choice).
Prints one JSON object: per configuration the median time, the stage's complex flops rate
(8 b entries / t) and the rate at which its factor entries are streamed (entry bytes / t).
No method arithmetic is involved: the blocks are random.
"""

from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nblk", type=int, default=1024)
    ap.add_argument("--rows", type=int, default=512)
    ap.add_argument("--cols", type=int, default=512)
    ap.add_argument("--b", default="8,32,64")
    ap.add_argument("--prec", default="fp32,tf32,bf16")
    ap.add_argument("--variants", default="0", help="kernel variants to pin (fio_set_variant)")
    ap.add_argument("--dirs", default="fwd", help="fwd (the stage in apply_K) and/or adj (in apply_Kadj)")
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args(argv)
    import torch

    from . import binding, build as fbuild
    from .builder.pack import pack
    from .builder.stages import KIND_MAP, Stage

    fbuild.build()
    nblk, R, C = a.nblk, a.rows, a.cols
    if R != C:
        raise SystemExit("rows must equal cols (the closing stage maps the output back to N)")
    N = nblk * C
    rng = np.random.default_rng(0)
    pin, pout = rng.permutation(N), rng.permutation(nblk * R)
    M = (rng.standard_normal((R, C)) + 1j * rng.standard_normal((R, C))) / np.sqrt(C)
    s1 = Stage(KIND_MAP, N, nblk * R)
    for i in range(nblk):
        s1.add(M, pin[i * C:(i + 1) * C], pout[i * R:(i + 1) * R])
    s2 = Stage(KIND_MAP, nblk * R, N)
    eye = np.eye(16)
    for i in range(nblk * R // 16):
        s2.add(eye, np.arange(16 * i, 16 * i + 16), np.arange(16 * i, 16 * i + 16))
    op = binding.Operator(pack(1, N, [s1, s2], [], [], 0.0, 0.0))
    precs = {"fp32": binding.FIO_P32, "tf32": binding.FIO_PTF32, "bf16": binding.FIO_PBF16,
             "tf32x3": binding.FIO_PTF32X3}
    out = {"nblk": nblk, "rows": R, "cols": C}
    for b in [int(v) for v in a.b.split(",")]:
        x = binding.colmajor(torch.randn(N, b, dtype=torch.complex64, device="cuda"))
        y = binding.colmajor(torch.empty_like(x))
        for name in a.prec.split(","):
            p = precs[name]
            for var in [int(v) for v in a.variants.split(",")]:
                try:
                    op.set_variant(b, p, var)
                except binding.FioError:
                    continue  # no such variant for this precision and batch
                for d in a.dirs.split(","):
                    # launch groups with b >= 5: apply_K [layout, stage 1, stage 2],
                    # apply_Kadj [layout, stage 2 adjoint, stage 1 adjoint]
                    which, grp = ("K", 1) if d == "fwd" else ("Kadj", 2)
                    for _ in range(2):
                        op.apply_profiled(which, x, y, precision=p)
                    ts = [op.apply_profiled(which, x, y, precision=p)[grp] for _ in range(a.reps)]
                    ms = float(np.median(ts))
                    ent = nblk * R * C
                    tag = f"{name}_b{b}" + (f"_v{var}" if var else "") + ("" if d == "fwd" else "_adj")
                    out[tag] = {"ms": round(ms, 4), "tflops": round(8 * ent * b / ms / 1e9, 1),
                                "factor_gbs": round(ent * (4 if name == "bf16" else 8) / ms / 1e6, 1)}
            op.set_variant(b, p, 0)
    print(json.dumps(out))
    op.release()


if __name__ == "__main__":
    main()
