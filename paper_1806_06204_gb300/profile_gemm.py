"""Time one building-block GEMM of libzolo: C = op(A) op(B) in FP64 (DFMA) or
split precision (nine BF16, eight FP16 or eleven FP8 slices on the tensor cores),
through zolo_dgemm.

    python -m paper_1806_06204_gb300.profile_gemm --m 4096 --n 4096 --k 4096 --prec split

Seeded N(0,1) operands; `--reps` timed calls after one warm-up call, timed with
CUDA events on the current stream.  `--tune-cache F`: the FP64 kernel comes
from the tuning file F when it holds this shape; otherwise the warm-up call
measures the candidates (zolo_autotune) and F is written with the choice.  Prints one JSON line: milliseconds per
call, FP64-equivalent TFLOP/s (2MNK per call), and for the split path the BF16
tensor TFLOP/s actually issued (53, 36 or 76 slice-pair products; FP8 at twice
the rate).  Also the launch
target for kernel profilers: each call is one row-exponent + slicing pass per
operand and one GEMM kernel (split), or one GEMM kernel (FP64).
"""
import argparse
import json

import torch

from . import build


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--prec", choices=["fp64", "split"], default="split")
    ap.add_argument("--slices", choices=["bf16", "fp16", "fp8"], default="bf16")
    ap.add_argument("--transA", action="store_true")
    ap.add_argument("--transB", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune-cache", default=None)
    args = ap.parse_args()
    build.build()
    from . import binding as zb

    g = torch.Generator(device="cuda").manual_seed(5000)
    shape_a = (args.k, args.m) if args.transA else (args.m, args.k)
    shape_b = (args.n, args.k) if args.transB else (args.k, args.n)
    A = torch.randn(shape_a[::-1], dtype=torch.float64, device="cuda", generator=g).t()
    B = torch.randn(shape_b[::-1], dtype=torch.float64, device="cuda", generator=g).t()
    C = zb.empty_colmajor(args.m, args.n)
    prec = ({"bf16": zb.ZOLO_SPLIT_BF16, "fp16": zb.ZOLO_SPLIT_FP16,
             "fp8": zb.ZOLO_SPLIT_FP8}[args.slices] if args.prec == "split" else zb.ZOLO_FP64)
    h = zb.Handle(torch.cuda.current_device())
    if args.tune_cache:
        import os
        if os.path.exists(args.tune_cache) and zb.tune_load(h, args.tune_cache) != 0:
            raise SystemExit(f"tuning cache {args.tune_cache} refused")
        zb.autotune(h, True)

    def call():
        zb.zolo_dgemm(h, A, B, C, transA=args.transA, transB=args.transB, prec=prec,
                      slices={"bf16": 9, "fp16": 8, "fp8": 11}[args.slices])

    call()
    torch.cuda.synchronize()
    kernel = None
    if args.tune_cache:
        zb.autotune(h, False)
        zb.tune_save(h, args.tune_cache)
        names = {0: "64x64", 1: "32x128", 2: "32x64", 3: "64x64 split-K 2", 4: "64x64 split-K 4",
                 5: "64x64 split-K 8", 8: "split"}
        for line in open(args.tune_cache).read().splitlines():
            f = line.split()
            if f[0] == "g" and [int(x) for x in f[1:4]] == [args.m, args.n, args.k]:
                kernel = names.get(int(f[-1]), f[-1])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    flops = 2.0 * args.m * args.n * args.k
    out = {"m": args.m, "n": args.n, "k": args.k, "prec": args.prec, "ms_per_call": ms,
           "fp64_equiv_tflops": flops / ms / 1e9}
    if args.prec == "split":
        # slice-pair products issued: 53 (nine BF16 slices), 36 (eight FP16
        # slices), 76 (eleven FP8 slices, whose peak is twice the 16-bit one)
        pairs = {"bf16": 53, "fp16": 36, "fp8": 76}[args.slices]
        out["slices"] = args.slices
        out["tensor_issued_tflops"] = pairs * flops / ms / 1e9
    if kernel:
        out["tuned_kernel"] = kernel
    ref = A @ B if not (args.transA or args.transB) else None
    if ref is not None:
        out["max_rel_err_vs_cublas"] = float((C - ref).abs().max() / ref.abs().max())
    print(json.dumps(out), flush=True)
    h.close()


if __name__ == "__main__":
    main()
