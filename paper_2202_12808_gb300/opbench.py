"""Operator and CG-kernel micro-benchmark (a profiling aid).

Runs one hot-path kernel group of libcofem a fixed number of times on seeded
data, with CUDA-event timings, so that a profiler can capture its launches
outside any fit graph:

    python -m paper_2202_12808_gb300.opbench --op dense-bf16 --N 4096 --D 32768 --ncols 33
    python -m paper_2202_12808_gb300.opbench --op dense-f32  --N 4096 --D 32768 --ncols 33
    python -m paper_2202_12808_gb300.opbench --op cg --D 1048576 --ncols 33
    python -m paper_2202_12808_gb300.opbench --op bcg --D 32768 --ncols 33
    python -m paper_2202_12808_gb300.opbench --op conv-tc --L 1048576 --C 8 --T 64 --ncols 17

dense-bf16 / dense-f32 / dense-fp8: A X = beta Phi^T (Phi X) + alpha . X on
the tensor cores (BF16 dictionary, FP32 dictionary as hi + lo, or FP8 E4M3
with per-tile scales expanded to BF16 in shared memory), packed layout,
pipeline autotuned unless --no-autotune; prints the per-kernel microseconds
of cofem_op_apply_timed.  cg: the CG update (direction fused where it fits),
the direction update and the diagonal estimate + M-step
(cofem_bench_cg_kernels).  bcg: the three passes of one block-CG iteration
(cofem_bench_bcg_kernels).  conv-tc / conv-f32: A X of the circular
convolutional dictionary with the products on the tensor cores (BF16
filters) or the CUDA cores (FP32 filters); prints the forward and adjoint
microseconds.
"""
import argparse
import json

import numpy as np
import torch

from . import api
from . import binding as B


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["dense-bf16", "dense-f32", "dense-fp8", "cg", "bcg", "conv-tc",
                                     "conv-f32"], required=True)
    ap.add_argument("--L", type=int, default=1 << 20)
    ap.add_argument("--C", type=int, default=8)
    ap.add_argument("--T", type=int, default=64)
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--D", type=int, default=32768)
    ap.add_argument("--ncols", type=int, default=33)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--pipeline", default=None,
                    help="STAGES,CTAS_PER_SM of the tensor-core products (skips the autotuner)")
    ap.add_argument("--tile-rows", type=int, default=128, choices=[128, 256],
                    help="output rows per tensor-core work unit (with --pipeline)")
    a = ap.parse_args()
    st = torch.cuda.current_stream().cuda_stream
    if a.op == "bcg":
        nb = B.cofem_bench_bcg_kernels_workspace_bytes(a.D, a.ncols)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        ms = B.cofem_bench_bcg_kernels(a.D, a.ncols, a.reps, ws.data_ptr(), nb, st)
        print(json.dumps({"op": "bcg", "D": a.D, "ncols": a.ncols, "xi_us": ms[0] * 1e3,
                          "v_us": ms[1] * 1e3, "row_us": ms[2] * 1e3, "sequence_us": ms[3] * 1e3}))
        return
    if a.op == "cg":
        nb = B.cofem_bench_cg_kernels_workspace_bytes(a.D, a.ncols)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        ms = B.cofem_bench_cg_kernels(a.D, a.ncols, a.reps, ws.data_ptr(), nb, st)
        print(json.dumps({"op": "cg", "D": a.D, "ncols": a.ncols, "update_us": ms[0] * 1e3,
                          "direction_us": ms[1] * 1e3, "mstep_us": ms[2] * 1e3,
                          "update_holds_direction": ms[3] > 0.5}))
        return
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    if a.op in ("conv-tc", "conv-f32"):
        h = torch.randn((a.C, a.T), generator=g, device="cuda") / float(np.sqrt(a.T))
        op = api.ConvOperator(h, a.L, tensor_cores=a.op == "conv-tc")
        D = a.C * a.L
        X = torch.randn((a.ncols, D), generator=g, device="cuda")
        Y = torch.empty_like(X)
        alpha = torch.rand(D, generator=g, device="cuda", dtype=torch.float64) + 1.0
        nb = B.cofem_apply_workspace_bytes(op.handle, B.COFEM_F32, a.ncols)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        runs = [B.cofem_op_apply_timed(op.handle, B.COFEM_F32, X.data_ptr(), D, a.ncols,
                                       alpha.data_ptr(), 400.0, Y.data_ptr(), ws.data_ptr(), nb)
                for _ in range(a.reps + 1)][1:]
        print(json.dumps({"op": a.op, "L": a.L, "C": a.C, "T": a.T, "ncols": a.ncols,
                          "forward_us": float(np.mean([r[-2] for r in runs])) * 1e3,
                          "adjoint_us": float(np.mean([r[-1] for r in runs])) * 1e3}))
        return
    Phi = torch.randn((a.N, a.D), generator=g, device="cuda") / float(np.sqrt(a.N))
    if a.op == "dense-fp8":
        op = api.Fp8DenseOperator(Phi)             # quantised, packed copy attached
        del Phi
    else:
        if a.op == "dense-bf16":
            Phi = Phi.to(torch.bfloat16)
        op = api.DenseOperator(Phi)
        nbp = B.cofem_op_dense_packed_bytes(op.handle)
        packed = torch.empty(nbp, dtype=torch.uint8, device="cuda")
        B.cofem_op_dense_attach_packed(op.handle, packed.data_ptr(), nbp, st)
    tuned = None
    if a.pipeline:
        stg, cps = (int(v) for v in a.pipeline.split(","))
        B.cofem_op_dense_set_pipeline(op.handle, stg, cps)
        B.cofem_op_dense_set_tile_rows(op.handle, a.tile_rows)
        tuned = (stg, cps, a.tile_rows)
    elif not a.no_autotune:
        nbt = B.cofem_op_dense_autotune_workspace_bytes(op.handle, a.ncols)
        wst = torch.empty(nbt, dtype=torch.uint8, device="cuda")
        tuned = B.cofem_op_dense_autotune(op.handle, a.ncols, wst.data_ptr(), nbt, st)
        tuned = tuned + (B.cofem_op_dense_get_pipeline(op.handle)[2],)
        del wst
    ld = (a.D + 63) // 64 * 64
    X = torch.zeros((a.ncols, ld), device="cuda")
    X[:, :a.D] = torch.randn((a.ncols, a.D), generator=g, device="cuda")
    Y = torch.empty_like(X)
    alpha = torch.rand(a.D, generator=g, device="cuda", dtype=torch.float64) + 0.5
    nb = B.cofem_apply_workspace_bytes(op.handle, B.COFEM_F32, a.ncols)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    per = [B.cofem_op_apply_timed(op.handle, B.COFEM_F32, X.data_ptr(), ld, a.ncols,
                                  alpha.data_ptr(), 1e4, Y.data_ptr(), ws.data_ptr(), nb, st)
           for _ in range(a.reps)]
    kus = [float(np.mean([p[i] for p in per[1:] or per])) * 1e3 for i in range(len(per[0]))]
    print(json.dumps({"op": a.op, "N": a.N, "D": a.D, "ncols": a.ncols, "pipeline": tuned,
                      "kernels_us": kus}))


if __name__ == "__main__":
    main()
