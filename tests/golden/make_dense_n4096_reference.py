"""Writes the FP64 oracle's 100-EM-iteration fit of the dense N = 4096,
D = 32768 workload (K = 32 probes, CG tol 1e-5 with residual replacement every
50 iterations, seed 0; Algorithm 1 and Sec. 3.2) to a golden text file.

It calls only oracle/ and the seeded input generator.  The dictionary is the
one the GPU path applies (reading R12): --phi bf16 rounds Phi to BF16, --phi
f32 uses hi + lo, its two BF16 terms (the FP32 dictionary on the tensor
cores).  y is rounded to FP32 as the GPU path stores it.

    python tests/golden/make_dense_n4096_reference.py --phi bf16
    python tests/golden/make_dense_n4096_reference.py --phi f32

The output (tests/golden/dense_n4096_d32768_em100_<phi>.txt) holds the
per-EM-iteration CG counts, relative residuals and support sizes, the final
NRMSE of mu against the generating coefficients, and the final alpha_d on a
fixed sample of coordinates: every 16th coordinate and the 655 coordinates
of the generating support (at 100 EM iterations every coordinate is still
below the 1e6 support threshold, so the sample stands for the support).  It
takes about 50 minutes of FP64 work on 8 host cores.
"""
import argparse
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sbl  # noqa: E402
from paper_2202_12808_gb300 import datagen  # noqa: E402


def dictionary(Phi32, phi):
    hi = torch.from_numpy(Phi32).to(torch.bfloat16)
    if phi == "bf16":
        return hi.double().numpy()
    lo = (torch.from_numpy(Phi32) - hi.float()).to(torch.bfloat16)
    return hi.double().numpy() + lo.double().numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--phi", choices=["bf16", "f32"], required=True)
    ap.add_argument("--em", type=int, default=100)
    a = ap.parse_args()
    c = datagen.CONFIGS["dense-n4096-d32768"]
    pr = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], c["sigma"], 0)
    Phi = dictionary(pr.Phi, a.phi)
    y = pr.y.astype(np.float32).astype(np.float64)
    t0 = time.time()
    alpha, mu, s, st = sbl.cofem_dense(Phi, y, pr.beta, c["K"], a.em, c["cg_tol"],
                                       c["cg_max_iters"],
                                       resid_replace_every=c["resid_replace_every"], seed=0)
    sec = time.time() - t0
    sup = np.nonzero(alpha < 1e6)[0]
    sample = np.union1d(np.arange(0, len(alpha), 16), pr.support)
    out = os.path.join(HERE, "dense_n4096_d32768_em%d_%s.txt" % (a.em, a.phi))
    with open(out, "w") as f:
        f.write("# FP64 oracle (oracle/sbl.py cofem_dense, Algorithm 1, Sec. 3.2 CG) on the dense\n"
                "# workload N=4096 D=32768, 655 nonzeros, sigma 0.01 (beta 1e4), K=32, CG tol 1e-5,\n"
                "# U=400, residual replacement every 50, seed 0, %d EM iterations, Phi = %s.\n"
                "# Written by tests/golden/make_dense_n4096_reference.py (%.0f s).\n"
                % (a.em, "bf16(Phi)" if a.phi == "bf16" else "hi + lo (two BF16 terms)", sec))
        f.write("cg_iters " + " ".join(str(v) for v in st.cg_iters) + "\n")
        f.write("relres " + " ".join("%.6e" % v for v in st.relres) + "\n")
        f.write("support_counts " + " ".join(str(v) for v in st.support) + "\n")
        f.write("nrmse_mu_vs_truth %.10e\n" % (np.linalg.norm(mu - pr.z) / np.linalg.norm(pr.z)))
        f.write("support %d\n" % len(sup))
        f.write("alpha_sample %d\n" % len(sample))
        for d in sample:
            f.write("%d %.17g\n" % (d, alpha[d]))
    print("wrote", out, "in %.0f s" % sec)


if __name__ == "__main__":
    main()
