"""Write the FP64 oracle's symmetric plmDCA rundown of the family workload
(N=120, B=5000, q=21) to ``symmetric_family_N120_B5000.npz``.

Every stored value comes from ``oracle/`` alone: the oracle reweights the
family, minimises l_pseudo + R_l2 (Eq. npll_1 with the penalty of Eq. l2reg)
over x = (h, J_ij for i < j) from the origin with L-BFGS to
||grad|| <= 1e-6, and scores the tied couplings (Ising gauge, FN, APC,
top-L over pairs with j - i >= 5).  The family's MSA is stored too, so that
the GPU test solves the very alignment the oracle solved.

Run from the repository root:  python tests/golden/make_symmetric_golden.py
(about two minutes on 8 host cores).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1401_4832_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "symmetric_family_N120_B5000.npz")
GTOL = 1e-6


def main():
    t0 = time.time()
    S = synth.protein_family().msa
    res = oracle.plmdca_symmetric(S, gtol=GTOL)
    N = S.shape[1]
    iu = np.triu_indices(N, 1)
    info = res["info"]
    np.savez_compressed(
        OUT, msa=S, fn_upper=res["fn"][iu].astype(np.float32),
        cfn_upper=res["cfn"][iu].astype(np.float32), gnorm=np.float64(info["gnorm"]),
        f=np.float64(info["f"]), iters=np.int32(info["iters"]), top=res["top"].astype(np.int32),
        gtol=np.float64(GTOL))
    print(f"wrote {OUT}: gnorm {info['gnorm']:.3g}, {time.time() - t0:.0f} s on "
          f"{oracle.num_threads()} threads")


if __name__ == "__main__":
    main()
