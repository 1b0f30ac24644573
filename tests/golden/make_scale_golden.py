"""Write the FP64 oracle's rundown of the scale workload's 2000-row
subsample (N=500, q=21) to ``scale_subsample_N500_B2000.npz``.

Every stored value comes from ``oracle/`` alone: the oracle reweights the
subsample, solves all 500 site problems from the origin with L-BFGS to
||grad g_r|| <= 1e-6 and scores the result (Ising gauge, average, FN, APC,
top-L over pairs with j - i >= 5).  The input is the synthetic scale family
(N=500, B=50000, 750 planted chain contacts, 20 % gaps, 20 Gibbs sweeps), of
which 2000 rows are drawn without replacement with seed 1; the subsample
itself is stored too, so that the GPU test reads the very MSA the oracle
solved whatever machine regenerates the family.

Run from the repository root:  python tests/golden/make_scale_golden.py
(about 20 minutes on 8 host cores).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1401_4832_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scale_subsample_N500_B2000.npz")
GTOL = 1e-6


def main():
    t0 = time.time()
    fam = synth.scale_family(sweeps=20)
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(fam.B, 2000, replace=False))
    S = np.ascontiguousarray(fam.msa[rows])
    res = oracle.plmdca(S, gtol=GTOL)
    N = S.shape[1]
    iu = np.triu_indices(N, 1)
    info = res["info"]
    np.savez_compressed(
        OUT, msa=S, rows=rows.astype(np.int32),
        fn_upper=res["fn"][iu].astype(np.float32),
        cfn_upper=res["cfn"][iu].astype(np.float32),
        gnorm=info["gnorm"], iters=info["iters"].astype(np.int32),
        top=res["top"].astype(np.int32), gtol=np.float64(GTOL),
        threads=np.int32(oracle.num_threads()))
    print(f"wrote {OUT}: max gnorm {info['gnorm'].max():.3g}, "
          f"{time.time() - t0:.0f} s on {oracle.num_threads()} threads")


if __name__ == "__main__":
    main()
