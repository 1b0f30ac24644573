"""Edge cases of the solve on the GPU against the oracle: the smallest
problem (N = 2), a single sequence, many copies of one sequence (the
0.8-identity weights make them count as one: B_eff = 1, Eq.
inverse_weights2), a column that is gap in every sequence, and a run
stopped by max_iter.

Bar: the strong-convexity bound of the other solve tests (each site problem
is mu-strongly convex, mu = 2 min(lambda_h, lambda'_J)) with the oracle's
FP64 gradient norms at both points.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = 21
LH, LJ = 0.01, 0.01
MU = 2 * min(LH, 0.5 * LJ)


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_4832_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def _check(S, h_g, J_g, gtol_o=1e-7):
    N = S.shape[1]
    m, w, w32, beff = oracle.reweight(S, 0.8)
    h_o, J_o, info = oracle.solve(S, w, beff, LH, LJ, gtol=gtol_o)
    h_g = h_g.cpu().numpy().astype(np.float64)
    J_g = J_g.cpu().numpy().astype(np.float64)
    for r in range(N):
        _, gh, gJ = oracle.site_objgrad(S, w, beff, r, h_g[r], J_g[r], LH, 0.5 * LJ)
        gn = math.sqrt((gh ** 2).sum() + (gJ ** 2).sum())
        d = np.linalg.norm(np.concatenate([h_g[r] - h_o[r], (J_g[r] - J_o[r]).ravel()]))
        assert d <= (gn + info["gnorm"][r]) / MU * (1 + 1e-6) + 1e-9, (r, d, gn)
        assert not J_g[r, :, r, :].any()
    return beff


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
@pytest.mark.parametrize("case", ["N2", "one_sequence", "copies", "gap_column"])
def test_solve_edge_cases(ctx, prec, case):
    from paper_1401_4832_gb300 import api
    if case == "N2":
        S = synth.small_random(2, 50, 31, gap_p=0.1)
    elif case == "one_sequence":
        S = synth.small_random(10, 1, 32)
    elif case == "copies":
        S = np.repeat(synth.small_random(10, 1, 32), 200, axis=0)
    else:
        S = synth.small_random(12, 150, 33, gap_p=0.1)
        S[:, 4] = 0
    h, J, rep = api.plm_solve(ctx, torch.from_numpy(np.ascontiguousarray(S)).cuda(), gtol=1e-5,
                              prec=prec)
    assert rep["n_converged"] == S.shape[1], rep
    beff = _check(S, h, J)
    if case == "copies":
        assert beff == pytest.approx(1.0, rel=1e-12)


def test_copies_equal_one_sequence(ctx):
    # B_eff = 1 from 200 copies: the same objective as the single sequence,
    # so the same minimiser (up to FP32 rounding of the weights' sums)
    from paper_1401_4832_gb300 import api
    one = synth.small_random(10, 1, 32)
    many = np.repeat(one, 200, axis=0)
    h1, J1, _ = api.plm_solve(ctx, torch.from_numpy(one).cuda(), gtol=1e-6, prec="fp32")
    h2, J2, _ = api.plm_solve(ctx, torch.from_numpy(many).cuda(), gtol=1e-6, prec="fp32")
    assert torch.allclose(J1, J2, atol=2e-4) and torch.allclose(h1, h2, atol=2e-4)


def test_max_iter_stops_and_reports(ctx):
    from paper_1401_4832_gb300 import api, _native
    S = torch.from_numpy(synth.tiny().msa).cuda()
    h, J, rep = api.plm_solve(ctx, S, gtol=1e-9, max_iter=2)
    assert rep["status"] == "PLM_ENOTCONV"
    assert rep["iters"] <= 2 and rep["n_converged"] == 0
    assert rep["n_failed"] + rep["n_noise"] == S.shape[1]
    with pytest.raises(_native.PlmError):
        api.plm_solve(ctx, S, gtol=1e-9, max_iter=2, raise_on_notconv=True)
