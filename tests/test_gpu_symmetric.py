"""GPU symmetric plmDCA (Sec. 3, Eq. npll_1 with the penalty of Eq. l2reg)
against the oracle's symmetric solve.

The problem l_pseudo + R_l2 is strongly convex in its parameters x = (h,
J_ij for i < j) with mu = 2 min(lambda_h, lambda_J), so for the GPU point
x_g and the oracle point x_o,
    ||x_g - x_o|| <= (||grad(x_g)|| + ||grad(x_o)||) / mu,
with both gradients evaluated by the oracle in FP64.  The GPU result must
also be exactly symmetric (J_ji = J_ij^T bit for bit) and give the oracle's
contact list.
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
MU = 2 * min(LH, LJ)


def _x(h, J):
    N = h.shape[0]
    parts = [h.ravel()]
    for i in range(N):
        for j in range(i + 1, N):
            parts.append(J[i, :, j, :].ravel())
    return np.concatenate(parts)


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_4832_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny_ref():
    S = synth.tiny().msa
    m, w, w32, beff = oracle.reweight(S, 0.8)
    ro = oracle.plmdca_symmetric(S, gtol=1e-7)
    return S, w, beff, ro


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_symmetric_solve_matches_oracle(ctx, tiny_ref, prec):
    from paper_1401_4832_gb300 import api
    S, w, beff, ro = tiny_ref
    N = S.shape[1]
    h_g, J_g, rep = api.plm_solve_symmetric(ctx, torch.from_numpy(S).cuda(), gtol=1e-5, prec=prec)
    assert rep["n_converged"] == N, rep
    h_g = h_g.cpu().numpy().astype(np.float64)
    J_g = J_g.cpu().numpy().astype(np.float64)
    for i in range(N):
        assert not J_g[i, :, i, :].any()
        for j in range(i + 1, N):
            assert np.array_equal(J_g[j, :, i, :], J_g[i, :, j, :].T)
    xg = _x(h_g, J_g)
    xo = ro["info"]["x"]
    _, gg = oracle.sym_objgrad(S, w, beff, xg, LH, LJ)
    _, go = oracle.sym_objgrad(S, w, beff, xo, LH, LJ)
    bound = (np.linalg.norm(gg) + np.linalg.norm(go)) / MU
    assert np.linalg.norm(xg - xo) <= bound * (1 + 1e-6), (np.linalg.norm(xg - xo), bound)
    assert np.linalg.norm(gg) <= 3e-5
    fn, cfn, top = api.fn_apc_scores(ctx, torch.from_numpy(J_g.astype(np.float32)).cuda())
    top_o = ro["top"]
    assert np.array_equal(top.cpu().numpy()[:len(top_o)], top_o)


def test_symmetric_family_size(ctx):
    # the family workload: converged, exactly symmetric, the stationarity
    # identities of Eq. symmetricgauge within the residual gradient
    from paper_1401_4832_gb300 import api
    S = synth.protein_family().msa
    N = S.shape[1]
    h_g, J_g, rep = api.plm_solve_symmetric(ctx, torch.from_numpy(S).cuda(), gtol=1e-4)
    assert rep["n_converged"] == N, rep
    h = h_g.cpu().numpy().astype(np.float64)
    J = J_g.cpu().numpy().astype(np.float64)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    _, g = oracle.sym_objgrad(S, w, beff, _x(h, J), LH, LJ)
    gn = np.linalg.norm(g)
    assert gn <= 3e-4, gn
    tol = math.sqrt(Q + 1) * gn / 2 + 1e-9
    for i in range(0, N, 7):
        for j in range(i + 1, N, 11):
            assert np.all(np.abs(LJ * J[i, :, j, :].sum(1) - LH * h[i]) <= tol)
