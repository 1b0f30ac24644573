"""The objective as a torch.autograd.Function, at the family workload
(N=120, B=5000): its hand-written adjoint against central differences of
the FP64 oracle objective (64 random coordinates, step 1e-4) and against the
oracle gradient.  FP32 couplings.

Tolerance: the FP32 path's gradient is within 1e-5 of max|g| (the bar of
the objective/gradient parity tests); central differences in FP64 add a
truncation error O(h^2 |g'''|) ~ 1e-8 and a rounding error ~1e-16 / 1e-4,
both far below it.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = 21


def test_autograd_adjoint_matches_fd_and_oracle():
    from paper_1401_4832_gb300.autograd import plm_objective
    from paper_1401_4832_gb300 import api
    fam = synth.protein_family()
    S = fam.msa
    B, N = S.shape
    m, w64, w32, beff = oracle.reweight(S, 0.8)
    rng = np.random.default_rng(42)
    h0 = rng.normal(0, 0.05, (N, Q)).astype(np.float32)
    J0 = rng.normal(0, 0.05, (N, Q, N, Q)).astype(np.float32)
    for r in range(N):
        J0[r, :, r, :] = 0
    h = torch.from_numpy(h0).cuda().requires_grad_(True)
    J = torch.from_numpy(J0).cuda().requires_grad_(True)
    Sd = torch.from_numpy(S).cuda()
    wd = torch.from_numpy(w32).cuda()
    # a scalar loss with a different weight per site exercises the chain rule
    site_w = torch.linspace(0.5, 1.5, N, dtype=torch.float64, device="cuda")
    f = plm_objective(h, J, Sd, wd, beff)
    loss = (f * site_w).sum()
    loss.backward()
    gh = h.grad.cpu().numpy().astype(np.float64)
    gJ = J.grad.cpu().numpy().astype(np.float64)
    sw = site_w.cpu().numpy()

    # oracle gradient (FP64), scaled the same way
    f_o, gh_o, gJ_o = oracle.objgrad(S, w64, beff, h0.astype(np.float64), J0.astype(np.float64))
    gh_o *= sw[:, None]
    gJ_o *= sw[:, None, None, None]
    assert np.max(np.abs(f.detach().cpu().numpy() - f_o) / f_o) <= 1e-6
    scale = max(np.abs(gh_o).max(), np.abs(gJ_o).max())
    assert np.max(np.abs(gh - gh_o)) <= 1e-5 * scale
    assert np.max(np.abs(gJ - gJ_o)) <= 1e-5 * scale

    # central differences of the FP64 oracle objective, 64 coordinates
    eps = 1e-4
    picks = []
    while len(picks) < 64:
        r, s, i, k = (int(rng.integers(0, N)), int(rng.integers(0, Q)),
                      int(rng.integers(0, N + 1)), int(rng.integers(0, Q)))
        if i == r:
            continue
        picks.append((r, s, i, k))  # i == N means the field h[r, s]
    for r, s, i, k in picks:
        hr = h0[r].astype(np.float64)
        Jr = J0[r].astype(np.float64)
        vals = []
        for sign in (+1, -1):
            hp, Jp = hr.copy(), Jr.copy()
            if i == N:
                hp[s] += sign * eps
            else:
                Jp[s, i, k] += sign * eps
            vals.append(oracle.site_objgrad(S, w64, beff, r, hp, Jp, 0.01, 0.005, grad=False))
        fd = sw[r] * (vals[0] - vals[1]) / (2 * eps)
        g = gh[r, s] if i == N else gJ[r, s, i, k]
        assert abs(g - fd) <= 1e-5 * scale + 1e-9, (r, s, i, k, g, fd)


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_objective_only_equals_objective_with_gradient(prec):
    # with no gradient asked for (torch.no_grad, or plm_site_objective_grad
    # with gh = gJ = NULL) the library runs the logits pass alone; the
    # objective is the same number as the full evaluation's
    from paper_1401_4832_gb300.autograd import plm_objective
    from paper_1401_4832_gb300 import api
    S = synth.add_clusters(synth.small_random(41, 600, 21), 0.3, 21, max_redraw=0.1)
    N = S.shape[1]
    m, w64, w32, beff = oracle.reweight(S, 0.8)
    rng = np.random.default_rng(3)
    h = torch.from_numpy(rng.normal(0, 0.1, (N, Q)).astype(np.float32)).cuda()
    J0 = rng.normal(0, 0.1, (N, Q, N, Q)).astype(np.float32)
    for r in range(N):
        J0[r, :, r, :] = 0
    J = torch.from_numpy(J0).cuda()
    Sd, wd = torch.from_numpy(S).cuda(), torch.from_numpy(w32).cuda()
    with api.Context(0) as c:
        f_full, gh, gJ = api.plm_site_objective_grad(c, Sd, wd, beff, h, J, prec=prec)
        f_only, gh0, gJ0 = api.plm_site_objective_grad(c, Sd, wd, beff, h, J, prec=prec, grad=False)
        assert gh0 is None and gJ0 is None
        assert torch.equal(f_full, f_only)
        with torch.no_grad():
            f_ng = plm_objective(h, J, Sd, wd, beff, prec=prec, plm_ctx=c)
        assert torch.equal(f_ng, f_full)
        # exactly one of the gradient outputs missing is an argument error
        from paper_1401_4832_gb300 import _native
        import ctypes
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        gh1 = torch.empty((N, Q), device="cuda")
        st = c.lib.plm_site_objective_grad(
            c.handle, ctypes.c_void_p(Sd.data_ptr()), ctypes.c_void_p(wd.data_ptr()), float(beff),
            S.shape[0], N, Q, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(J.data_ptr()),
            0.01, 0.01, _native.PRECISIONS[prec], ctypes.c_void_p(f.data_ptr()),
            ctypes.c_void_p(gh1.data_ptr()), None)
        assert st == _native.PLM_EINVAL
