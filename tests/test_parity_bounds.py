"""The CFN error bound and the top-L comparison the reduced-precision parity
tests use, checked on the CPU against the oracle's APC (Eq. corr_norm2)."""
import numpy as np

import oracle
from parity_bounds import cfn_bound, compare_top, fn_bound


def _sym(rng, N, lo, hi):
    M = rng.uniform(lo, hi, (N, N))
    M = np.triu(M, 1)
    return M + M.T


def test_cfn_bound_holds_for_perturbed_fn():
    rng = np.random.default_rng(0)
    for trial in range(20):
        N = int(rng.integers(6, 40))
        fn = _sym(rng, N, 0.05, 2.0)
        gn_a = rng.uniform(0, 2e-4, N)
        gn_b = rng.uniform(0, 1e-6, N)
        b = fn_bound(gn_a, gn_b, 0.01)
        e = cfn_bound(fn, b)
        cfn = oracle.apc(fn)
        for sign in (None, 1.0, -1.0):
            d = _sym(rng, N, -1.0, 1.0) if sign is None else sign * np.ones((N, N))
            fn2 = fn + np.clip(d, -1, 1) * b
            assert np.all(np.abs(oracle.apc(fn2) - cfn) <= e * (1 + 1e-12) + 1e-15)


def test_cfn_bound_is_not_vacuous():
    # with row means close to the overall mean the correction term moves by
    # about three times b (both row means and the mean), so e is about 4 b
    N = 10
    rng = np.random.default_rng(1)
    fn = _sym(rng, N, 0.9, 1.1)
    b = np.full((N, N), 1e-3)
    np.fill_diagonal(b, 0)
    e = cfn_bound(fn, b)
    off = ~np.eye(N, dtype=bool)
    assert np.all(e[off] <= 4.5 * b[off]) and np.all(e[off] >= b[off])


def test_compare_top_identical_tie_and_mismatch():
    N = 12
    cfn = np.zeros((N, N))
    vals = {(0, 5): 3.0, (1, 7): 2.0, (2, 8): 1.0, (3, 9): 0.999, (4, 10): 0.5}
    for p, v in vals.items():
        cfn[p] = cfn[p[::-1]] = v
    e = np.full((N, N), 0.01)
    top_o = np.array([(0, 5), (1, 7), (2, 8)])
    assert compare_top(top_o, top_o, cfn, e)[:2] == (True, True)
    # boundary swap inside the band: a tie, not a mismatch
    swap = np.array([(0, 5), (1, 7), (3, 9)])
    assert compare_top(swap, top_o, cfn, e)[:2] == (False, True)
    # a pair far below the boundary is a mismatch
    far = np.array([(0, 5), (1, 7), (4, 10)])
    assert compare_top(far, top_o, cfn, e)[1] is False
    # an order swap of distant scores is a mismatch
    order = np.array([(1, 7), (0, 5), (2, 8)])
    assert compare_top(order, top_o, cfn, e)[1] is False
