"""Error bounds the reduced-precision parity tests use (no GPU needed).

Strong convexity (mu = 2 min(lambda_h, lambda'_J)) bounds each site's
distance to its unique minimiser by ||grad g_r|| / mu.  The Ising gauge is an
orthogonal projection and the average halves, so the Frobenius score of a
pair moves by at most

    b_ij = (||g_i|| + ||g_j|| + ||g_i*|| + ||g_j*||) / (2 mu)

between two solutions whose gradient norms are g and g* (Eqs. gauge_change2,
average2, frob_normtrans2).  The APC score (Eq. corr_norm2)

    CFN_ij = FN_ij - r_i r_j / t,   r_i = mean_{j != i} FN_ij,  t = mean FN

then moves by at most b_ij plus the largest change of r_i r_j / t over the
box r_i +- rb_i, r_j +- rb_j, t +- tb (rb, tb the same means of b): the
correction is increasing in r_i and r_j and decreasing in t, so its extremes
sit at two corners of the box.
"""
import numpy as np


def fn_bound(gn_a, gn_b, mu):
    """b_ij for per-site gradient norms of two solutions (arrays of N)."""
    gn_a = np.asarray(gn_a, np.float64)
    gn_b = np.asarray(gn_b, np.float64)
    b = (gn_a[:, None] + gn_a[None, :] + gn_b[:, None] + gn_b[None, :]) / (2.0 * mu)
    np.fill_diagonal(b, 0.0)
    return b


def _off_diag_means(M):
    N = M.shape[0]
    off = M.copy()
    np.fill_diagonal(off, 0.0)
    return off.sum(1) / (N - 1), off.sum() / (N * (N - 1))


def cfn_bound(fn, b):
    """Bound on |CFN' - CFN| for any FN' with |FN'_ij - FN_ij| <= b_ij."""
    r, t = _off_diag_means(fn)
    rb, tb = _off_diag_means(b)
    base = np.outer(r, r) / t
    hi = np.outer(r + rb, r + rb) / max(t - tb, 1e-300)
    lo = np.outer(np.maximum(r - rb, 0.0), np.maximum(r - rb, 0.0)) / (t + tb)
    e = b + np.maximum(hi - base, base - lo)
    if t - tb <= 0.0:
        e[:] = np.inf  # the bound says nothing when the mean FN may vanish
    np.fill_diagonal(e, 0.0)
    return e


def compare_top(top_g, top_o, cfn_o, e):
    """Compare two top-L lists (rows (i, j), best first) of the same length.

    Returns (identical, within_bound, detail): identical when the lists are
    equal; within_bound when every pair in only one list scores (by the
    reference's CFN) within e_p + e_last of the reference's last pair, and
    every out-of-order neighbour pair of top_g is within e_p + e_q."""
    top_g = np.asarray(top_g).reshape(-1, 2)
    top_o = np.asarray(top_o).reshape(-1, 2)
    if np.array_equal(top_g, top_o):
        return True, True, "identical"
    a = set(map(tuple, top_g.tolist()))
    o = set(map(tuple, top_o.tolist()))
    last = tuple(top_o[-1])
    bad = []
    for p in a ^ o:
        if abs(cfn_o[p] - cfn_o[last]) > e[p] + e[last]:
            bad.append(("set", p, float(cfn_o[p] - cfn_o[last]), float(e[p] + e[last])))
    sg = [cfn_o[tuple(p)] for p in top_g]
    for k in range(len(top_g) - 1):
        p, q = tuple(top_g[k]), tuple(top_g[k + 1])
        if sg[k + 1] - sg[k] > e[p] + e[q]:
            bad.append(("order", p, q, float(sg[k + 1] - sg[k])))
    detail = f"{len(a ^ o) // 2} boundary swaps, sets {'equal' if a == o else 'differ'}"
    return False, not bad, detail if not bad else f"{detail}; outside the bound: {bad[:5]}"
