"""Chi-square statistics of the paper's two failing BigCrush tests (Sec. 4.2),
computed on the host from the counts that the GPU data reductions
(mtgp_gap_histogram, mtgp_hamming_pairs) return.

Test 35 (gap test, r = 25, alpha = 0, beta = 1/32): a value visits [0, 2^-b)
with probability p = 2^-b, independently, so a gap (the run of non-visits
before a visit) has length s with probability p (1 - p)^s; lengths >= t are
pooled.

Test 100 (Hamming-weight independence, r = 25, s = 5, L = 1200): under the
null hypothesis the L bits of a block are independent fair bits, so a block
weight is Binomial(L, 1/2) and the weights of the two blocks of a pair are
independent; the C x C table of weight classes then has cell probabilities
q_i q_j with q the class probabilities of Binomial(L, 1/2).
"""
import math

import numpy as np


def gap_probabilities(b: int, t: int) -> np.ndarray:
    """pi_s = p (1-p)^s for s < t and pi_t = (1-p)^t, p = 2^-b."""
    p = 2.0 ** -b
    s = np.arange(t, dtype=np.float64)
    return np.concatenate([p * (1.0 - p) ** s, [(1.0 - p) ** t]])


def binomial_class_probabilities(L: int, bounds) -> np.ndarray:
    """Probabilities of the weight classes [bounds[c-1], bounds[c]) of a
    Binomial(L, 1/2) weight (class c holds w with c bounds <= w), exact in
    rational arithmetic before the final division."""
    edges = [0] + [int(x) for x in bounds] + [L + 1]
    tot = 1 << L
    return np.array([sum(math.comb(L, w) for w in range(max(lo, 0), min(hi, L + 1))) / tot
                     for lo, hi in zip(edges[:-1], edges[1:])])


def _chi2_sf(x: float, df: int) -> float:
    from scipy.stats import chi2
    return float(chi2.sf(x, df))


def chi2_statistic(observed, probabilities):
    """Pearson chi-square of the counts against n * probabilities (n = total
    count); cells with zero expectation must have zero counts."""
    obs = np.asarray(observed, dtype=np.float64).ravel()
    prob = np.asarray(probabilities, dtype=np.float64).ravel()
    n = obs.sum()
    exp = n * prob
    keep = exp > 0
    if np.any(obs[~keep] > 0):
        return float("inf")
    return float(np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep]))


def gap_test(hist, b: int = 5) -> dict:
    """Chi-square of a gap-length histogram (t + 1 classes, df = t)."""
    hist = np.asarray(hist)
    t = hist.size - 1
    x = chi2_statistic(hist, gap_probabilities(b, t))
    return {"gaps": int(hist.sum()), "chi2": x, "df": t, "p_value": _chi2_sf(x, t)}


def hamming_test(table, L: int = 1200, bounds=()) -> dict:
    """Chi-square of the C x C table of successive block-weight classes
    against independent Binomial(L, 1/2) weights (df = C*C - 1)."""
    table = np.asarray(table)
    q = binomial_class_probabilities(L, bounds)
    x = chi2_statistic(table, np.outer(q, q))
    df = q.size * q.size - 1
    return {"pairs": int(table.sum()), "chi2": x, "df": df, "p_value": _chi2_sf(x, df)}


def default_hamming_bounds(L: int = 1200, classes: int = 4):
    """Class bounds at the Binomial(L, 1/2) quantiles k/classes (so the
    classes are about equally likely)."""
    cdf, acc, bounds = [], 0, []
    tot = 1 << L
    for w in range(L + 1):
        acc += math.comb(L, w)
        cdf.append(acc / tot)
    for k in range(1, classes):
        bounds.append(next(w for w in range(L + 1) if cdf[w] >= k / classes) + 1)
    return bounds
