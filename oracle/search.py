"""Brute-force parameter search (Sec. 4): the best parameter gives the fewest
preconditioned FGMRES iterations to a 1e8 reduction of the residual; ties
go to the smallest convergence factor, the geometric mean of the residual
reduction factors over the last 10 iterations; a tie range containing 1.0
selects 1.0."""
import numpy as np

from . import cycle, krylov


def convergence_factor(history, last=10):
    h = np.asarray(history)
    k = min(last, h.size - 1)
    if k <= 0:
        return 0.0
    return float((h[-1] / h[-1 - k]) ** (1.0 / k))


def search(prob, make_params, values, restart=30, maxit=200, reduction=1e-8):
    """Try each value; return (best value, table of (value, its, factor))."""
    table = []
    for v in values:
        o = cycle.Oracle(prob, make_params(v))
        hist = []
        _, its, rr = krylov.fgmres(prob.K[0], prob.b, o.apply, rtol=reduction,
                                   restart=restart, maxit=maxit, history=hist)
        if rr > reduction:
            its = maxit + 1
        table.append((v, its, convergence_factor(hist)))
    best_its = min(t[1] for t in table)
    tied = [t for t in table if t[1] == best_its]
    if any(abs(t[0] - 1.0) < 1e-12 for t in tied):
        return 1.0, table
    best = min(tied, key=lambda t: t[2])
    return best[0], table
