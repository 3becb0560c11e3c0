"""Time-to-target (oracle side), section "Results" / Table 1. Test infrastructure only.

The target is 99.9 % of the lowest energy found (read for negative QUBO
energies as E_target = E_best + 0.001 |E_best|); TTT is the time to reach it
with 99 % probability.  With p_s(k) the fraction of independent runs whose
energy after checkpoint k is <= E_target and t(k) the time of one run to that
checkpoint, the usual repetition count gives
  TTT(k) = t(k) ln(1 - 0.99) / ln(1 - p_s(k))   (TTT = t(k) when p_s = 1),
and TTT = min_k TTT(k); no k with p_s > 0 means "not reached" (None).
"""
import math


def target_energy(e_best, frac=0.999):
    return e_best + (1.0 - frac) * abs(e_best)


def ttt_at(t_run, p_s, prob=0.99):
    if p_s <= 0.0:
        return math.inf
    if p_s >= 1.0:
        return t_run
    return t_run * math.log(1.0 - prob) / math.log(1.0 - p_s)


def ttt(times, energies, e_target, prob=0.99):
    """``times[k]`` seconds to checkpoint k, ``energies[k]`` energies of the runs there."""
    best = math.inf
    for t, es in zip(times, energies):
        es = list(es)
        p = sum(1 for e in es if e <= e_target) / len(es) if es else 0.0
        best = min(best, ttt_at(t, p, prob))
    return None if best == math.inf else best
