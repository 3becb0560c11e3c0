"""Time-to-target (oracle side), section "Results" / Table 1. Test infrastructure only.

The target is 99.9 % of the lowest energy found (read for negative QUBO
energies as E_target = E_best + 0.001 |E_best|); TTT is the time to reach it
with 99 % probability.  With p_s(k) the probability that one run has reached
E_target at checkpoint k and t(k) the time of one run to that checkpoint,
the repetition count gives
  TTT(k) = t(k) max(1, ln(1 - 0.99) / ln(1 - p_s(k)))   (t(k) once p_s >= 0.99),
and TTT = min_k TTT(k); no k with p_s > 0 means "not reached" (None).
A run of R independent replicas reaches the target when any replica does:
p_run = 1 - (1 - p_rep)^R (``p_batch``).
"""
import math


def target_energy(e_best, frac=0.999):
    return e_best + (1.0 - frac) * abs(e_best)


def ttt_at(t_run, p_s, prob=0.99):
    if p_s <= 0.0:
        return math.inf
    if p_s >= prob:
        return t_run
    return t_run * math.log(1.0 - prob) / math.log(1.0 - p_s)


def p_batch(p_rep, R):
    """Success probability of a run of R independent replicas."""
    return 1.0 - (1.0 - p_rep) ** R


def ttt(times, energies, e_target, prob=0.99, replicas_per_run=1):
    """``times[k]`` seconds of one run to checkpoint k, ``energies[k]`` the
    energies of the sampled replicas there (p_rep = fraction at or below the
    target); a run holds ``replicas_per_run`` replicas."""
    best = math.inf
    for t, es in zip(times, energies):
        es = list(es)
        p = sum(1 for e in es if e <= e_target) / len(es) if es else 0.0
        best = min(best, ttt_at(t, p_batch(p, replicas_per_run), prob))
    return None if best == math.inf else best
