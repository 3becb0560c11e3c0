"""Track finding and scoring (oracle side): section "QUBO Generation and Track
Finding" (last paragraph) and Eq. 18-19. Test infrastructure only.

* selected triplets -> their two doublets (a,b) and (b,c); duplicates merged;
* unresolved conflicts (reading): a hit with more than one selected outgoing
  doublet, or more than one selected incoming doublet, loses all of them;
* the remaining doublets are chained into track candidates; candidates with
  fewer than four hits are dropped;
* a reconstructed doublet is true when both hits come from one particle
  (doublets always join consecutive layers); the true doublets are the
  consecutive-layer hit pairs of every generated particle;
  efficiency = TP / (TP + FN) (Eq. 18), purity = TP / (TP + FP) (Eq. 19).
"""


def doublets_of(q, T):
    out = set()
    for i in range(q.n):
        if T[i]:
            a, b, c = (int(v) for v in q.trip[i])
            out.add((a, b))
            out.add((b, c))
    return out


def resolve_conflicts(doublets):
    n_out = {}
    n_in = {}
    for (u, v) in doublets:
        n_out[u] = n_out.get(u, 0) + 1
        n_in[v] = n_in.get(v, 0) + 1
    return {(u, v) for (u, v) in doublets if n_out[u] == 1 and n_in[v] == 1}


def chain(doublets, min_hits=4):
    """Track candidates (lists of hit ids) ordered by their first hit."""
    nxt = {u: v for (u, v) in doublets}
    has_in = {v for (_, v) in doublets}
    tracks = []
    for start in sorted(nxt):
        if start in has_in:
            continue
        path = [start]
        while path[-1] in nxt:
            path.append(nxt[path[-1]])
        if len(path) >= min_hits:
            tracks.append(path)
    return tracks


def assemble(q, T, min_hits=4):
    """Selected triplets -> (tracks, reconstructed doublets on kept tracks)."""
    d = resolve_conflicts(doublets_of(q, T))
    tracks = chain(d, min_hits)
    reco = set()
    for t in tracks:
        for k in range(len(t) - 1):
            reco.add((t[k], t[k + 1]))
    return tracks, reco


def true_doublets(ev):
    by_part = {}
    for h, part in enumerate(ev.particle):
        if part >= 0:
            by_part.setdefault(part, []).append(h)
    out = set()
    for hits in by_part.values():
        hits = sorted(hits, key=lambda h: ev.layer[h])
        for k in range(len(hits) - 1):
            if ev.layer[hits[k + 1]] == ev.layer[hits[k]] + 1:
                out.add((hits[k], hits[k + 1]))
    return out


def score(ev, reco):
    """(TP, FP, FN, efficiency, purity); an empty denominator gives 0."""
    truth = true_doublets(ev)
    tp = len(reco & truth)
    fp = len(reco) - tp
    fn = len(truth) - tp
    eff = tp / (tp + fn) if tp + fn else 0.0
    pur = tp / (tp + fp) if tp + fp else 0.0
    return tp, fp, fn, eff, pur
