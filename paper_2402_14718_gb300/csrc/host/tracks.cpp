// Track finding and scoring: last paragraph of section "QUBO Generation and
// Track Finding" and Eq. 18-19 (efficiency = TP / (TP + FN), purity =
// TP / (TP + FP), counted on doublets).
#include <algorithm>
#include <map>
#include <set>
#include <utility>
#include <vector>

#include "host_internal.h"
#include "../guard.h"

extern "C" sb_status sb_tracks(const sb_event* ev, const sb_qubo* q, const uint8_t* T,
                               int32_t min_hits, int32_t* n_tracks, int32_t* track_ptr,
                               int32_t* track_hits, int64_t* counts, double* eff_pur) {
  return sbh::guarded("sb_tracks", [&]() -> sb_status {
    if (!ev || !q || (!T && q->n > 0)) {
      sbh::set_error("sb_tracks: null argument");
      return SB_ERR_ARG;
    }
    typedef std::pair<int32_t, int32_t> D;
    // selected triplets -> doublets, duplicates merged
    std::set<D> sel;
    for (int32_t i = 0; i < q->n; ++i)
      if (T[i]) {
        const int32_t a = q->trip[3 * (size_t)i], b = q->trip[3 * (size_t)i + 1],
                      c = q->trip[3 * (size_t)i + 2];
        sel.insert(D(a, b));
        sel.insert(D(b, c));
      }
    // unresolved conflicts: a hit with > 1 outgoing or > 1 incoming doublet loses them all
    std::map<int32_t, int32_t> n_out, n_in;
    for (const D& d : sel) {
      n_out[d.first]++;
      n_in[d.second]++;
    }
    std::map<int32_t, int32_t> nxt;
    std::set<int32_t> has_in;
    for (const D& d : sel)
      if (n_out[d.first] == 1 && n_in[d.second] == 1) {
        nxt[d.first] = d.second;
        has_in.insert(d.second);
      }
    // chain into candidates, ordered by first hit; drop those with < min_hits hits
    std::vector<std::vector<int32_t>> tracks;
    for (const auto& kv : nxt) {
      if (has_in.count(kv.first)) continue;
      std::vector<int32_t> path(1, kv.first);
      for (auto it = nxt.find(path.back()); it != nxt.end(); it = nxt.find(path.back()))
        path.push_back(it->second);
      if ((int32_t)path.size() >= min_hits) tracks.push_back(path);
    }
    std::set<D> reco;
    for (const auto& t : tracks)
      for (size_t k = 0; k + 1 < t.size(); ++k) reco.insert(D(t[k], t[k + 1]));
    // truth: consecutive-layer hit pairs of every particle
    std::map<int32_t, std::vector<int32_t>> by_part;
    for (int32_t h = 0; h < (int32_t)ev->particle.size(); ++h)
      if (ev->particle[h] >= 0) by_part[ev->particle[h]].push_back(h);
    std::set<D> truth;
    for (auto& kv : by_part) {
      std::vector<int32_t>& hs = kv.second;
      std::stable_sort(hs.begin(), hs.end(),
                       [&](int32_t u, int32_t v) { return ev->layer[u] < ev->layer[v]; });
      for (size_t k = 0; k + 1 < hs.size(); ++k)
        if (ev->layer[hs[k + 1]] == ev->layer[hs[k]] + 1) truth.insert(D(hs[k], hs[k + 1]));
    }
    int64_t tp = 0;
    for (const D& d : reco) tp += truth.count(d);
    const int64_t fp = (int64_t)reco.size() - tp, fn = (int64_t)truth.size() - tp;
    if (n_tracks) *n_tracks = (int32_t)tracks.size();
    if (track_ptr) {
      track_ptr[0] = 0;
      for (size_t k = 0; k < tracks.size(); ++k)
        track_ptr[k + 1] = track_ptr[k] + (int32_t)tracks[k].size();
    }
    if (track_hits) {
      size_t o = 0;
      for (const auto& t : tracks)
        for (int32_t h : t) track_hits[o++] = h;
    }
    if (counts) {
      counts[0] = tp;
      counts[1] = fp;
      counts[2] = fn;
    }
    if (eff_pur) {
      eff_pur[0] = (tp + fn) ? (double)tp / (double)(tp + fn) : 0.0;
      eff_pur[1] = (tp + fp) ? (double)tp / (double)(tp + fp) : 0.0;
    }
    return SB_OK;
  });
}
