"""Named synthetic workloads (numbers only; no arithmetic of the method).

Each entry fixes the event recipe (tracks, noise fraction, seed), the builder
cuts and the SB run shape. The cut values are one family scaled by a looseness
factor s: dphi_slope = 4e-4 s rad/mm, dphi_margin = 0.5 s mm, z0_max = 50 s mm,
kappa_max = 8e-4 s mm^-1, dtheta_max = 0.1 s rad (s = 1 is the printed Eq. 16
cut read in mm^-1), with the quadruplet curvature cut dkappa_max = 5e-4 mm^-1.
s is chosen per workload so the QUBO size matches the workload's stated N.
"""


def _cuts(dphi_slope, dphi_margin, z0_max, kappa_max, dtheta_max, dkappa_max=5e-4):
    return dict(dphi_slope=dphi_slope, dphi_margin=dphi_margin, z0_max=z0_max,
                kappa_max=kappa_max, dtheta_max=dtheta_max, dkappa_max=dkappa_max,
                w_q=1.0, w_c=1.0, five_hit_rule=1)


# s = 8: 100 tracks -> N ~ 1.7k
CUTS_S8 = _cuts(3.2e-3, 4.0, 400.0, 6.4e-3, 0.8)
# s = 2.35: 1000 tracks -> N ~ 40k
CUTS_S2_35 = _cuts(9.4e-4, 1.175, 117.5, 1.88e-3, 0.235)
# s = 2.8: 500 tracks -> N ~ 10k
CUTS_S2_8 = _cuts(1.12e-3, 1.4, 140.0, 2.24e-3, 0.28)
# s = 1.6: the batch of uneven events (N ~ 0.4k - 92k per event)
CUTS_S1_6 = _cuts(6.4e-4, 0.8, 80.0, 1.28e-3, 0.16)
# paper values of Eq. 16 / 17 read in mm^-1 (s = 1, dkappa = 1e-4)
CUTS_PAPER = _cuts(4e-4, 0.5, 50.0, 8e-4, 0.1, 1e-4)
# dense pile-up events: windows at the track resolution (dtheta of a true
# triplet is < 0.003 rad at 0.1 mm smear); 10k tracks -> N ~ 0.47M, ~21M couplings
CUTS_DENSE = _cuts(3.5e-4, 0.3, 25.0, 8e-4, 0.04)

# the pile-up event at N ~ 1M: windows between the dense preset and the printed
# cuts; 10k tracks + 20 % noise -> N = 1.03M, 109M couplings (106 per row)
CUTS_PILEUP_1M = _cuts(4.4e-4, 0.44, 34.0, 8e-4, 0.057)

WORKLOADS = {
    # plain bSB / dSB on one small event, FP32 J, one replica
    "event100": dict(n_tracks=100, noise_frac=0.1, seed=0, cuts=CUTS_S8,
                     replicas=1, steps=2000, dt=0.5, a0=1.0, jprec="fp32"),
    # replica-parallel run on one dense event, BF16 J
    "event1000": dict(n_tracks=1000, noise_frac=0.1, seed=1000, cuts=CUTS_S2_35,
                      replicas=256, steps=4000, dt=0.5, a0=1.0, jprec="bf16"),
    # adjoint workload
    "event500": dict(n_tracks=500, noise_frac=0.1, seed=3000, cuts=CUTS_S2_8,
                     replicas=32, steps=1000, dt=0.5, a0=1.0, jprec="fp32"),
    # high pile-up event
    "event10k": dict(n_tracks=10000, noise_frac=0.2, seed=4000, cuts=CUTS_DENSE,
                     replicas=128, steps=5000, dt=0.5, a0=1.0, jprec="bf16"),
    # the same event at the stated N ~ 1M (looser cuts)
    "event10k_1m": dict(n_tracks=10000, noise_frac=0.2, seed=4000, cuts=CUTS_PILEUP_1M,
                        replicas=128, steps=5000, dt=0.5, a0=1.0, jprec="bf16"),
}

# 512 uneven events in one context: event e has BATCH512_TRACKS[e] tracks
# (log-uniform in [50, 2000], drawn once from numpy's PCG64 with seed 2000) and
# event seed 2000 + e; 10 % noise; dSB, 64 replicas, 2000 steps.
BATCH512 = dict(n_events=512, tracks_min=50, tracks_max=2000, track_seed=2000, seed0=2000,
                noise_frac=0.1, cuts=CUTS_S1_6, replicas=64, steps=2000, dt=0.5, a0=1.0,
                variant="dsb", jprec="bf16")


def batch512_tracks():
    import math

    import numpy as np
    rng = np.random.default_rng(BATCH512["track_seed"])
    u = rng.uniform(math.log(BATCH512["tracks_min"]), math.log(BATCH512["tracks_max"]),
                    BATCH512["n_events"])
    return [int(v) for v in np.round(np.exp(u))]


# Events whose QUBO sizes match the four examples of the paper's Fig. 2 / Fig. 4
# (778, 10,295, 67,570, 109,498 triplets): every synthetic track crosses all ten
# layers, so the sizes are matched by track count under the dense-event cuts.
PAPER_SIZES = [
    dict(paper_N=778, n_tracks=95, seed=5095),
    dict(paper_N=10295, n_tracks=1064, seed=6064),
    dict(paper_N=67570, n_tracks=4133, seed=9133),
    dict(paper_N=109498, n_tracks=5406, seed=10406),
]
