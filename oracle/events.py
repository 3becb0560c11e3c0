"""Synthetic barrel events (oracle side) -- stand-in for the TrackML events of
the paper's section "Dataset" (tt-bar + pile-up, barrel only, 10 layers, 2 T).

Test infrastructure only. Plain Python loops over ``math`` so every libm call
is the platform's scalar libm (the product's C++ generator calls the same
functions, in the same formula order, and must agree bit for bit).

Recipe (one event):
* tracks: charge q = +-1 (p = 1/2), 1/pT ~ U[0.1, 1] GeV^-1, eta ~ U(-1, 1),
  phi0 ~ U[0, 2 pi), vertex (0, 0, z0) with z0 ~ N(0, 5 mm);
* helix in a uniform field B = 2 T along z: transverse radius
  Rc [mm] = 1000 pT / (0.3 B); on a barrel cylinder of radius r the hit sits at
  phi = phi0 - q asin(r / 2Rc) and z = z0 + 2 Rc asin(r / 2Rc) sinh(eta);
* 10 cylinders at r = 32, 72, 116, 172, 260, 360, 500, 660, 820, 1000 mm
  (unbounded in z, so every track leaves one hit per layer);
* Gaussian smear of r*phi and z by 0.1 mm each (Box-Muller);
* noise: floor(f * n_true + 0.5) hits, layer uniform, phi ~ U[-pi, pi),
  z ~ U[zmin_l, zmax_l] (the z range of the true hits on that layer);
* hits sorted by (layer, phi, generation index); generation index of a true
  hit is track * 10 + layer, of noise hit k it is n_true + k.

Random numbers: Philox4x32-10 keyed by the seed; counter =
(object, variate, purpose, 0).
"""
import math
from dataclasses import dataclass, field

from .philox import draw, PURPOSE_TRACK, PURPOSE_NOISE

LAYER_RADII = (32.0, 72.0, 116.0, 172.0, 260.0, 360.0, 500.0, 660.0, 820.0, 1000.0)
TWO_PI = 2.0 * math.pi


@dataclass
class EventParams:
    n_tracks: int = 100
    noise_frac: float = 0.1
    bz: float = 2.0               # tesla
    inv_pt_min: float = 0.1       # GeV^-1
    inv_pt_max: float = 1.0
    eta_max: float = 1.0
    z0_sigma: float = 5.0         # mm
    smear_rphi: float = 0.1       # mm
    smear_z: float = 0.1          # mm
    radii: tuple = field(default=LAYER_RADII)


@dataclass
class Event:
    layer: list      # int per hit
    r: list          # float per hit (the layer radius)
    phi: list        # float per hit, in [-pi, pi)
    z: list          # float per hit
    x: list          # r cos(phi)
    y: list          # r sin(phi)
    particle: list   # track index, -1 for noise
    n_true: int
    truth: list = None   # per track: (q, pT, eta, phi0, z0, Rc)


def wrap_phi(phi):
    """Map an angle to [-pi, pi): phi - 2 pi floor((phi + pi) / 2 pi)."""
    return phi - TWO_PI * math.floor((phi + math.pi) / TWO_PI)


def gauss(seed, purpose, obj, var):
    """Standard normal by Box-Muller from one Philox block."""
    u1, u2 = draw(seed, purpose, obj, var)
    return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(TWO_PI * u2)


def generate(seed, p: EventParams = EventParams()):
    """Generate one event; returns an ``Event`` with hits in sorted order."""
    nl = len(p.radii)
    raw = []  # (layer, phi, z, particle, gen)
    truth = []
    for t in range(p.n_tracks):
        uq, _ = draw(seed, PURPOSE_TRACK, t, 0)
        q = 1.0 if uq < 0.5 else -1.0
        ui, _ = draw(seed, PURPOSE_TRACK, t, 1)
        inv_pt = p.inv_pt_min + (p.inv_pt_max - p.inv_pt_min) * ui
        ue, _ = draw(seed, PURPOSE_TRACK, t, 2)
        eta = -p.eta_max + 2.0 * p.eta_max * ue
        up, _ = draw(seed, PURPOSE_TRACK, t, 3)
        phi0 = TWO_PI * up
        z0 = p.z0_sigma * gauss(seed, PURPOSE_TRACK, t, 4)
        pt = 1.0 / inv_pt
        rc = (1000.0 * pt) / (0.3 * p.bz)
        sh = math.sinh(eta)
        truth.append((q, pt, eta, phi0, z0, rc))
        for l in range(nl):
            r = p.radii[l]
            a = math.asin(r / (2.0 * rc))
            phi = phi0 - q * a
            z = z0 + (2.0 * rc * a) * sh
            phi = phi + (p.smear_rphi * gauss(seed, PURPOSE_TRACK, t, 5 + l)) / r
            z = z + p.smear_z * gauss(seed, PURPOSE_TRACK, t, 5 + nl + l)
            raw.append((l, wrap_phi(phi), z, t, t * nl + l))
    n_true = len(raw)
    zmin = [math.inf] * nl
    zmax = [-math.inf] * nl
    for (l, _, z, _, _) in raw:
        zmin[l] = min(zmin[l], z)
        zmax[l] = max(zmax[l], z)
    n_noise = int(math.floor(p.noise_frac * n_true + 0.5)) if n_true else 0
    for k in range(n_noise):
        ul, _ = draw(seed, PURPOSE_NOISE, k, 0)
        l = min(int(math.floor(ul * nl)), nl - 1)
        up, _ = draw(seed, PURPOSE_NOISE, k, 1)
        phi = -math.pi + TWO_PI * up
        uz, _ = draw(seed, PURPOSE_NOISE, k, 2)
        z = zmin[l] + (zmax[l] - zmin[l]) * uz
        raw.append((l, wrap_phi(phi), z, -1, n_true + k))
    raw.sort(key=lambda h: (h[0], h[1], h[4]))
    ev = Event([], [], [], [], [], [], [], n_true, truth)
    for (l, phi, z, part, _) in raw:
        r = p.radii[l]
        ev.layer.append(l)
        ev.r.append(r)
        ev.phi.append(phi)
        ev.z.append(z)
        ev.x.append(r * math.cos(phi))
        ev.y.append(r * math.sin(phi))
        ev.particle.append(part)
    return ev
