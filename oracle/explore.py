"""Candidate scoring and generation of Sec. 3.2 -- TEST INFRASTRUCTURE (same
rules as the rest of ``oracle``: only tests, smoke and the benchmark's CPU
leg use it; it shares no code with the product).

Written from the paper's definitions, in float64, one candidate at a time:

* Eq. 6: I_geo = softmax over candidates of log N_S (log 0 = -inf, whose
  exponential is 0);
* Eq. 7: I_sem = softmax over candidates of the per-view entropy sum;
* Eq. 8: I = (1 - softmax(l)) I_geo I_sem with l the Euclidean distance from
  the candidate's position to the current camera position;
* the pool's pruning rule: a candidate whose N_S is below 0.5 % of its
  pixels is dropped ("Exploration Strategy");
* viewing directions: the n-point Fibonacci lattice on the unit sphere
  (heights 1 - (2i + 1)/n, azimuth i times the golden angle pi (3 - sqrt 5));
* positions: the lattice points of spacing v1 over newly freed voxels, at
  the sampled heights.

Readings where the paper is silent: the softmaxes run
over the candidates scored together; when no candidate has N_S > 0 the
geometric factor is 0 for all (the softmax of all -inf is undefined); the
best candidate is the largest I among the kept ones, the lowest index on
ties; a camera looking along d has rows right = d x z (normalised),
down = d x right, forward = d.

Parity: pinned by closed forms (softmax of log N equals N / sum N, uniform
factors for equal inputs, a hand-evaluated three-candidate case, the pruning
boundary) and by properties of the lattice and the poses
(tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np

PRUNE_FRAC = 0.005


def softmax(x: np.ndarray) -> np.ndarray:
    """exp(x_v) / sum_u exp(x_u), evaluated with the maximum subtracted;
    -inf entries give 0; all -inf gives NaN (caller decides)."""
    x = np.asarray(x, np.float64)
    mx = np.max(x)
    if not np.isfinite(mx):
        return np.full_like(x, np.nan)
    e = np.exp(x - mx)
    return e / e.sum()


def score(sums: np.ndarray, npix: np.ndarray, positions: np.ndarray, current: np.ndarray,
          prune_frac: float = PRUNE_FRAC):
    """sums [V, 3] = (sum U, sum H, N_S) per candidate; npix [V]; positions
    [V, 3]; current [3].  Returns (scores [V, 4] = (I, I_geo, I_sem,
    1 - softmax(l)), keep [V] bool, best index or -1)."""
    sums = np.asarray(sums, np.float64)
    ns, sh = sums[:, 2], sums[:, 1]
    with np.errstate(divide="ignore"):
        igeo = softmax(np.log(ns))
    if np.isnan(igeo).any():
        igeo = np.zeros_like(ns)
    isem = softmax(sh)
    dist = np.linalg.norm(np.asarray(positions, np.float64) - np.asarray(current, np.float64), axis=1)
    mov = 1.0 - softmax(dist)
    iv = mov * igeo * isem
    keep = ns >= prune_frac * np.asarray(npix, np.float64)
    best = -1
    for v in range(len(iv)):
        if keep[v] and (best < 0 or iv[v] > iv[best]):
            best = v
    return np.stack([iv, igeo, isem, mov], axis=1), keep, best


def fibonacci_directions(n: int) -> np.ndarray:
    """[n, 3] unit vectors of the n-point Fibonacci lattice on the sphere."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def look_along(position, d) -> np.ndarray:
    """3x4 world-to-camera [R|t] of a camera at `position` looking along the
    unit vector d (OpenCV axes, world z up)."""
    d = np.asarray(d, np.float64)
    up = np.array([0.0, 0.0, 1.0]) if abs(d[2]) <= 1.0 - 1e-6 else np.array([0.0, 1.0, 0.0])
    right = np.cross(d, up)
    right /= np.linalg.norm(right)
    down = np.cross(d, right)
    r = np.stack([right, down, d])
    return np.concatenate([r, (-r @ np.asarray(position, np.float64))[:, None]], axis=1)


def candidate_positions(centres: np.ndarray, step: float, heights, band: float) -> np.ndarray:
    """Distinct lattice points (round(x/step) step, round(y/step) step, h) of
    the voxel centres within `band` of a height h, ascending (i, j, h index)."""
    step = float(np.float32(step))  # the sizes as the float32 arguments hold them
    band = float(np.float32(band))
    hs = [float(np.float32(h)) for h in heights]
    pts = set()
    for x, y, z in np.asarray(centres, np.float32).astype(np.float64).reshape(-1, 3):
        for hi, h in enumerate(hs):
            if abs(z - h) <= band:
                pts.add((math.floor(x / step + 0.5), math.floor(y / step + 0.5), hi))
    out = [(i * step, j * step, hs[hi]) for i, j, hi in sorted(pts)]
    return np.asarray(out, np.float64).reshape(-1, 3)
