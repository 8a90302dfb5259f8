"""The mapping objective of Sec. 3.1 on rendered maps -- TEST INFRASTRUCTURE
(same rules as the rest of ``oracle``: only tests, smoke and the benchmark's
CPU leg use it; it shares no code with the CUDA path).

Written from the paper's definitions, in float64, per pixel, no fusion:

* geometry and colour (Sec. 3.1, the objective after Eq. 1): pixels whose
  silhouette exceeds 0.99 contribute the L1 error of depth plus 0.5 times
  the L1 error of colour (summed over the three channels); the pixel terms
  are summed;
* semantics (Sec. 3.1 "Semantic Loss", Eq. 4 and Eq. 5): for the target
  distribution Q (pseudo ground truth) and the rendered distribution P of a
  pixel, the entropy mask M_H = [H(Q) < ln k] with H(Q) = -sum_m Q_m ln Q_m
  (0 ln 0 = 0), the Hellinger distance D_HD = sqrt(0.5 sum_m (sqrt Q_m -
  sqrt P_m)^2) and the cosine similarity cos = Q.P / (|Q| |P|); the pixel
  term M_H (0.8 D_HD + 0.2 (1 - cos)) is averaged over the pixels.

Readings where the paper is silent: the colour L1 sums
its channels; the semantic term is a mean over pixels while the geometric
one is a sum, as printed; the two are added; P_m < 0 counts as 0 under the
square root (weights are not constrained in the optimisation); the square
roots use sqrt(x + 1e-12) for both distributions, so that the derivative
stays finite at P_m = 0 and identical distributions are at distance exactly
0; zero norms give cos = 0 and a zero cosine gradient; a zero Hellinger
distance gives a zero Hellinger gradient (the distance is a cone there: no
derivative exists).

Parity: the loss is pinned by closed forms (identical, disjoint and uniform
distributions, the silhouette threshold) and the gradient by central finite
differences of the loss itself (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

SIL_MIN = 0.99          # silhouette threshold of the geometric term
W_COLOUR = 0.5          # colour weight of the geometric term
LAM_HD, LAM_COS = 0.8, 0.2
EPS_SQRT = 1e-12        # inside sqrt(P_m + eps)
EPS_DIV = 1e-12         # floor of denominators


def semantic_terms(q: np.ndarray, p: np.ndarray, k: int):
    """Per-pixel semantic loss terms and their gradient with respect to P.
    q, p: [..., M].  Returns (term [...], dterm/dP [..., M])."""
    q = np.asarray(q, np.float64)
    p = np.asarray(p, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        qlogq = np.where(q > 0, q * np.log(np.where(q > 0, q, 1.0)), 0.0)
    h = -qlogq.sum(-1)
    mask = (h < np.log(k)).astype(np.float64)
    pc = np.maximum(p, 0.0)
    sp = np.sqrt(pc + EPS_SQRT)
    sq = np.sqrt(np.maximum(q, 0.0) + EPS_SQRT)
    d_hd = np.sqrt(0.5 * ((sq - sp) ** 2).sum(-1))
    nq = np.sqrt((q * q).sum(-1))
    npn = np.sqrt((p * p).sum(-1))
    dot = (q * p).sum(-1)
    den = nq * npn
    cos = np.where(den > EPS_DIV, dot / np.maximum(den, EPS_DIV), 0.0)
    term = mask * (LAM_HD * d_hd + LAM_COS * (1.0 - cos))
    # d D_HD / d P_m = 0.5 * (sqrt(P_m) - sqrt(Q_m)) / sqrt(P_m) / (2 D_HD), P_m > 0 branch
    dhd = np.where((d_hd > EPS_DIV)[..., None] & (p >= 0),
                   (sp - sq) / (2.0 * sp) / (2.0 * np.maximum(d_hd, EPS_DIV))[..., None], 0.0)
    dcos = np.where((den > EPS_DIV)[..., None],
                    q / np.maximum(den, EPS_DIV)[..., None]
                    - (cos / np.maximum(npn * npn, EPS_DIV))[..., None] * p, 0.0)
    grad = mask[..., None] * (LAM_HD * dhd - LAM_COS * dcos)
    return term, grad


def mapping_loss(rgb, depth, sil, sem, t_rgb, t_depth, t_sem, k: int):
    """Loss of the mapping step on rendered maps rgb [H,W,3], depth [H,W],
    sil [H,W], sem [H,W,M] against targets, and its gradients with respect
    to rgb, depth and sem (the silhouette enters only through the mask:
    zero gradient).  Returns (loss, d_rgb, d_depth, d_sem) in float64."""
    rgb = np.asarray(rgb, np.float64)
    depth = np.asarray(depth, np.float64)
    sil = np.asarray(sil, np.float64)
    t_rgb = np.asarray(t_rgb, np.float64)
    t_depth = np.asarray(t_depth, np.float64)
    mg = (sil > SIL_MIN).astype(np.float64)
    e_d = depth - t_depth
    e_c = rgb - t_rgb
    loss_geo = (mg * (np.abs(e_d) + W_COLOUR * np.abs(e_c).sum(-1))).sum()
    d_depth = mg * np.sign(e_d)
    d_rgb = W_COLOUR * mg[..., None] * np.sign(e_c)
    npix = depth.size
    term, g = semantic_terms(t_sem, sem, k)
    loss = loss_geo + term.sum() / npix
    d_sem = g / npix
    return float(loss), d_rgb, d_depth, d_sem
