"""Efficiency-aware pruning and scale decay, FP64 reference (TEST
INFRASTRUCTURE ONLY: only tests/ may import this module).

Definitions written out from the paper, Sec. 3.2 "Intersection-Aware
Pruning" and Sec. 3.3 "Scale Decay":

* CE_i = Val_i / Comp_i (Eq. 2).  Val_i = pixels dominated by point i (the
  point with the largest T_i alpha_i of the pixel), Comp_i = tiles that
  intersect and use the point.  Reading: Comp_i = tiles whose list holds the
  point (every such tile pays for it); points no tile holds have no CE in
  that pose.  The final CE is the maximum over the poses.
* Pruning removes a fraction of the points with the lowest CE (R = 10% per
  round, Sec. 3.4).  Reading: floor(fraction * N) points; ties in CE are
  removed lower point index first; points that never got a CE count as 0.
* WS = (1/N) sum_i S_i G_i (Eq. 3), G_i = (U_i > T) (U_i - T) (Eq. 4), with
  S_i the largest extent of the point's ellipsoid (reading: the largest of
  its three activated scales; the paper's constant factor of the span goes
  into the loss weight gamma) and U_i the tiles that use the point in
  rendering (reading: tiles where at least one pixel blended it).
  L = L_quality + gamma WS (Eq. 5): dL/ds_ik = gamma G_i / N for the first
  axis k holding the largest scale, 0 for the others (G_i does not depend
  on the scales at the current iterate).
"""
from __future__ import annotations

import numpy as np

STAT_TOUCHED, STAT_USED, STAT_BLENDED, STAT_DOMINATED = range(4)


def ce_of_pose(stats):
    """CE of one pose from a (4, N) statistics array; NaN where Comp = 0."""
    st = np.asarray(stats, np.float64)
    comp, val = st[STAT_TOUCHED], st[STAT_DOMINATED]
    out = np.full(comp.shape, np.nan)
    nz = comp > 0
    out[nz] = val[nz] / comp[nz]
    return out


def ce_max(poses_stats):
    """Maximum CE over poses (points never held by a tile: 0)."""
    ce = None
    for st in poses_stats:
        c = ce_of_pose(st)
        ce = c if ce is None else np.fmax(ce, c)
    return np.nan_to_num(ce, nan=0.0)


def prune_keep(ce, fraction):
    """keep[i] = False for the floor(fraction * N) lowest-CE points."""
    ce = np.asarray(ce, np.float64)
    n = len(ce)
    k = int(np.floor(fraction * n))
    order = np.lexsort((np.arange(n), ce))      # by CE, then by index
    keep = np.ones(n, bool)
    keep[order[:k]] = False
    return keep


def weighted_scale(scales, used, T):
    """WS of Eq. 3-4 and its gradient with respect to the (N, 3) scales."""
    s = np.asarray(scales, np.float64)
    u = np.asarray(used, np.float64)
    n = len(s)
    G = np.where(u > T, u - T, 0.0)
    S = s.max(axis=1)
    ws = float((S * G).sum() / n) if n else 0.0
    grad = np.zeros_like(s)
    if n:
        grad[np.arange(n), s.argmax(axis=1)] = G / n
    return ws, grad
