"""Instance segmentation quality (§IV, Segmentation Results) of labels against per-pixel
ground-truth instance ids: the mean IoU of the matched instances and the precision at
IoU thresholds.

For every ground-truth instance with at least ``min_points`` measurements, the cluster
with the largest overlap is its match and the Jaccard index of the two point sets is its
IoU.  When one cluster is the match of several instances, only the instance with the
highest IoU keeps it; the others count as not found (IoU 0).  IoU_mu is the mean over the
instances; P_x is the fraction of instances matched with IoU >= x; P_mu is the mean of
P_x over x = 0.50, 0.55, ..., 0.95.

Host-side numpy over labels already copied back (the metric is evaluation, not part of
the labelling path).
"""
from __future__ import annotations

import numpy as np

THRESHOLDS = tuple(round(0.5 + 0.05 * i, 2) for i in range(10))


def instance_ious(labels, gt, min_points: int = 100) -> dict:
    """{instance id: IoU} for the instances of ``gt`` (ids >= 1; 0 and below are ground or
    background) with at least ``min_points`` pixels; ``labels`` are cluster ids (>= 0) or
    -1 for unsegmented pixels."""
    lab = np.asarray(labels).reshape(-1).astype(np.int64)
    g = np.asarray(gt).reshape(-1).astype(np.int64)
    if lab.shape != g.shape:
        raise ValueError("labels and ground truth must have the same size")
    ids, sizes = np.unique(g[g >= 1], return_counts=True)
    inst = ids[sizes >= min_points]
    if inst.size == 0:
        return {}
    # cluster sizes and the overlap table of (instance, cluster) pairs
    clus, csize = np.unique(lab[lab >= 0], return_counts=True)
    cluster_size = dict(zip(clus.tolist(), csize.tolist()))
    inst_size = dict(zip(ids.tolist(), sizes.tolist()))
    both = np.isin(g, inst) & (lab >= 0)
    pairs, counts = np.unique(np.stack([g[both], lab[both]]), axis=1, return_counts=True)
    best = {}  # instance -> (overlap, -cluster) of its largest overlap, lowest cluster on ties
    for (i, c), n in zip(pairs.T.tolist(), counts.tolist()):
        key = (n, -c)
        if i not in best or key > best[i]:
            best[i] = key
    iou = {}
    owner = {}  # cluster -> instance keeping it
    for i in inst.tolist():
        if i not in best:
            iou[i] = 0.0
            continue
        n, negc = best[i]
        c = -negc
        iou[i] = n / (inst_size[i] + cluster_size[c] - n)
        j = owner.get(c)
        if j is None or iou[i] > iou[j] or (iou[i] == iou[j] and i < j):
            if j is not None:
                iou[j] = 0.0
            owner[c] = i
        else:
            iou[i] = 0.0
    return iou


def scores(labels, gt, min_points: int = 100) -> dict:
    """{"instances", "iou_mu", "p_50", "p_75", "p_95", "p_mu"} of one or many frames (pass
    lists of arrays to pool the instances of several frames, as the paper pools its
    sequences)."""
    if isinstance(labels, (list, tuple)):
        vals = []
        for lab, g in zip(labels, gt):
            vals += list(instance_ious(lab, g, min_points).values())
    else:
        vals = list(instance_ious(labels, gt, min_points).values())
    v = np.asarray(vals, np.float64)
    if v.size == 0:
        return {"instances": 0}
    p = {x: float((v >= x - 1e-12).mean()) for x in THRESHOLDS}
    return {"instances": int(v.size), "iou_mu": round(float(v.mean()), 4),
            "p_50": round(p[0.5], 4), "p_75": round(p[0.75], 4), "p_95": round(p[0.95], 4),
            "p_mu": round(float(np.mean(list(p.values()))), 4)}
