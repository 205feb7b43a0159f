"""Map quality metrics of the FP64 oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module; the product package never does, and the two
share no code.

What it follows (Liu et al., 2024, Sec. IV-B.1, "Evaluation Metrics"): the
map's mesh vertices form a point cloud M, compared with a ground-truth cloud
G; with d(p, X) = min(2 nu, |p - q|), q the point of X nearest p,
  RE  = sqrt(mean over p in M of d(p, G)^2)                 (Reconstruction Error)
  CD  = mean_M d(p, G) / 2 + mean_G d(q, M) / 2              (Chamfer-L1)
  RC  = fraction of q in G with a point of M within 2 nu     (Reconstruction Coverage)
  mIoU, Acc over the vertices that have a ground-truth point within 2 nu:
        the vertex's class against the class of its nearest ground-truth point;
        IoU_c = TP_c / (TP_c + FP_c + FN_c) averaged over the classes that
        occur (TP + FP + FN > 0), Acc = sum TP / number of such vertices.
Readings (also in the design notes): the truncation applies to both terms
of CD (the paper's d(.,.) carries it); "within 2 nu" includes 2 nu; the map
cloud is the welded vertex set (one point per lattice-edge key).

Plain numpy in FP64; nearest neighbours from scipy's k-d tree (a library
primitive).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def quality(map_points, map_labels, gt_points, gt_labels, trunc, n_classes, tie_rel=1e-6):
    """Metrics dict (re, cd, rc, miou, acc, counts, confusion [gt class][map class]) plus per-vertex
    flags `label_tie` where the two nearest ground-truth points of a vertex are within tie_rel trunc of
    each other in distance and differ in class, and `trunc_edge` where a distance lies within
    tie_rel trunc of the truncation (single precision may decide those the other way)."""
    M = np.asarray(map_points, np.float64).reshape(-1, 3)
    G = np.asarray(gt_points, np.float64).reshape(-1, 3)
    lm = np.asarray(map_labels, np.int64)
    lg = np.asarray(gt_labels, np.int64)
    tg, tm = cKDTree(G), cKDTree(M)
    d2g, i2g = tg.query(M, k=2)                # two nearest ground-truth points of each vertex
    dmg = d2g[:, 0]
    igm = i2g[:, 0]
    dgm, _ = tm.query(G)
    dpg = np.minimum(dmg, trunc)
    dqm = np.minimum(dgm, trunc)
    re = float(np.sqrt(np.mean(dpg ** 2))) if len(M) else 0.0
    cd = float(0.5 * np.mean(dpg) + 0.5 * np.mean(dqm)) if len(M) and len(G) else 0.0
    rc = float(np.mean(dgm <= trunc)) if len(G) else 0.0
    lab = dmg <= trunc
    conf = np.zeros((n_classes, n_classes), np.int64)
    np.add.at(conf, (lg[igm[lab]], lm[lab]), 1)
    tp = np.diag(conf).astype(np.float64)
    fp = conf.sum(axis=0) - tp
    fn = conf.sum(axis=1) - tp
    den = tp + fp + fn
    occ = den > 0
    miou = float(np.mean(tp[occ] / den[occ])) if occ.any() else 0.0
    acc = float(tp.sum() / conf.sum()) if conf.sum() else 0.0
    tie = (np.abs(d2g[:, 1] - d2g[:, 0]) <= tie_rel * trunc) & (lg[i2g[:, 1] % len(G)] != lg[igm])
    edge = np.abs(dmg - trunc) <= tie_rel * trunc
    return dict(re=re, cd=cd, rc=rc, miou=miou, acc=acc, n_map=len(M), n_gt=len(G), n_labeled=int(lab.sum()),
                n_correct=int(tp.sum()), confusion=conf, label_tie=tie, trunc_edge=edge,
                gt_edge=np.abs(dgm - trunc) <= tie_rel * trunc, d_map=dmg, d_gt=dgm)
