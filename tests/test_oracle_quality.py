"""Pins of the oracle's map quality metrics (Sec. IV-B.1) against closed forms and brute force."""
import numpy as np

from oracle.quality import quality


def plane_cloud(n, h, rng=None, labels=3):
    xs, ys = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
    P = np.stack([xs.ravel(), ys.ravel(), np.zeros(n * n)], axis=1)
    lab = np.full(n * n, labels, np.int64) if np.isscalar(labels) else labels
    return P, lab


def test_identical_clouds():
    G, lg = plane_cloud(30, 0.05)
    lg = np.arange(len(G)) % 4
    q = quality(G, lg, G, lg, trunc=0.2, n_classes=5)
    assert q["re"] == 0.0 and q["cd"] == 0.0 and q["rc"] == 1.0 and q["miou"] == 1.0 and q["acc"] == 1.0
    assert q["n_labeled"] == len(G)


def test_offset_along_the_normal():
    """Each map point sits delta above its ground-truth point on a grid of spacing h > delta:
    its nearest ground-truth point is the one below (at delta), and every ground-truth point's
    nearest map point is the one above, so RE = CD = delta and RC = 1."""
    G, lg = plane_cloud(40, 0.05)
    delta = 0.03
    M = G + np.array([0.0, 0.0, delta])
    q = quality(M, lg, G, lg, trunc=0.2, n_classes=5)
    assert abs(q["re"] - delta) < 1e-12 and abs(q["cd"] - delta) < 1e-12 and q["rc"] == 1.0
    # beyond the truncation: every distance is cut to 2 nu, nothing covered, nothing labelled
    M2 = G + np.array([0.0, 0.0, 0.5])
    q2 = quality(M2, lg, G, lg, trunc=0.2, n_classes=5)
    assert abs(q2["re"] - 0.2) < 1e-12 and abs(q2["cd"] - 0.2) < 1e-12 and q2["rc"] == 0.0
    assert q2["n_labeled"] == 0 and q2["acc"] == 0.0


def test_semantic_scores_closed_form():
    """Ground truth: classes 0 and 1 on halves of the grid; the map relabels a known number
    of class-0 points as 1: TP_0 = n0 - k, FN_0 = k, FP_1 = k, TP_1 = n1."""
    G, _ = plane_cloud(20, 0.05)
    lg = (np.arange(len(G)) >= 200).astype(np.int64)
    lm = lg.copy()
    k = 37
    lm[:k] = 1
    q = quality(G, lm, G, lg, trunc=0.2, n_classes=2)
    n0, n1 = 200, 200
    iou0 = (n0 - k) / n0
    iou1 = n1 / (n1 + k)
    assert abs(q["miou"] - 0.5 * (iou0 + iou1)) < 1e-12
    assert abs(q["acc"] - (n0 + n1 - k) / (n0 + n1)) < 1e-12
    np.testing.assert_array_equal(q["confusion"], [[n0 - k, k], [0, n1]])


def test_brute_force_distances():
    rng = np.random.default_rng(4)
    M = rng.uniform(-1, 1, size=(300, 3))
    G = rng.uniform(-1, 1, size=(400, 3))
    lm = rng.integers(0, 3, size=300)
    lg = rng.integers(0, 3, size=400)
    t = 0.25
    q = quality(M, lm, G, lg, trunc=t, n_classes=3)
    D = np.linalg.norm(M[:, None, :] - G[None, :, :], axis=2)
    dpg = np.minimum(D.min(axis=1), t)
    dqm = np.minimum(D.min(axis=0), t)
    assert abs(q["re"] - np.sqrt(np.mean(dpg ** 2))) < 1e-12
    assert abs(q["cd"] - (0.5 * dpg.mean() + 0.5 * dqm.mean())) < 1e-12
    assert abs(q["rc"] - np.mean(D.min(axis=0) <= t)) < 1e-12
    lab = D.min(axis=1) <= t
    conf = np.zeros((3, 3), np.int64)
    for i in np.flatnonzero(lab):
        conf[lg[np.argmin(D[i])], lm[i]] += 1
    np.testing.assert_array_equal(q["confusion"], conf)
