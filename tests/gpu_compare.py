"""Comparison helpers for the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (FP32 storage against FP64):
  D      |dD| <= 1e-4 * voxel_size (acceptance rule of the hot path); D is a
         weighted mean of truncated distances whose FP32 error is ~1e-7 m.
  W      |dW| <= n_frames * 2^-23 * W + 1e-6: a sum of <= n_frames weights in
         [0, 1], each exact to ~1e-7, accumulated in FP32.
  logP   |d logP| <= 1e-4 * n_frames^(1/2) + 1e-5 (FP32 log-sum-exp per update).
  label  equal wherever the oracle's top-two gap exceeds 1e-4 (near-ties are
         legitimately decided either way in FP32).
Voxels the oracle marks tainted (a projection within 1e-3 px of a pixel
boundary, or psi within 1e-5 nu of +-tau, at any frame) are excluded from
the strict comparison and counted.
"""
import numpy as np

BV = 512


def compare_blocks(gpu, orc, coords, nu, n_frames, n_classes, d_tol=None, lp_tol=None, label_gap=1e-4,
                   w_rel=None):
    d_tol = 1e-4 * nu if d_tol is None else d_tol
    lp_tol = 1e-4 * np.sqrt(n_frames) + 1e-5 if lp_tol is None else lp_tol
    w_rel = n_frames * 2.0 ** -23 if w_rel is None else w_rel
    g = gpu.read_blocks(coords)
    assert g["found"].all(), "allocated blocks missing on the GPU"
    rep = dict(voxels=0, observed=0, tainted_metric=0, tainted_sem=0, max_dD=0.0, max_dW_rel=0.0, max_dlogP=0.0,
               label_checked=0, label_near_tie=0, semantic=0)
    for i, b in enumerate(coords):
        o = orc.read_block(b)
        assert o is not None
        mt = (o["taint"] & 1) == 0
        st = (o["taint"] & 2) == 0
        rep["voxels"] += BV
        rep["tainted_metric"] += int((~mt).sum())
        rep["tainted_sem"] += int((~st).sum())
        obs = (o["W"] > 0) | (g["W"][i] > 0)
        rep["observed"] += int(obs.sum())
        # observation pattern: W > 0 on exactly the same untainted voxels
        bad = mt & ((o["W"] > 0) != (g["W"][i] > 0))
        assert not bad.any(), f"block {b}: W>0 differs at {np.flatnonzero(bad)[:8]}"
        dD = np.abs(g["D"][i] - o["D"])[mt]
        rep["max_dD"] = max(rep["max_dD"], float(dD.max(initial=0)))
        assert (dD <= d_tol).all(), f"block {b}: |dD| {dD.max()} > {d_tol}"
        dW = np.abs(g["W"][i] - o["W"])[mt]
        lim = w_rel * o["W"][mt] + 1e-6
        rep["max_dW_rel"] = max(rep["max_dW_rel"], float((dW / np.maximum(o["W"][mt], 1e-30)).max(initial=0)))
        assert (dW <= lim).all(), f"block {b}: |dW| {dW.max()}"
        if g["logP"] is not None:
            sem = st & mt
            dl = np.abs(g["logP"][i] - o["logP"])[:, sem]
            rep["max_dlogP"] = max(rep["max_dlogP"], float(dl.max(initial=0)))
            assert (dl <= lp_tol).all(), f"block {b}: |dlogP| {dl.max()} > {lp_tol}"
            upd = sem & (np.abs(o["logP"] + np.log(n_classes)).max(axis=0) > 1e-12)
            rep["semantic"] += int(upd.sum())
        clear = st & mt & (o["gap"] > label_gap)
        rep["label_near_tie"] += int((st & mt & (o["gap"] <= label_gap)).sum())
        lab_bad = clear & (g["label"][i] != o["label"])
        assert not lab_bad.any(), f"block {b}: label differs at {np.flatnonzero(lab_bad)[:8]}"
        rep["label_checked"] += int(clear.sum())
    return rep


def _tainted_cubes(orc, anchors, nu):
    """Anchors whose cube has a corner tainted for distance, or |D| < 1e-6, per the oracle."""
    cache = {}

    def blk(c):
        c = tuple(int(x) for x in c)
        if c not in cache:
            cache[c] = orc.read_block(c)
        return cache[c]
    out = np.zeros(len(anchors), bool)
    for i, a in enumerate(anchors):
        for c in range(8):
            v = np.array([a[0] + (c & 1), a[1] + ((c >> 1) & 1), a[2] + (c >> 2)])
            b = np.floor_divide(v, 8)
            o = blk(b)
            if o is None:
                continue
            li = int((v - 8 * b) @ np.array([1, 8, 64]))
            if (o["taint"][li] & 1) or (o["W"][li] > 0 and abs(o["D"][li]) < 1e-6):
                out[i] = True
                break
    return out


def compare_meshes(gm, om, orc, nu, pos_tol=1e-4, label_gap=1e-4):
    """GPU mesh (extract_mesh dict, numpy) vs oracle mesh; returns a report."""
    gk = gm["vertex_keys"]
    # seam vertices appear once per block: all copies must agree exactly
    order = np.argsort(gk, kind="stable")
    gk_s = gk[order]
    first = np.concatenate([[True], gk_s[1:] != gk_s[:-1]])
    gpos = gm["positions"][order]
    gcol = gm["colors"][order]
    grp = np.cumsum(first) - 1
    upos = gpos[first]
    assert np.all(gpos == upos[grp]) and np.all(gcol == gcol[first][grp]), "seam copies disagree"
    ukeys = gk_s[first]
    ucol = gcol[first]
    okeys = om["vkey"]
    # triangles as key triples + anchors
    gt = gk[gm["triangles"]]
    ga = gm["triangle_anchors"]
    ot = om["tkeys"]
    oa = om["tanchor"]
    g_taint = _tainted_cubes(orc, ga, nu)
    o_taint = _tainted_cubes(orc, oa, nu)
    gset = {tuple(t) for t, bad in zip(gt.tolist(), g_taint) if not bad}
    oset = {tuple(t) for t, bad in zip(ot.tolist(), o_taint) if not bad}
    rep = dict(gpu_tris=len(gt), oracle_tris=len(ot), tainted_tris=int(g_taint.sum() + o_taint.sum()),
               gpu_verts=len(ukeys), oracle_verts=len(okeys))
    only_g, only_o = gset - oset, oset - gset
    assert not only_g and not only_o, f"{len(only_g)} GPU-only, {len(only_o)} oracle-only triangles"
    # vertex positions and labels on keys used by untainted triangles
    used = np.unique(np.array(sorted(oset), dtype=np.int64).reshape(-1)) if oset else np.zeros(0, np.int64)
    gi = np.searchsorted(ukeys, used)
    oi = np.searchsorted(okeys, used)
    assert np.all(ukeys[gi] == used) and np.all(okeys[oi] == used)
    dp = np.abs(upos[gi].astype(np.float64) - om["vpos"][oi]).max(initial=0)
    rep["max_dpos"] = float(dp)
    assert dp <= pos_tol, f"vertex position error {dp}"
    vt = om["vtaint"][oi]
    clear = ((vt & 2) == 0) & ((vt & 1) == 0) & (om["vgap"][oi] > label_gap)
    lab_bad = clear & (ucol[gi, 3] != om["vlab"][oi])
    assert not lab_bad.any(), f"{lab_bad.sum()} vertex labels differ"
    rep["labels_checked"] = int(clear.sum())
    return rep
