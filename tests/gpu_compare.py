"""Comparison helpers for the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (FP32 storage against FP64):
  D      |dD| <= 1e-4 * voxel_size (acceptance rule of the hot path); D is a
         weighted mean of truncated distances whose FP32 error is ~1e-7 m.
  W      |dW| <= n_frames * 2^-23 * W + 1e-6: a sum of <= n_frames weights in
         [0, 1], each exact to ~1e-7, accumulated in FP32.
  logP   |d logP| <= 1e-4 * n_frames^(1/2) + 1e-5 (FP32 log-sum-exp per update).
  label  equal wherever the oracle's top-two gap exceeds 1e-4 (near-ties are
         legitimately decided either way in FP32).
Decisions (candidate acceptance): the GPU map records, for every scan, the
integer decisions its FP32 kernels took (each point's validity and pixel,
each pixel's winner, the touched block set, each voxel's pixel and whether
it was updated and class-updated).  The oracle takes every decision in FP64;
where its own computation lies in an ambiguity band (a projection within
1e-3 px of a pixel boundary, a range within 2^-20 relative of r_min, r_max
or of the pixel's nearest range, a block whose clearance from the band
segment is within the FP32 margin, psi within 1e-5 nu of +-tau) it accepts
the GPU's choice if that choice is one of its FP64 candidates and uses it;
everywhere else the GPU's choice must equal its own.  A rejected decision
fails the test, so every voxel is compared strictly: nothing is excluded.
Only the non-projective mode keeps taint marks, for its own FP32-sensitive
branches (normal orientation, the curvature branch, a vanishing tangent or
gradient sum), sticky per voxel.
"""
from collections import Counter

import numpy as np

BV = 512


class Lockstep:
    """A GPU map and the FP64 oracle fed the same scans in step (candidate acceptance of the
    GPU's recorded decisions, none rejected)."""

    def __init__(self, gm, om, exact_voxel_counts=True):
        import oracle
        gm.record_decisions(True)
        self.gm, self.om = gm, om
        self.rejections = oracle.REJECTIONS
        self.totals = Counter()
        self.frames = 0
        self.exact = exact_voxel_counts

    def scan(self, lid_gpu, lidar, points, T, labels=None, probs=None, nthreads=0):
        import torch

        def dev(a):
            return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.gm.integrate(lid_gpu, dev(points), T, labels=dev(labels), probs=dev(probs))
        d = self.gm.decisions(len(points), lidar.H * lidar.W)
        os_ = self.om.integrate(lidar, points, T, labels=labels, probs=probs, nthreads=nthreads, decisions=d)
        ck = self.om.check()
        bad = {k: ck[k] for k in self.rejections if ck[k]}
        assert not bad, (self.frames, bad, ck)
        self.totals.update(ck)
        self.frames += 1
        gs = self.gm.stats()
        keys = ["valid_points", "pixel_points", "touched_blocks", "new_blocks"]
        if self.exact:
            keys += ["voxels_updated", "voxels_semantic"]
        for key in keys:
            assert gs[key] == os_[key], (self.frames, key, gs[key], os_[key])
        return gs, os_, ck

    def report(self):
        t = self.totals
        return dict(frames=self.frames, points=t["points"], points_ambiguous=t["points_ambiguous"],
                    winners_ambiguous=t["winners_ambiguous"], blocks_sure=t["blocks_sure"],
                    blocks_ambiguous=t["blocks_ambiguous"], blocks_ambiguous_taken=t["blocks_ambiguous_taken"],
                    voxels=t["voxels"], voxel_pixels_ambiguous=t["voxel_pixels_ambiguous"],
                    voxel_updates_ambiguous=t["voxel_updates_ambiguous"],
                    voxel_classes_ambiguous=t["voxel_classes_ambiguous"])


# FP16 storage against FP64, per voxel: each store rounds to half an FP16 ulp (2^-11 relative)
# and the FP32 arithmetic between stores is exact by comparison.  After a voxel's n_upd
# distance updates: |dD| <= 2 n_upd 2^-11 tau (the stored D's own roundings, plus those of W
# shifting the running average by at most as much), |dW| <= n_upd (2^-11 W + 2^-25) (2^-25: the
# absolute step of FP16 subnormals, W < 2^-14); after its n_sem class
# updates: |dlogP| <= 2 n_sem 2^-11 |logp_floor| (each renormalisation passes on the error of the
# most probable class, whose log-probability is near 0), plus the FP16 rounding of the uniform
# prior (1e-3); labels compared where the oracle's top-two gap exceeds 0.05.
FP16_EPS = 2.0 ** -11


def compare_blocks(gpu, orc, coords, nu, n_frames, n_classes, d_tol=None, lp_tol=None, label_gap=1e-4,
                   w_rel=None, fp16=None):
    """GPU blocks against the oracle's, voxel by voxel.  fp16 = (tau, |logp_floor|): FP16-storage
    bounds per voxel from the oracle's update counts (FP16_EPS above) instead of the FP32 ones."""
    d_tol = 1e-4 * nu if d_tol is None else d_tol
    lp_tol = 1e-4 * np.sqrt(n_frames) + 1e-5 if lp_tol is None else lp_tol
    w_rel = n_frames * 2.0 ** -23 if w_rel is None else w_rel
    if fp16 is not None:
        label_gap = max(label_gap, 0.05)
    g = gpu.read_blocks(coords)
    assert g["found"].all(), "allocated blocks missing on the GPU"
    rep = dict(voxels=0, observed=0, tainted_metric=0, tainted_sem=0, max_dD=0.0, max_dW_rel=0.0, max_dlogP=0.0,
               label_checked=0, label_near_tie=0, semantic=0, label_mismatch=0)
    dd_all, dl_all, ratio_d, ratio_l = [], [], 0.0, 0.0
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
        if fp16 is not None:
            tau, lfloor = fp16
            dtol_v = (2.0 * o["n_upd"] * FP16_EPS * tau + 1e-4 * nu)[mt]
            wtol_v = (o["n_upd"] * (FP16_EPS * o["W"] + 2.0 ** -25) + 1e-6)[mt]   # 2^-25: subnormal W
            ltol_v = (2.0 * o["n_sem"] * FP16_EPS * lfloor + 1e-3)
        else:
            dtol_v = np.full(int(mt.sum()), d_tol)
            wtol_v = (w_rel * o["W"] + 1e-6)[mt]
            ltol_v = np.full(BV, lp_tol)
        dD = np.abs(g["D"][i] - o["D"])[mt]
        dd_all.append(dD[o["W"][mt] > 0])
        rep["max_dD"] = max(rep["max_dD"], float(dD.max(initial=0)))
        ratio_d = max(ratio_d, float((dD / dtol_v).max(initial=0)))
        assert (dD <= dtol_v).all(), f"block {b}: |dD| {dD.max()} > {dtol_v[np.argmax(dD - dtol_v)]}"
        dW = np.abs(g["W"][i] - o["W"])[mt]
        rep["max_dW_rel"] = max(rep["max_dW_rel"], float((dW / np.maximum(o["W"][mt], 1e-30)).max(initial=0)))
        assert (dW <= wtol_v).all(), f"block {b}: |dW| {dW.max()}"
        if g["logP"] is not None:
            sem = st & mt
            dl = np.abs(g["logP"][i] - o["logP"])[:, sem]
            lt = ltol_v[sem][None, :]
            rep["max_dlogP"] = max(rep["max_dlogP"], float(dl.max(initial=0)))
            ratio_l = max(ratio_l, float((dl / lt).max(initial=0)))
            assert (dl <= lt).all(), f"block {b}: |dlogP| {dl.max()} > {lp_tol}"
            upd = sem & (np.abs(o["logP"] + np.log(n_classes)).max(axis=0) > 1e-12)
            rep["semantic"] += int(upd.sum())
            dl_all.append(dl[:, upd[sem]].ravel())
        clear = st & mt & (o["gap"] > label_gap)
        rep["label_near_tie"] += int((st & mt & (o["gap"] <= label_gap)).sum())
        lab_bad = clear & (g["label"][i] != o["label"])
        assert not lab_bad.any(), f"block {b}: label differs at {np.flatnonzero(lab_bad)[:8]}"
        rep["label_checked"] += int(clear.sum())
        rep["label_mismatch"] += int((st & mt & (o["W"] > 0) & (g["label"][i] != o["label"])).sum())
    dd = np.concatenate(dd_all) if dd_all else np.zeros(0)
    dl = np.concatenate(dl_all) if dl_all else np.zeros(0)
    rep.update(p99_dD=float(np.percentile(dd, 99)) if len(dd) else 0.0, mean_dD=float(dd.mean()) if len(dd) else 0.0,
               p99_dlogP=float(np.percentile(dl, 99)) if len(dl) else 0.0,
               max_dD_over_bound=ratio_d, max_dlogP_over_bound=ratio_l)
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
