"""Semantic update from a camera label image, FP64 oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module; the product package never does, and the two
share no code.

What it follows (Liu et al., 2024, Sec. III-C.3): given a label image and
its pose, only the visible and observed voxels (W > 0) inside the camera
frustum are updated; they are found by ray casting, each voxel is projected
onto the image to take its pixel's class likelihood, and the distribution is
updated by the recursive Bayesian filter (Eq. bayesian_filter).  Readings
(also in the design notes):
  - pinhole camera, x right, y down, z forward; pixel (u, v) looks along
    ((u - cx) / fx, (v - cy) / fy, 1), and a point projects to the pixel
    nearest (fx x / z + cx, fy y / z + cy);
  - ray casting: the voxels a pixel's ray passes through, in order (exact
    3D traversal of the cells [nu (v - 1/2), nu (v + 1/2)) from the camera
    centre up to r_max); the visible surface is the first pair of
    consecutive voxels, both observed, with D >= 0 then D < 0; its range
    along the ray is interpolated between the two voxel centres' ranges,
    t0 + (t1 - t0) D0 / (D0 - D1), t the centre's projection onto the ray;
  - a voxel is updated when it is observed, projects to a pixel with a hit,
    and |psi| <= tau with psi = hit range - distance of the voxel centre
    from the camera (the projective distance of the metric update);
  - the candidates are all voxels of the map (those outside the frustum
    project outside the image or behind the camera);
  - the likelihood of a pixel is that of a scan point: p_hit / (1 - p_hit)
    / (C - 1) for a hard label, max(q_c, lik_floor) for probabilities.
Ambiguity flags (the GPU decides these in single precision, so its
traversal parameters, hit ranges and distances carry relative errors of a
few 1e-7): a pixel whose traversal met two crossing parameters within 1e-5
of each other (relative), a D within 1e-6 nu of 0 in the decisive pair, a
projection within 1e-3 px of a pixel boundary, or |psi| within
1e-4 m + 1e-6 of the hit range of tau.
"""
from __future__ import annotations

import math

import numpy as np

BS = 8


class VoxelStore:
    """Block access over an oracle map: D, W, logP of allocated blocks (read once)."""

    def __init__(self, om, C):
        self.C = C
        self.blocks = {}
        for b in om.alloc_blocks():
            blk = om.read_block(b)
            if blk is not None:
                self.blocks[tuple(int(x) for x in b)] = blk

    def voxel(self, v):
        b = (v[0] // BS, v[1] // BS, v[2] // BS)
        blk = self.blocks.get(b)
        if blk is None:
            return None
        li = (v[0] - BS * b[0]) + BS * ((v[1] - BS * b[1]) + BS * (v[2] - BS * b[2]))
        return blk, li


def pixel_ray(cam, u, v):
    d = np.array([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], 1.0])
    return d / np.linalg.norm(d)


def traverse(nu, c, d, r_max):
    """The voxels met by the ray c + t d, 0 <= t <= r_max, in order (exact cell traversal:
    each step crosses the nearest cell face), each with a flag set when the step that reached it
    had a second face within 1e-5 (relative) of the first."""
    v = [int(math.floor(c[k] / nu + 0.5)) for k in range(3)]
    step, tmax, tdelta = [0] * 3, [math.inf] * 3, [math.inf] * 3
    for k in range(3):
        if d[k] > 0:
            step[k] = 1
            tmax[k] = ((v[k] + 0.5) * nu - c[k]) / d[k]
            tdelta[k] = nu / d[k]
        elif d[k] < 0:
            step[k] = -1
            tmax[k] = ((v[k] - 0.5) * nu - c[k]) / d[k]
            tdelta[k] = -nu / d[k]
    amb = False
    t = 0.0
    while t <= r_max:
        yield tuple(v), amb
        order = sorted(range(3), key=lambda k: tmax[k])
        k = order[0]
        amb = tmax[order[1]] - tmax[k] <= 1e-5 * max(1.0, tmax[k])
        t = tmax[k]
        v[k] += step[k]
        tmax[k] += tdelta[k]


def raycast_pixel(store, nu, c, d, r_max):
    """Hit range along unit ray d from c (None if none) and an ambiguity flag."""
    amb = False
    prev = None   # (t of centre, D) of the previous voxel when observed
    for v, a in traverse(nu, c, d, r_max):
        amb = amb or a
        cell = store.voxel(v)
        cur = None
        if cell is not None:
            blk, li = cell
            if blk["W"][li] > 0:
                centre = np.array(v, np.float64) * nu
                cur = (float((centre - c) @ d), float(blk["D"][li]))
        if prev is not None and cur is not None and prev[1] >= 0.0 and cur[1] < 0.0:
            if abs(prev[1]) < 1e-6 * nu or abs(cur[1]) < 1e-6 * nu:
                amb = True
            t0, d0 = prev
            t1, d1 = cur
            return t0 + (t1 - t0) * d0 / (d0 - d1), amb
        prev = cur
    return None, amb


def camera_update(om, cam, T_wc, labels=None, probs=None, r_max=50.0, n_classes=20, p_hit=0.9,
                  lik_floor=1e-6, logp_floor=-30.0, nu=None, tau=None):
    """Expected result of one label image on the map held by oracle map `om`.

    cam: dict fx, fy, cx, cy, width, height.  Returns (updated: dict block -> (mask [512], new logP
    [C][512])), hits [H][W] (NaN: no hit), pixel ambiguity [H][W], voxel ambiguity dict."""
    C = n_classes
    store = VoxelStore(om, C)
    R, c = T_wc[:3, :3], T_wc[:3, 3]
    H, Wd = cam["height"], cam["width"]
    hits = np.full((H, Wd), np.nan)
    pamb = np.zeros((H, Wd), bool)
    for vv in range(H):
        for uu in range(Wd):
            d = R @ pixel_ray(cam, uu, vv)
            t, a = raycast_pixel(store, nu, c, d, r_max)
            pamb[vv, uu] = a
            if t is not None:
                hits[vv, uu] = t
    cand = list(store.blocks)
    if labels is not None:
        lo, hi = math.log((1.0 - p_hit) / (C - 1)), math.log(p_hit)
    updated, vamb = {}, {}
    Rt = R.T
    for b in cand:
        blk = store.blocks[b]
        mask = np.zeros(512, bool)
        amb = np.zeros(512, bool)
        newlp = blk["logP"].copy()
        for li in range(512):
            if not blk["W"][li] > 0:
                continue
            lx, ly, lz = li % 8, (li // 8) % 8, li // 64
            x = np.array([BS * b[0] + lx, BS * b[1] + ly, BS * b[2] + lz], np.float64) * nu
            xc = Rt @ (x - c)
            if xc[2] <= 0:
                continue
            uc = cam["fx"] * xc[0] / xc[2] + cam["cx"]
            vc = cam["fy"] * xc[1] / xc[2] + cam["cy"]
            u, v = int(math.floor(uc + 0.5)), int(math.floor(vc + 0.5))
            if 0.5 - abs(uc - u) < 1e-3 or 0.5 - abs(vc - v) < 1e-3:
                amb[li] = True
            if not (0 <= u < Wd and 0 <= v < H) or math.isnan(hits[v, u]):
                continue
            if pamb[v, u]:
                amb[li] = True
            psi = hits[v, u] - float(np.linalg.norm(x - c))
            if abs(abs(psi) - tau) < 1e-4 + 1e-6 * hits[v, u]:
                amb[li] = True
            if abs(psi) > tau:
                continue
            if labels is not None:
                l = int(labels[v, u])
                if not (0 <= l < C):
                    continue
                lik = np.full(C, lo)
                lik[l] = hi
            else:
                lik = np.log(np.maximum(probs[v, u].astype(np.float64), lik_floor))
            a = newlp[:, li] + lik
            m = a.max()
            lse = m + math.log(np.exp(a - m).sum())
            newlp[:, li] = np.maximum(a - lse, logp_floor)
            mask[li] = True
        updated[b] = (mask, newlp)
        vamb[b] = amb
    return updated, hits, pamb, vamb
