"""Mesh traversability of the FP64 oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module; the product package never does, and the two
share no code.

What it follows (Liu et al., 2024, Sec. III-D, "Traversability Extraction";
parameters from Table II): for every vertex of the metric-semantic mesh,
within the ball B of radius r around it,
  height difference  v_hd = the largest elevation difference of two
                     vertices of B (max z - min z),
  steepness          v_s  = arccos(n . e_z), the angle of the vertex normal
                     from the vertical,
  roughness          v_r  = the angle between the vertex normal and the
                     mean normal of B, (1 / |B|) sum over B of n_v,
and the vertex is traversable when v_hd < t_hd, v_s < t_s, v_r < t_r and its
class is one the robot may drive on.  Readings where the paper is garbled
(each also in the design notes): the printed height difference is an arg
max of vertex distances and is read as the elevation range; the printed
steepness and roughness apply arccos to a vector and compare a vector with
an angle, read as the angles above; the printed selection keeps vertices
whose properties all exceed the thresholds and is read the other way round
(below all thresholds is traversable).  A vertex is one welded mesh vertex
(equal lattice-edge keys); its normal is the area-weighted sum of the normals
of the triangles around it, normalised (triangles wound toward free space).

Plain numpy in FP64; the ball query uses scipy's k-d tree (a library
primitive), each vertex's ball is then reduced in order by numpy.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def weld(positions, colors, vertex_keys, triangles):
    """Unique vertices by key: (positions [U][3], labels [U], triangles over unique ids, index map [nv])."""
    keys = np.asarray(vertex_keys, np.int64)
    uk, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    pos = np.asarray(positions, np.float64).reshape(-1, 3)[first]
    lab = np.asarray(colors).reshape(-1, 4)[first, 3].astype(np.int64)
    tri = inv[np.asarray(triangles, np.int64).reshape(-1, 3)]
    return pos, lab, tri, inv


def vertex_normals(pos, tri):
    """Area-weighted vertex normals: sum of (b - a) x (c - a) over incident triangles, normalised
    (zero where a vertex has no triangle of non-zero area); and each normal's condition number
    sum |(b - a) x (c - a)| / |sum (b - a) x (c - a)| (large where incident faces nearly cancel, so
    that a rounding error in any one face turns the normal)."""
    a, b, c = pos[tri[:, 0]], pos[tri[:, 1]], pos[tri[:, 2]]
    fn = np.cross(b - a, c - a)
    acc = np.zeros_like(pos)
    mag = np.zeros(len(pos))
    fl = np.linalg.norm(fn, axis=1)
    for k in range(3):
        np.add.at(acc, tri[:, k], fn)
        np.add.at(mag, tri[:, k], fl)
    ln = np.linalg.norm(acc, axis=1)
    out = np.zeros_like(acc)
    ok = ln > 0
    out[ok] = acc[ok] / ln[ok, None]
    cond = np.full(len(pos), np.inf)
    cond[ok] = mag[ok] / ln[ok]
    return out, cond


def properties(pos, normals, r, amb_rel=1e-6):
    """(v_hd, v_s, v_r) per vertex, radians for the angles; the ball includes the vertex itself.

    Also flags each vertex whose ball has a candidate at squared distance within amb_rel r^2 of
    r^2 (single-precision distances may decide its membership the other way)."""
    tree = cKDTree(pos)
    balls = tree.query_ball_point(pos, r)
    wide = tree.query_ball_point(pos, r * (1.0 + amb_rel))
    n = len(pos)
    hd = np.zeros(n)
    vr = np.zeros(n)
    amb = np.zeros(n, bool)
    for i, b in enumerate(balls):
        b = np.asarray(b, np.int64)
        z = pos[b, 2]
        hd[i] = z.max() - z.min()
        m = normals[b].mean(axis=0)
        lm = np.linalg.norm(m)
        vr[i] = np.arccos(np.clip(normals[i] @ (m / lm), -1.0, 1.0)) if lm > 0 else 0.0
        w = np.asarray(wide[i], np.int64)
        d2 = np.sum((pos[w] - pos[i]) ** 2, axis=1)
        amb[i] = bool(np.any(np.abs(d2 - r * r) < amb_rel * r * r))
    vs = np.arccos(np.clip(normals[:, 2], -1.0, 1.0))
    return hd, vs, vr, balls, amb


def traversability(positions, colors, vertex_keys, triangles, r=0.25, t_hd=0.6, t_s_deg=20.0, t_r_deg=30.0,
                   allowed=None):
    """Per welded vertex: dict with positions, labels, normals, hd, s, r (radians), traversable, and
    `index` mapping every input vertex (seam copies included) to its welded vertex.

    allowed: iterable of classes a vertex may carry to be traversable (None: every class)."""
    pos, lab, tri, inv = weld(positions, colors, vertex_keys, triangles)
    nrm, cond = vertex_normals(pos, tri)
    hd, vs, vr, balls, amb = properties(pos, nrm, r)
    ok_cls = np.ones(len(pos), bool) if allowed is None else np.isin(lab, np.asarray(list(allowed), np.int64))
    trav = (hd < t_hd) & (vs < np.radians(t_s_deg)) & (vr < np.radians(t_r_deg)) & ok_cls
    return dict(positions=pos, labels=lab, normals=nrm, hd=hd, s=vs, r=vr, traversable=trav, index=inv,
                ball_sizes=np.array([len(b) for b in balls]), ball_ambiguous=amb, normal_cond=cond)
