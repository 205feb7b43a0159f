"""Pins of the oracle's mesh traversability (Sec. III-D, Table II parameters).

Expected values come from the geometry of hand-built meshes (planes, a
tilted plane, a step, a sphere) and from brute force over all vertex pairs,
not from the oracle's formulas retyped.
"""
import math

import numpy as np

from oracle.traversability import traversability


def grid_mesh(nx, ny, h, z=lambda x, y: 0.0 * x, label=0):
    """Triangulated grid over [0, (nx-1) h] x [0, (ny-1) h], normals up; keys = vertex ids."""
    xs, ys = np.meshgrid(np.arange(nx) * h, np.arange(ny) * h, indexing="ij")
    pos = np.stack([xs.ravel(), ys.ravel(), z(xs, ys).ravel()], axis=1)
    idx = np.arange(nx * ny).reshape(nx, ny)
    a, b, c, d = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel(), idx[:-1, 1:].ravel(), idx[1:, 1:].ravel()
    tri = np.concatenate([np.stack([a, b, c], 1), np.stack([b, d, c], 1)])
    col = np.zeros((len(pos), 4), np.uint8)
    col[:, 3] = label
    return pos, col, np.arange(len(pos), dtype=np.int64), tri


def rotate_x(pos, ang):
    c, s = math.cos(ang), math.sin(ang)
    R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    return pos @ R.T


def test_flat_ground_is_traversable():
    pos, col, key, tri = grid_mesh(30, 30, 0.05)
    t = traversability(pos, col, key, tri)
    assert np.all(t["hd"] == 0.0) and np.allclose(t["s"], 0.0, atol=1e-12) and np.allclose(t["r"], 0.0, atol=1e-7)
    assert t["traversable"].all()
    np.testing.assert_allclose(t["normals"], np.broadcast_to([0, 0, 1.0], t["normals"].shape), atol=1e-12)


def test_tilted_plane_steepness_and_height_range():
    r, h = 0.25, 0.02
    for deg in (5.0, 15.0, 25.0):
        ang = math.radians(deg)
        pos, col, key, tri = grid_mesh(60, 60, h)
        pos = rotate_x(pos, ang)
        t = traversability(pos, col, key, tri, r=r)
        np.testing.assert_allclose(t["s"], ang, atol=1e-9)
        assert np.allclose(t["r"], 0.0, atol=1e-7)
        # interior vertices: the ball meets the plane in a disc of radius r, elevation range 2 r sin(angle)
        xy = rotate_x(t["positions"], -ang)
        inner = ((xy[:, 0] > r + h) & (xy[:, 0] < 59 * h - r - h) & (xy[:, 1] > r + h) & (xy[:, 1] < 59 * h - r - h))
        assert inner.sum() > 100
        hd = t["hd"][inner]
        assert np.all(hd <= 2 * r * math.sin(ang) + 1e-12)
        assert np.all(hd >= 2 * (r - h) * math.sin(ang))
        assert t["traversable"].all() == (deg < 20.0)


def test_height_difference_brute_force():
    rng = np.random.default_rng(3)
    pos, col, key, tri = grid_mesh(25, 25, 0.04, z=lambda x, y: 0.3 * np.sin(7 * x) * np.cos(5 * y))
    pos = pos + rng.normal(scale=0.005, size=pos.shape)
    t = traversability(pos, col, key, tri, r=0.1)
    P = t["positions"]
    d = np.linalg.norm(P[:, None, :] - P[None, :, :], axis=2)
    inb = d <= 0.1
    z = P[:, 2]
    hd = np.array([z[m].max() - z[m].min() for m in inb])
    np.testing.assert_allclose(t["hd"], hd, atol=1e-12)
    np.testing.assert_array_equal(t["ball_sizes"], inb.sum(axis=1))
    # roughness: angle to the ball's mean normal, by brute force over the same balls
    N = t["normals"]
    for i in range(0, len(P), 37):
        m = N[inb[i]].mean(axis=0)
        ang = math.acos(max(-1.0, min(1.0, float(N[i] @ m / np.linalg.norm(m)))))
        assert abs(t["r"][i] - ang) < 1e-9


def test_step_height_and_vertical_face():
    # lower ground (x < 0), a 0.3 m vertical face at x = 0, upper ground (x > 0)
    h, r = 0.05, 0.25
    low, _, _, tl = grid_mesh(11, 21, h)
    low[:, 0] -= 10 * h
    face = np.array([[0.0, j * h, k * 0.1] for j in range(21) for k in range(4)])
    up, _, _, tu = grid_mesh(11, 21, h)
    up[:, 2] = 0.3
    pos = np.concatenate([low, face, up])
    nl, nf = len(low), len(face)
    # face triangles: columns j, rows k; wound toward -x (the lower side, free space)
    fidx = nl + np.arange(nf).reshape(21, 4)
    ft = []
    for j in range(20):
        for k in range(3):
            a, b, c, d = fidx[j, k], fidx[j + 1, k], fidx[j, k + 1], fidx[j + 1, k + 1]
            ft += [[a, c, b], [b, c, d]]
    tri = np.concatenate([tl, np.array(ft), tu + nl + nf])
    col = np.zeros((len(pos), 4), np.uint8)
    t = traversability(pos, col, np.arange(len(pos)), tri, r=r)
    P = t["positions"]
    on_face = (np.abs(P[:, 0]) < 1e-12) & (P[:, 2] > 0.05) & (P[:, 2] < 0.25)
    np.testing.assert_allclose(t["s"][on_face], math.pi / 2, atol=1e-9)
    assert not t["traversable"][on_face].any()
    # face vertices at 0.1 and 0.2 m reach both ground levels (0.1 / 0.2 m below, 0.2 / 0.1 m above)
    mid = on_face & (P[:, 1] > r) & (P[:, 1] < 1.0 - r)
    assert mid.sum() > 10
    np.testing.assert_allclose(t["hd"][mid], 0.3, atol=1e-12)
    far = (np.abs(P[:, 0]) > r + 1e-9)
    assert np.all(t["hd"][far] == 0.0) and t["traversable"][far].all()


def _sphere_steepness_error(nt, npp, R=2.0):
    th = np.linspace(0.05, math.pi - 0.05, nt)
    ph = np.arange(npp) * 2 * math.pi / npp
    pos = np.array([[R * math.sin(a) * math.cos(b), R * math.sin(a) * math.sin(b), R * math.cos(a)]
                    for a in th for b in ph])
    idx = np.arange(nt * npp).reshape(nt, npp)
    tri = []
    for i in range(nt - 1):
        for j in range(npp):
            a, b, c, d = idx[i, j], idx[i, (j + 1) % npp], idx[i + 1, j], idx[i + 1, (j + 1) % npp]
            tri += [[a, c, b], [b, c, d]]
    tri = np.array(tri)
    col = np.zeros((len(pos), 4), np.uint8)
    t = traversability(pos, col, np.arange(len(pos)), tri, r=0.3)
    inner = (np.arange(len(pos)) // npp > 0) & (np.arange(len(pos)) // npp < nt - 1)
    polar = np.arccos(t["positions"][:, 2] / R)
    return float(np.max(np.abs(t["s"][inner] - polar[inner]))), th[1] - th[0]


def test_sphere_steepness_is_polar_angle():
    """UV sphere with outward normals: steepness = the vertex's polar angle up to the
    discretisation error of area-weighted normals on a mesh with one diagonal per quad:
    below 0.15 of the polar step, and shrinking faster than the step when refined."""
    e1, h1 = _sphere_steepness_error(40, 80)
    e2, h2 = _sphere_steepness_error(80, 160)
    assert e1 < 0.15 * h1 and e2 < 0.15 * h2
    assert e2 / e1 < 0.6


def test_class_mask_and_welded_copies():
    pos, col, key, tri = grid_mesh(20, 20, 0.05, label=3)
    col[::7, 3] = 5
    a = traversability(pos, col, key, tri, allowed=[3])
    assert not a["traversable"][col[:, 3] == 5].any() and a["traversable"][col[:, 3] == 3].all()
    # duplicate every 3rd vertex (same key, same position): the welded result is unchanged
    dup = np.arange(0, len(pos), 3)
    pos2 = np.concatenate([pos, pos[dup]])
    col2 = np.concatenate([col, col[dup]])
    key2 = np.concatenate([key, key[dup]])
    remap = np.arange(len(pos))
    remap[dup] = len(pos) + np.arange(len(dup))
    tri2 = tri.copy()
    tri2[::2] = remap[tri[::2]]                       # half the triangles use the copies
    b = traversability(pos2, col2, key2, tri2, allowed=[3])
    for k in ("hd", "s", "r", "traversable"):
        np.testing.assert_allclose(b[k], a[k], atol=1e-12)
    np.testing.assert_array_equal(b["index"][len(pos):], dup)
