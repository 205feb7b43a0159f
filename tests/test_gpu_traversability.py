"""Mesh traversability (Sec. III-D): CUDA path vs the FP64 oracle, on meshes the map extracts.

Tolerances: positions are the same FP32 values on both sides, so the height
difference agrees to the rounding of one FP32 subtraction (|dz| <= 2^-23 |z|,
checked at 1e-5 m); ball sizes are exact except for vertices whose ball has a
candidate within 1e-6 r^2 of the radius in squared distance (the oracle flags
them; FP32 distances may decide those the other way); normals are sums of FP32
cross products of exactly representable differences, each with a relative
error of a few 2^-24, turned by at most the normal's condition number (sum of
face-normal lengths over the length of their sum, from the oracle) times
that; where it is <= 100, steepness and roughness agree to 1e-4 rad (angles
formed as atan2 of a cross and a dot product on the GPU), and vertices with
worse-conditioned normals (faces that nearly cancel) are left out of the
angle checks.  Traversable flags agree wherever no property is within those
tolerances of its threshold.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle.traversability import traversability as oracle_trav  # noqa: E402


def _lib():
    import paper_2412_00291_b300 as p
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _compare(p, gm, allowed, r=0.25, t_hd=0.6, t_s_deg=20.0, t_r_deg=30.0, min_vertices=5000):
    mesh = {k: v.cpu().numpy() for k, v in gm.mesh().items()}
    nv = len(mesh["vertex_keys"])
    assert nv >= min_vertices, nv
    props, trav = gm.traversability(nv, radius=r, max_height_diff=t_hd, max_steepness=math.radians(t_s_deg),
                                    max_roughness=math.radians(t_r_deg), allowed_classes=allowed)
    props, trav = props.cpu().numpy().astype(np.float64), trav.cpu().numpy().astype(bool)
    o = oracle_trav(mesh["positions"], mesh["colors"], mesh["vertex_keys"], mesh["triangles"], r=r, t_hd=t_hd,
                    t_s_deg=t_s_deg, t_r_deg=t_r_deg, allowed=allowed)
    ix = o["index"]
    clean = ~o["ball_ambiguous"][ix]
    well = o["normal_cond"][ix] <= 100.0
    assert clean.mean() > 0.95 and well.mean() > 0.99
    np.testing.assert_array_equal(props[clean, 3], o["ball_sizes"][ix][clean])
    dhd = np.abs(props[:, 0] - o["hd"][ix])[clean]
    ds = np.abs(props[:, 1] - o["s"][ix])[well]
    dr = np.abs(props[:, 2] - o["r"][ix])[clean & well]
    assert dhd.max() <= 1e-5, dhd.max()
    assert ds.max() <= 1e-4, ds.max()
    assert dr.max() <= 1e-4, dr.max()
    near = ((np.abs(o["hd"][ix] - t_hd) <= 1e-5) | (np.abs(o["s"][ix] - math.radians(t_s_deg)) <= 1e-4) |
            (np.abs(o["r"][ix] - math.radians(t_r_deg)) <= 1e-4) | ~clean | ~well)
    bad = (trav != o["traversable"][ix]) & ~near
    assert not bad.any(), np.flatnonzero(bad)[:10]
    return dict(vertices=nv, welded=len(o["hd"]), clean=int(clean.sum()), ill_conditioned=int((~well).sum()),
                traversable=int(trav.sum()),
                max_dhd=float(dhd.max()), max_ds=float(ds.max()), max_dr=float(dr.max()),
                mean_ball=float(props[:, 3].mean()))


def test_traversability_line16():
    p = _lib()
    w = synth.line16()
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    with pytest.raises(p.MapError) as e:          # nothing extracted yet
        gm.traversability(1)
    assert e.value.status == 6
    for f in synth.sequence(w):
        gm.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
    # the ground class only (class 0 of the generated scenes), and every class; two radii
    rep = _compare(p, gm, allowed=[0])
    print("line16 traversability (ground class):", rep)
    assert 0.1 * rep["vertices"] < rep["traversable"] < 0.9 * rep["vertices"]
    rep2 = _compare(p, gm, allowed=None, r=0.5, t_hd=0.3)
    print("line16 traversability (r 0.5 m, t_hd 0.3 m):", rep2)
    gm.close()


def test_traversability_loop64_two_scans():
    """Two 64 x 2048 scans at 0.1 m voxels: a mesh of ~10^5 vertices, scratch grown from the first call."""
    p = _lib()
    w = synth.loop64()
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=65536, hash_capacity=1 << 17,
                        mesh_vertex_capacity=1 << 23, mesh_triangle_capacity=1 << 24)
    for k, f in enumerate(synth.sequence(w, 2)):
        gm.integrate(L, _dev(f.points), f.T, probs=_dev(f.probs))
        rep = _compare(p, gm, allowed=[0, 1], min_vertices=5000)
        print(f"loop64 traversability after {k + 1} scan(s):", rep)
    gm.close()
