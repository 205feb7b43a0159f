"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Workloads are the seeded synthetic scans of ``synth`` (16 x 1024 straight
drive with hard labels; 64 x 2048 loop with probability vectors), plus
edge cases: empty scans, ragged point counts, all-invalid points, capacity
limits and bad poses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.fields import block_voxels  # noqa: E402
from tests.gpu_compare import Lockstep, compare_blocks, compare_meshes  # noqa: E402


def _lib():
    import paper_2412_00291_b300 as p
    return p



def _lidar(p, L):
    return p.lidar_intrinsics(L.H, L.W, L.fov_up, L.fov_down, L.r_min, L.r_max)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sorted(c):
    c = np.asarray(c).reshape(-1, 3)
    return c[np.lexsort((c[:, 2], c[:, 1], c[:, 0]))]


def _mesh_np(m):
    return {k: v.cpu().numpy() for k, v in m.items()}


@pytest.fixture(scope="module")
def line16_run():
    p = _lib()
    w = synth.line16()
    frames = list(synth.sequence(w))
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    L = _lidar(p, w.lidar)
    ls = Lockstep(gm, om)
    per_frame = []
    for k, f in enumerate(frames):
        gs, os_, ck = ls.scan(L, w.lidar, f.points, f.T, labels=f.labels)
        per_frame.append((gs, os_, ck, _sorted(gm.blocks()), _sorted(om.alloc_blocks())))
    return dict(p=p, w=w, gm=gm, om=om, frames=frames, per_frame=per_frame, lockstep=ls)


def test_line16_counts_and_block_sets(line16_run):
    """Every recorded decision of every scan accepted (Lockstep: point validity and pixel, pixel
    winners, voxel pixels and update / class-update flags equal the FP64 ones or, inside the FP64
    ambiguity bands, are FP64 candidates); the touched block set lies between the FP64 sure set and
    sure + ambiguous; counters and the allocated block set are then equal."""
    for k, (gs, os_, ck, gb, ob) in enumerate(line16_run["per_frame"]):
        assert gs["error_bits"] == 0
        assert os_["ambiguous_points"] == 0         # centre-ray points: no point is near a pixel edge
        assert ck["blocks_sure"] > 500 and ck["voxels"] == 512 * gs["touched_blocks"]
        np.testing.assert_array_equal(gb, ob)       # allocated block set
    print("line16 decisions:", line16_run["lockstep"].report())


def test_line16_voxels(line16_run):
    r = line16_run
    w = r["w"]
    coords = r["om"].alloc_blocks()
    rep = compare_blocks(r["gm"], r["om"], coords, w.voxel_size, w.frames, w.n_classes)
    print("line16 voxels:", rep)
    assert rep["tainted_metric"] == 0 and rep["tainted_sem"] == 0      # every voxel compared
    assert rep["label_checked"] > 0.5 * rep["semantic"]


def test_line16_mesh_and_incremental(line16_run):
    r = line16_run
    gm, om = r["gm"], r["om"]
    inc = _mesh_np(gm.mesh())
    rep = compare_meshes(inc, om.mesh(), om, r["w"].voxel_size)
    print("line16 mesh:", rep)
    assert rep["gpu_tris"] > 10000
    # incremental meshing equals meshing every block from scratch
    gm.remesh_all()
    full = _mesh_np(gm.mesh())

    def canon(m):
        k = m["vertex_keys"]
        t = k[m["triangles"]]
        tri = sorted(map(tuple, np.concatenate([t, m["triangle_anchors"]], axis=1).tolist()))
        v = sorted(zip(k.tolist(), map(tuple, m["positions"].tolist()), map(tuple, m["colors"].tolist())))
        return tri, v
    assert canon(inc) == canon(full)


def _canon_mesh(m):
    k = m["vertex_keys"]
    t = k[m["triangles"]]
    tri = sorted(map(tuple, np.concatenate([t, m["triangle_anchors"]], axis=1).tolist()))
    v = sorted(zip(k.tolist(), map(tuple, m["positions"].tolist()), map(tuple, m["colors"].tolist())))
    return tri, v


def test_fixed_rate_full_meshing(line16_run):
    """Per-frame meshing off, a full marching-cubes pass every 4 scans (the paper's fixed-rate
    global mesh): the voxels are unaffected and each full pass equals the incremental map's mesh
    at the same scan, and the oracle's."""
    r = line16_run
    p, w = r["p"], r["w"]
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    inc = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                         max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                         mesh_triangle_capacity=1 << 23)
    gm.set_incremental_mesh(False)
    with pytest.raises(p.MapError):                      # only 0 and 1 are valid
        p._check(p._lib.map_set_incremental_mesh(gm.h, 2), gm.h)
    passes = 0
    for k, f in enumerate(r["frames"]):
        for m in (gm, inc):
            m.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
        s = gm.stats()
        assert s["mesh_vertices"] == 0 and s["mesh_triangles"] == 0
        if k % 4 == 3 or k == len(r["frames"]) - 1:
            gm.remesh_all()
            a, b = _mesh_np(gm.mesh()), _mesh_np(inc.mesh())
            assert len(a["triangles"]) > 1000
            assert _canon_mesh(a) == _canon_mesh(b)
            passes += 1
    assert passes == 3
    # a second full pass rebuilds the same mesh from an emptied arena
    before = _canon_mesh(_mesh_np(gm.mesh()))
    gm.remesh_all()
    st = gm.stats()                                      # the counters describe the full pass
    again = _mesh_np(gm.mesh())
    assert _canon_mesh(again) == before
    assert st["dirty_blocks"] == st["total_blocks"]
    assert st["mesh_vertices"] == len(again["vertex_keys"]) and st["mesh_triangles"] == len(again["triangles"])
    coords = r["om"].alloc_blocks()
    x, y = gm.read_blocks(coords), inc.read_blocks(coords)
    for key in ("D", "W", "label"):
        assert np.array_equal(x[key], y[key])
    compare_meshes(_mesh_np(gm.mesh()), r["om"].mesh(), r["om"], w.voxel_size)
    gm.close()
    inc.close()


def test_edge_cases_empty_ragged_invalid():
    p = _lib()
    w = synth.line16()
    f = next(iter(synth.sequence(w, 1)))
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=16384, hash_capacity=1 << 15,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 21,
                        mesh_triangle_capacity=1 << 22)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    ls = Lockstep(gm, om)
    # empty scan
    gs, os_, _ = ls.scan(L, w.lidar, np.zeros((0, 3), np.float32), f.T, labels=np.zeros(0, np.int32))
    assert gs["valid_points"] == 0 and gs["touched_blocks"] == 0 and gs["total_blocks"] == 0
    # all points invalid: NaN, too near, too far
    bad = np.full((300, 3), np.nan, np.float32)
    bad[100:200] = [0.1, 0.0, 0.0]
    bad[200:] = [500.0, 0.0, 0.0]
    gs, _, ck = ls.scan(L, w.lidar, bad, f.T, labels=np.zeros(300, np.int32))
    assert gs["valid_points"] == 0 and ck["points"] == 300
    # ragged count (not a multiple of the block size), labels out of range ignored
    n = 16384 - 37
    lab = f.labels[:n].copy()
    lab[::97] = 99
    ls.scan(L, w.lidar, f.points[:n], f.T, labels=lab)
    np.testing.assert_array_equal(_sorted(gm.blocks()), _sorted(om.alloc_blocks()))
    rep = compare_blocks(gm, om, om.alloc_blocks(), w.voxel_size, 1, w.n_classes)
    assert rep["observed"] > 10000


def test_changing_image_sizes_and_interleaved_calls():
    """Scans whose range images alternate between 16 x 1024 and 32 x 2048 pixels, with a full re-mesh
    between some of them.  Each scan's range image and counters are reset
    ahead of time by the previous scan's per-point kernel (two sets in turn), so a larger image after a
    smaller one, or a re-mesh that reuses the counters between scans, must leave nothing stale: per-scan
    counters, the download ring's copies of them, the block set, the voxels and the mesh all against
    the oracle fed the same scans."""
    import dataclasses
    p = _lib()
    w = synth.line16()
    wide = dataclasses.replace(w, lidar=synth.lidar_deg(32, 2048, 15.0, -15.0, 50.0))
    scene = synth.make_scene(w)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=65536, max_pixels=65536, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    ls = Lockstep(gm, om)
    seen = []
    for k, T in enumerate(synth.trajectory(w, 7)):
        wk = wide if k in (1, 2, 5) else w
        f = synth.make_frame(wk, scene, T, k)
        gs, os_, _ = ls.scan(_lidar(p, wk.lidar), wk.lidar, f.points, f.T, labels=f.labels)
        seen.append(gs)
        assert gs["error_bits"] == 0
        if k in (2, 3):
            gm.remesh_all()
            assert gm.stats()["mesh_triangles"] > 0
    for k, gs in enumerate(seen):
        fs = gm.frame_stats(k)
        for key in ("valid_points", "pixel_points", "touched_blocks", "new_blocks", "voxels_updated",
                    "voxels_semantic", "mesh_vertices", "mesh_triangles"):
            assert fs[key] == gs[key], (k, key)
    np.testing.assert_array_equal(_sorted(gm.blocks()), _sorted(om.alloc_blocks()))
    rep = compare_blocks(gm, om, om.alloc_blocks(), w.voxel_size, 7, w.n_classes)
    assert rep["tainted_metric"] == 0
    compare_meshes(_mesh_np(gm.mesh()), om.mesh(), om, w.voxel_size)
    gm.close()


def test_capacities_at_their_limits():
    """Sizes at the configured maxima: a scan of exactly max_points points on an image of exactly
    max_pixels pixels into a pool of exactly the blocks it needs integrates without an error bit
    and matches the oracle; one point more is refused on the host, and a pool one block short
    latches the pool-full error on the device with the pool exactly full."""
    p = _lib()
    w = synth.line16()
    f = next(iter(synth.sequence(w, 1)))
    L = _lidar(p, w.lidar)
    npix = w.lidar.H * w.lidar.W
    assert len(f.points) == npix
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    os_ = om.integrate(w.lidar, f.points, f.T, labels=f.labels)

    def make(max_blocks):
        return p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=max_blocks,
                              hash_capacity=4 * max_blocks, max_points=npix, max_pixels=npix,
                              mesh_vertex_capacity=1 << 21, mesh_triangle_capacity=1 << 22)
    # the blocks the scan needs: the GPU's own set (the oracle alone takes every FP64-ambiguous block)
    big = make(1 << 14)
    big.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
    need = big.stats()["total_blocks"]
    big.close()
    assert os_["sure_blocks"] <= need <= os_["sure_blocks"] + os_["ambiguous_blocks"]
    gm = make(need)
    om2 = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    s, _, _ = Lockstep(gm, om2).scan(L, w.lidar, f.points, f.T, labels=f.labels)
    assert s["error_bits"] == 0 and s["total_blocks"] == need
    np.testing.assert_array_equal(_sorted(gm.blocks()), _sorted(om2.alloc_blocks()))
    rep = compare_blocks(gm, om2, om2.alloc_blocks(), w.voxel_size, 1, w.n_classes)
    assert rep["observed"] > 10000
    extra = np.concatenate([f.points, f.points[:1]])
    with pytest.raises(p.MapError) as e:
        gm.integrate(L, _dev(extra), f.T, labels=_dev(np.concatenate([f.labels, f.labels[:1]])))
    assert e.value.status == 1
    gm.close()
    short = make(need - 1)
    short.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
    s = short.stats(check=False)
    assert s["error_bits"] & 1 and s["total_blocks"] == need - 1
    short.close()


def test_crowded_hash_table():
    """The hash at the most crowded load the API allows (capacity: the smallest power of two at least
    twice the pool): a pool of exactly the blocks k scans need, k chosen so that the load ends nearest
    50 %.  Home slots then often hold another key (linear probing), neighbouring points of different
    warps race to insert the same new block, and every scan must still match the oracle in lockstep:
    the block set, the counters, every voxel, and no error bit."""
    p = _lib()
    w = synth.line16()
    frames = list(synth.sequence(w, 10))
    L = _lidar(p, w.lidar)
    probe = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=1 << 14, hash_capacity=1 << 16,
                           max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 21,
                           mesh_triangle_capacity=1 << 22)
    need = []
    for f in frames:
        probe.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
        need.append(probe.stats()["total_blocks"])
    probe.close()

    def load(n):
        cap = 1
        while cap < 2 * n:
            cap <<= 1
        return n / cap
    k = max(range(len(need)), key=lambda i: load(need[i]))
    assert load(need[k]) > 0.4
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=need[k], hash_capacity=2,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 21,
                        mesh_triangle_capacity=1 << 22)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    ls = Lockstep(gm, om)
    for f in frames[:k + 1]:
        s, _, _ = ls.scan(L, w.lidar, f.points, f.T, labels=f.labels)
        assert s["error_bits"] == 0
    assert gm.stats()["total_blocks"] == need[k]
    np.testing.assert_array_equal(_sorted(gm.blocks()), _sorted(om.alloc_blocks()))
    rep = compare_blocks(gm, om, om.alloc_blocks(), w.voxel_size, k + 1, w.n_classes)
    assert rep["observed"] > 10000
    gm.close()


def test_azimuth_seam_and_elevation_edges():
    """Points on the azimuth seam behind the sensor (y = +0.0, -0.0 and a few ulps either side, where
    atan2 jumps from pi to -pi and the column index wraps from W to 0), and points just inside and
    well outside the top and bottom beams: pixel assignment, winners, the block set and the voxels
    against the oracle, with a rotated, translated pose."""
    p = _lib()
    w = synth.line16()
    Lw = w.lidar
    L = _lidar(p, Lw)
    pts = []
    for v in range(Lw.H):
        th = Lw.theta0 + v * Lw.dtheta
        for r in (4.0, 9.5, 17.25, 31.0):
            for y in (0.0, -0.0, 1e-6, -1e-6, 3e-7, -3e-7):
                x = -r * np.sin(th)
                pts.append((x, y, r * np.cos(th)))
    for th in (Lw.theta0 - 0.2 * Lw.dtheta, Lw.theta0 + (Lw.H - 1.2) * Lw.dtheta,
               Lw.theta0 - 1.0 * Lw.dtheta, Lw.theta0 + (Lw.H + 0.0) * Lw.dtheta):
        for phi in np.linspace(-3.0, 3.0, 41):
            r = 12.0
            pts.append((r * np.sin(th) * np.cos(phi), r * np.sin(th) * np.sin(phi), r * np.cos(th)))
    pts = np.array(pts, np.float32)
    lab = (np.arange(len(pts)) % w.n_classes).astype(np.int32)
    T = synth.pose(synth.rot_rpy(0.01, -0.02, 0.7), [3.2, -1.1, 1.8])
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=16384, hash_capacity=1 << 15,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 21,
                        mesh_triangle_capacity=1 << 22)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    gs, os_, ck = Lockstep(gm, om).scan(L, Lw, pts, T, labels=lab)
    assert os_["ambiguous_points"] == 0
    assert gs["pixel_points"] < gs["valid_points"]          # the points outside the beams have no pixel
    np.testing.assert_array_equal(_sorted(gm.blocks()), _sorted(om.alloc_blocks()))
    rep = compare_blocks(gm, om, om.alloc_blocks(), w.voxel_size, 1, w.n_classes)
    print("seam and edges:", gs, rep, ck)
    assert rep["observed"] > 300 and rep["tainted_metric"] == 0
    gm.close()


def test_errors_bad_pose_args_capacity():
    p = _lib()
    w = synth.line16()
    f = next(iter(synth.sequence(w, 1)))
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=64, hash_capacity=256,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 16,
                        mesh_triangle_capacity=1 << 16)
    pts, lab = _dev(f.points), _dev(f.labels)
    T = f.T.copy()
    T[0, 0] *= 1.01
    with pytest.raises(p.MapError) as e:
        gm.integrate(L, pts, T, labels=lab)
    assert e.value.status == 4
    with pytest.raises(p.MapError) as e:
        gm.integrate(L, pts, f.T, labels=lab, probs=torch.zeros((len(pts), 20), device="cuda"))
    assert e.value.status == 1
    big = p.lidar_intrinsics(512, 1024, 0.3, -0.3)
    with pytest.raises(p.MapError) as e:
        gm.integrate(big, pts, f.T, labels=lab)
    assert e.value.status == 1
    # the pool holds 64 blocks: the scan needs more -> latched capacity error, no fault
    gm.integrate(L, pts, f.T, labels=lab)
    s = gm.stats(check=False)
    assert s["error_bits"] & 1
    with pytest.raises(p.MapError) as e:
        gm.sync()
    assert e.value.status == 3
    assert s["total_blocks"] == 64


def test_far_pose_refused_and_map_unchanged():
    """A scan whose reach leaves the map's coordinate range (|voxel| < 2^19 - 16) is refused with
    MAP_ERR_BAD_POSE before any launch, and the map, its frame count and its queries stay as they
    were; a query point beyond the range is invalid (its block key would alias)."""
    p = _lib()
    w = synth.line16()
    f = next(iter(synth.sequence(w, 1)))
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=8192, hash_capacity=1 << 15,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 20,
                        mesh_triangle_capacity=1 << 21)
    pts, lab = _dev(f.points), _dev(f.labels)
    gm.integrate(L, pts, f.T, labels=lab)
    before = _sorted(gm.blocks())
    n0 = gm.frame_count()
    lim = (2 ** 19 - 16) * w.voxel_size
    for axis in range(3):
        T = f.T.copy()
        T[axis, 3] = lim - w.lidar.r_max - w.truncation + 0.5 * w.voxel_size
        with pytest.raises(p.MapError) as e:
            gm.integrate(L, pts, T, labels=lab)
        assert e.value.status == 4 and "coordinate range" in str(e.value)
    gm.sync()
    assert gm.frame_count() == n0
    np.testing.assert_array_equal(_sorted(gm.blocks()), before)
    # a query at a voxel aliasing onto an allocated block (block x + 2^21) is invalid
    b = before[len(before) // 2].astype(np.float64)
    x = (8 * b + 3.25) * w.voxel_size
    xa = x.copy()
    xa[0] += 8 * (2 ** 21) * w.voxel_size
    sdf, valid = gm.query(torch.tensor(np.stack([x, xa]), dtype=torch.float32, device="cuda"))
    assert not bool(valid[1]) and torch.isnan(sdf[1])


@pytest.mark.slow
def test_loop64_full_size_sampled():
    """The 200-scan 64 x 2048 workload at full size, in the benchmark's launch configuration.

    The GPU integrates all 200 scans; the oracle recomputes the complete
    allocated block set (integer work) and, for a seeded sample of blocks
    drawn from its own set plus their +x/+y/+z neighbours, every voxel value.
    """
    p = _lib()
    w = synth.loop64()
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes)
    scene = synth.make_scene(w)
    Ts = synth.trajectory(w)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    # sample: blocks of an oracle-only allocation pass over the first 3 scans
    probe = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    probe.set_track(np.zeros((0, 3), np.int32))
    fr = None
    for k in range(3):
        fr = synth.make_frame(w, scene, Ts[k], k, out=fr)
        probe.integrate(w.lidar, fr.points, fr.T, probs=fr.probs)
    cand = probe.alloc_blocks()
    rng = np.random.default_rng(2024)
    base = cand[rng.choice(len(cand), size=48, replace=False)]
    track = np.unique(np.concatenate([base + np.array([dx, dy, dz]) for dx in (0, 1) for dy in (0, 1)
                                      for dz in (0, 1)]), axis=0)
    om.set_track(track)
    ls = Lockstep(gm, om, exact_voxel_counts=False)
    fr = None
    for k in range(w.frames):
        fr = synth.make_frame(w, scene, Ts[k], k, out=fr)
        ls.scan(L, w.lidar, fr.points, fr.T, probs=fr.probs)
    np.testing.assert_array_equal(_sorted(gm.blocks()), _sorted(om.alloc_blocks()))
    dec = ls.report()
    print("loop64 decisions:", dec)
    assert dec["blocks_sure"] > 100 * w.frames
    have = np.array([b for b in track if om.read_block(b) is not None])
    rep = compare_blocks(gm, om, have, w.voxel_size, w.frames, w.n_classes)
    print("loop64 sampled voxels:", rep)
    assert rep["observed"] > 5000 and rep["tainted_metric"] == 0
    # mesh segments of the sampled base blocks (their cubes only need the tracked neighbours)
    full = _mesh_np(gm.mesh())
    anc_blk = np.floor_divide(full["triangle_anchors"], 8)
    keep = np.zeros(len(anc_blk), bool)
    base_set = {tuple(b) for b in base if om.read_block(b) is not None}
    for i, b in enumerate(map(tuple, anc_blk.tolist())):
        keep[i] = b in base_set
    sub_t = full["triangles"][keep]
    used = np.unique(sub_t)
    remap = np.full(len(full["vertex_keys"]), -1, np.int64)
    remap[used] = np.arange(len(used))
    sub = dict(vertex_keys=full["vertex_keys"][used], positions=full["positions"][used],
               colors=full["colors"][used], triangles=remap[sub_t], triangle_anchors=full["triangle_anchors"][keep])
    mrep = compare_meshes(sub, om.mesh(np.array(sorted(base_set))), om, w.voxel_size)
    print("loop64 sampled mesh:", mrep)


def test_loop64_error_binned_by_range():
    """|dD| of the 64 x 2048 scans (0.1 m voxels, 100 m range) by the voxel's distance from the
    sensor: blocks sampled evenly from four range bins; every bin within 1e-4 nu."""
    p = _lib()
    w = synth.loop64()
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=65536, hash_capacity=1 << 17,
                        mesh_vertex_capacity=1 << 23, mesh_triangle_capacity=1 << 24)
    scene = synth.make_scene(w)
    Ts = synth.trajectory(w)
    K = 3
    frames = [synth.make_frame(w, scene, Ts[k], k) for k in range(K)]
    probe = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    probe.set_track(np.zeros((0, 3), np.int32))
    for fr in frames:
        probe.integrate(w.lidar, fr.points, fr.T, probs=fr.probs)
    cand = probe.alloc_blocks()
    centre = (cand + 0.5) * 8 * w.voxel_size
    rng_m = np.linalg.norm(centre - frames[0].T[:3, 3], axis=1)
    bins = [(0.0, 16.0), (16.0, 32.0), (32.0, 64.0), (64.0, 100.0)]
    rs = np.random.default_rng(11)
    pick = []
    for lo, hi in bins:
        idx = np.flatnonzero((rng_m >= lo) & (rng_m < hi))
        pick.append(cand[rs.choice(idx, size=min(24, len(idx)), replace=False)])
    track = np.concatenate(pick)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    om.set_track(track)
    ls = Lockstep(gm, om, exact_voxel_counts=False)
    for fr in frames:
        ls.scan(L, w.lidar, fr.points, fr.T, probs=fr.probs)
    g = gm.read_blocks(track, want_logp=False)
    tol = 1e-4 * w.voxel_size
    rep = []
    for lo, hi in bins:
        d_all = []
        for i, b in enumerate(track):
            o = om.read_block(b)
            if o is None:
                continue
            r = np.linalg.norm(block_voxels(b) * w.voxel_size - frames[0].T[:3, 3], axis=1)
            sel = (o["W"] > 0) & (r >= lo) & (r < hi)
            d_all.append(np.abs(g["D"][i] - o["D"])[sel])
        d = np.concatenate(d_all) if d_all else np.zeros(0)
        rep.append((lo, hi, len(d), float(d.max(initial=0)), float(np.percentile(d, 99)) if len(d) else 0.0))
        assert len(d) > 100, (lo, hi, len(d))
        assert d.max() <= tol, (lo, hi, d.max())
    print("loop64 |dD| by range (m): " + "; ".join(f"[{lo:.0f}, {hi:.0f}) n {n} max {mx:.2e} p99 {p9:.2e}"
                                                   for lo, hi, n, mx, p9 in rep))
    gm.close()


@pytest.mark.parametrize("storage,cls", [(0, "probs"), (1, "labels"), (1, "probs"), (0, "labels")])
def test_generic_class_count(storage, cls):
    """C = 7 classes (the kernels' generic class-count path) against the oracle, both class
    inputs, both storage precisions (FP16 at its stated bound)."""
    p = _lib()
    w = synth.line16()
    C = 7
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, C, storage=storage, max_blocks=32768,
                        hash_capacity=1 << 16, max_points=32768, max_pixels=32768,
                        mesh_vertex_capacity=1 << 22, mesh_triangle_capacity=1 << 23)
    om = oracle.OracleMap(w.voxel_size, w.truncation, C)
    ls = Lockstep(gm, om)
    rng = np.random.default_rng(7)
    frames = list(synth.sequence(w, 4))
    for f in frames:
        lab = np.where(f.labels >= 0, f.labels % C, -1).astype(np.int32)
        if cls == "probs":
            q = rng.uniform(0.0, 1.0, size=(len(lab), C)).astype(np.float32)
            q[np.arange(len(lab)), np.clip(lab, 0, C - 1)] += 4.0
            q = (q / q.sum(axis=1, keepdims=True)).astype(np.float32)
            ls.scan(L, w.lidar, f.points, f.T, probs=q)
        else:
            ls.scan(L, w.lidar, f.points, f.T, labels=lab)
    coords = _sorted(gm.blocks())
    assert np.array_equal(coords, _sorted(om.alloc_blocks()))
    if storage == 0:
        rep = compare_blocks(gm, om, coords, w.voxel_size, len(frames), C)
    else:
        K = len(frames)
        rep = compare_blocks(gm, om, coords, w.voxel_size, K, C, fp16=(w.truncation, 30.0))
    print(f"C = 7, storage {storage}, {cls}:", rep)
    assert rep["semantic"] > 1000 and rep["label_checked"] > 100
    gm.close()


def test_probability_floors_against_oracle():
    """Sharply peaked probability vectors with exact zeros: every class but the winner's enters at
    the likelihood floor, and after three scans the log-probability floor binds for them.  The 20-
    class fast path against the oracle, floored entries included (both sit at logp_floor)."""
    p = _lib()
    w = synth.line16()
    C = w.n_classes
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, C, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    om = oracle.OracleMap(w.voxel_size, w.truncation, C)
    ls = Lockstep(gm, om)
    frames = list(synth.sequence(w, 4))
    for f in frames:
        q = np.zeros((len(f.labels), C), np.float32)
        q[np.arange(len(f.labels)), np.clip(f.labels, 0, C - 1)] = 1.0
        ls.scan(L, w.lidar, f.points, f.T, probs=q)
    coords = _sorted(om.alloc_blocks())
    rep = compare_blocks(gm, om, coords, w.voxel_size, len(frames), C)
    g = gm.read_blocks(coords)
    n_floor_g = int((g["logP"] == -30.0).sum())
    n_floor_o = sum(int((om.read_block(b)["logP"] == -30.0).sum()) for b in coords)
    print("floors:", rep, n_floor_g, n_floor_o)
    assert rep["semantic"] > 1000 and n_floor_o > 10000
    assert abs(n_floor_g - n_floor_o) <= 0.01 * n_floor_o and rep["tainted_metric"] == 0
    gm.close()


def test_far_from_origin():
    """The whole drive 10 km / -7 km / +30 m away from the world origin: the sensor-relative
    voxel offsets (integer + float pair) keep FP32 psi at the same accuracy."""
    p = _lib()
    w = synth.line16()
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    ls = Lockstep(gm, om)
    shift = np.array([10000.0, -7000.0, 30.0])
    frames = list(synth.sequence(w, 3))
    for f in frames:
        T = f.T.copy()
        T[:3, 3] += shift
        ls.scan(L, w.lidar, f.points, T, labels=f.labels)
    print("far from origin decisions:", ls.report())
    coords = _sorted(gm.blocks())
    assert np.array_equal(coords, _sorted(om.alloc_blocks()))
    assert coords[:, 0].min() > 5000          # blocks really are far away (0.2 m voxels, 8 per block)
    rep = compare_blocks(gm, om, coords, w.voxel_size, len(frames), w.n_classes)
    assert rep["max_dD"] <= 1e-4 * w.voxel_size and rep["observed"] > 50000
    g = _mesh_np(gm.mesh())
    # vertex positions are FP32 world coordinates: at 10 km one ulp is ~1 mm
    ulp = np.spacing(np.float32(np.abs(g["positions"]).max()))
    compare_meshes(g, om.mesh(), om, w.voxel_size, pos_tol=1e-4 + 2.0 * float(ulp))


def test_duplicate_points_nearest_lowest_index_wins():
    """Points sharing a pixel: the nearest wins the range image, equal ranges the lower index
    (its label is the one fused)."""
    p = _lib()
    w = synth.line16()
    L = _lidar(p, w.lidar)
    f = next(iter(synth.sequence(w, 1)))
    ok = np.isfinite(f.points).all(axis=1)
    pts, lab = f.points[ok][:4000], f.labels[ok][:4000]
    # every point twice: identical copies with another label, and a copy 1 cm farther
    far = pts * (1.0 + 0.01 / np.linalg.norm(pts, axis=1, keepdims=True)).astype(np.float32)
    P2 = np.concatenate([pts, pts, far]).astype(np.float32)
    L2 = np.concatenate([lab, (lab + 1) % w.n_classes, (lab + 2) % w.n_classes]).astype(np.int32)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=16384, hash_capacity=1 << 15,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 21,
                        mesh_triangle_capacity=1 << 22)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    _, _, ck = Lockstep(gm, om).scan(L, w.lidar, P2, f.T, labels=L2)
    assert ck["winners_ambiguous"] >= 3000       # the identical copies: two candidates, lower index taken
    coords = _sorted(gm.blocks())
    assert np.array_equal(coords, _sorted(om.alloc_blocks()))
    rep = compare_blocks(gm, om, coords, w.voxel_size, 1, w.n_classes)
    assert rep["label_checked"] > 1000


def test_mesh_arena_full_is_reported():
    """A mesh arena too small for the scan: the capacity error is latched and reported, the
    blocks that did not fit keep no segment, and nothing faults."""
    p = _lib()
    w = synth.line16()
    L = _lidar(p, w.lidar)
    f = next(iter(synth.sequence(w, 1)))
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=16384, hash_capacity=1 << 15,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=4096,
                        mesh_triangle_capacity=8192)
    gm.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
    s = gm.stats(check=False)
    assert s["error_bits"] & 8            # ERR_ARENA_FULL
    with pytest.raises(p.MapError) as e:
        gm.sync()
    assert e.value.status == 3
    m = gm.mesh()                          # what did fit is still a valid mesh
    tri = m["triangles"].cpu().numpy()
    assert tri.size == 0 or tri.max() < m["positions"].shape[0]
    gm.close()


def test_line16_jittered_rays():
    """Points off their pixel's centre ray (each ray turned by N(0, 0.35 px) in both angles):
    points within 1e-3 px of a pixel boundary, pixels with two or more points and pixels with
    none.  Every recorded decision (point pixel, winner, block set, voxel pixel and gates) is
    accepted by the oracle, and all voxels and the mesh match."""
    p = _lib()
    w = synth.line16_jitter()
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    ls = Lockstep(gm, om)
    collisions = 0
    for f in synth.sequence(w):
        gs, os_, ck = ls.scan(L, w.lidar, f.points, f.T, labels=f.labels)
        d = gm.decisions(len(f.points), w.lidar.H * w.lidar.W)
        won = int((d["winner"] != np.uint64(2 ** 64 - 1)).sum())
        collisions += gs["pixel_points"] - won          # points that lost their pixel to a nearer one
    dec = ls.report()
    print("line16 jittered decisions:", dec, "collisions:", collisions)
    assert dec["points_ambiguous"] > 50            # points within 1e-3 px of a boundary (~0.4 %)
    assert collisions > 1000
    coords = om.alloc_blocks()
    rep = compare_blocks(gm, om, coords, w.voxel_size, w.frames, w.n_classes)
    print("line16 jittered voxels:", rep)
    assert rep["tainted_metric"] == 0 and rep["label_checked"] > 0.5 * rep["semantic"]
    mrep = compare_meshes(_mesh_np(gm.mesh()), om.mesh(), om, w.voxel_size)
    print("line16 jittered mesh:", mrep)
    gm.close()


@pytest.mark.slow
def test_loop64_fp16_full_size_sampled():
    """The 200-scan 64 x 2048 workload with 20-way probability vectors and FP16 storage (half
    {D, W} and half log-probabilities, FP32 arithmetic) in the benchmark's launch configuration,
    against the FP64 oracle on a seeded block sample: D, W, logP and labels within the per-voxel
    FP16 bounds (tests/gpu_compare.py), measured errors printed per quantity."""
    p = _lib()
    w = synth.loop64()
    L = _lidar(p, w.lidar)
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, storage=1)
    scene = synth.make_scene(w)
    Ts = synth.trajectory(w)
    probe = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    probe.set_track(np.zeros((0, 3), np.int32))
    fr = None
    for k in range(3):
        fr = synth.make_frame(w, scene, Ts[k], k, out=fr)
        probe.integrate(w.lidar, fr.points, fr.T, probs=fr.probs)
    cand = probe.alloc_blocks()
    rng = np.random.default_rng(2025)
    track = cand[rng.choice(len(cand), size=64, replace=False)]
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    om.set_track(track)
    ls = Lockstep(gm, om, exact_voxel_counts=False)
    fr = None
    for k in range(w.frames):
        fr = synth.make_frame(w, scene, Ts[k], k, out=fr)
        ls.scan(L, w.lidar, fr.points, fr.T, probs=fr.probs)
    assert gm.stats()["error_bits"] == 0
    have = np.array([b for b in track if om.read_block(b) is not None])
    rep = compare_blocks(gm, om, have, w.voxel_size, w.frames, w.n_classes, fp16=(w.truncation, 30.0))
    n_upd = np.concatenate([om.read_block(b)["n_upd"] for b in have])
    print("loop64 fp16 vs FP64:", rep, "decisions:", ls.report(), "updates per voxel: max", int(n_upd.max()),
          "mean", float(n_upd[n_upd > 0].mean()))
    assert rep["observed"] > 5000 and rep["tainted_metric"] == 0 and rep["label_checked"] > 1000
    gm.close()
