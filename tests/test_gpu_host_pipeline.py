"""integrate_scan_host as a pipelined serving loop: scan k's upload overlaps scan k-1's kernels
(two staging sets, copy stream), and map_frame_stats reads one scan's counters without waiting for
later scans.  The result must equal the device-buffer path exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402

COUNTERS = ("valid_points", "pixel_points", "touched_blocks", "new_blocks", "voxels_updated", "voxels_semantic",
            "mesh_vertices", "mesh_triangles", "total_blocks", "error_bits")


def _map(P, w):
    return P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                          max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                          mesh_triangle_capacity=1 << 23)


def test_pipelined_host_path_matches_device_path():
    import paper_2412_00291_b300 as P
    w = synth.line16()
    L = P.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    frames = list(synth.sequence(w, 6))
    a, b = _map(P, w), _map(P, w)
    ref = []
    for f in frames:
        a.integrate(L, torch.from_numpy(f.points).cuda(), f.T, labels=torch.from_numpy(f.labels).cuda())
        ref.append(a.stats())
    # host path: every scan issued before the previous scan's counters are read
    host = [(torch.from_numpy(f.points).pin_memory(), torch.from_numpy(f.labels).pin_memory()) for f in frames]
    got = []
    for k, f in enumerate(frames):
        b.integrate_host(L, host[k][0], f.T, labels=host[k][1])
        if k > 0:
            got.append(b.frame_stats(k - 1))
    got.append(b.frame_stats(len(frames) - 1))
    assert b.frame_count() == len(frames)
    for k, (r, g) in enumerate(zip(ref, got)):
        for name in COUNTERS:
            assert r[name] == g[name], (k, name, r[name], g[name])
    ca = np.asarray(sorted(map(tuple, a.blocks().tolist())))
    cb = np.asarray(sorted(map(tuple, b.blocks().tolist())))
    assert np.array_equal(ca, cb)
    ra, rb = a.read_blocks(ca), b.read_blocks(ca)
    for key in ("D", "W", "label", "logP"):
        assert np.array_equal(ra[key].view(np.uint8), rb[key].view(np.uint8)), key
    with pytest.raises(P.MapError) as e:
        b.frame_stats(len(frames))          # not integrated yet
    assert e.value.status == 1
    a.close()
    b.close()
