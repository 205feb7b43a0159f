"""Per-phase profiling (map_profile_begin / map_profile_end) through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


def test_profile_phases_and_counters():
    import paper_2412_00291_b300 as P
    w = synth.line16()
    L = P.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    m = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                       max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                       mesh_triangle_capacity=1 << 23)
    frames = list(synth.sequence(w, 4))
    m.integrate(L, torch.from_numpy(frames[0].points).cuda(), frames[0].T,
                labels=torch.from_numpy(frames[0].labels).cuda())
    P.map_profile_begin(m.h, 8)
    per = []
    for f in frames[1:]:
        m.integrate(L, torch.from_numpy(f.points).cuda(), f.T, labels=torch.from_numpy(f.labels).cuda())
        per.append(m.stats())
    ms, st = P.map_profile_end(m.h, 8)
    assert ms.shape == (3, len(P.PHASES)) and st.shape == (3, 16)
    assert np.all(ms >= 0) and np.all(ms[:, 1:].sum(axis=1) > 0)
    names = P.MAP_STAT_NAMES
    for k in range(3):
        for j, name in enumerate(names[:9]):
            assert st[k, j] == per[k][name], (k, name)
    m.close()
