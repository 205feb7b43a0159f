"""FP16 storage form (half {D, W}, half log-probabilities, FP32 arithmetic) vs FP32 and the oracle.

Stated bounds, per voxel, from the oracle's count of that voxel's updates
(tests/gpu_compare.py, FP16_EPS): each store rounds to half an FP16 ulp
(2^-11 relative; 2^-25 absolute for subnormal weights below 2^-14), so after
n_upd distance updates |dD| <= 2 n_upd 2^-11 tau and |dW| <= n_upd (2^-11 W +
2^-25), and after n_sem class updates |dlogP| <= 2 n_sem 2^-11 |logp_floor| +
1e-3; labels agree wherever the oracle's top-two gap exceeds 0.05.  The maps
run in lockstep with the oracle (every recorded integer decision accepted),
so every voxel is compared.  Measured errors are printed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.gpu_compare import Lockstep, compare_blocks  # noqa: E402


def test_fp16_storage_line16():
    import paper_2412_00291_b300 as P
    w = synth.line16()
    L = w.lidar
    lid = P.lidar_intrinsics(L.H, L.W, L.fov_up, L.fov_down, L.r_min, L.r_max)
    kw = dict(max_blocks=32768, hash_capacity=1 << 16, max_points=32768, max_pixels=32768,
              mesh_vertex_capacity=1 << 22, mesh_triangle_capacity=1 << 23)
    g16 = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, storage=1, **kw)
    g32 = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, storage=0, **kw)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    ls = Lockstep(g16, om)
    for f in synth.sequence(w):
        ls.scan(lid, L, f.points, f.T, labels=f.labels)
        g32.integrate(lid, torch.from_numpy(f.points).cuda(), f.T, labels=torch.from_numpy(f.labels).cuda())
    s16, s32 = g16.stats(), g32.stats()
    assert s16["error_bits"] == 0 and s16["total_blocks"] == s32["total_blocks"]
    coords = om.alloc_blocks()
    rep = compare_blocks(g16, om, coords, w.voxel_size, w.frames, w.n_classes, fp16=(w.truncation, 30.0))
    a = g16.read_blocks(coords, want_logp=False)
    b = g32.read_blocks(coords, want_logp=False)
    obs = b["W"] > 0
    d32 = np.abs(a["D"] - b["D"])[obs]
    print(f"fp16 line16 vs FP64: {rep}; |dD| vs FP32 max {d32.max():.3e}")
    assert rep["tainted_metric"] == 0 and rep["label_checked"] > 10000
    assert rep["max_dD"] < 1e-3 * w.truncation * w.frames
