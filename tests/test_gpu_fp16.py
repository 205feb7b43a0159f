"""FP16 storage form (half {D, W}, half log-probabilities, FP32 arithmetic) vs FP32 and the oracle.

Stated bound for D: each update rounds the stored D once (at most half an
FP16 ulp, 2^-11 |D| <= 2^-11 tau) and earlier rounding errors are carried
with weight W / (W + w) < 1, so after K updates |dD| <= K 2^-11 tau (plus
the FP32 path's 1e-4 nu).  W: each store rounds to half an ulp, relative
2^-11 for normal values and absolute 2^-25 in the subnormal range below
2^-14 (tiny weights of voxels observed at psi close to -tau), so
|dW| <= K (2^-11 W + 2^-25).  Labels must agree wherever the oracle's top-two gap
exceeds 2e-2 (FP16 log-probabilities near -30 have a 2^-6 grid).  Measured
errors are printed and must sit well inside these bounds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402


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
    for f in synth.sequence(w):
        pts, lab = torch.from_numpy(f.points).cuda(), torch.from_numpy(f.labels).cuda()
        g16.integrate(lid, pts, f.T, labels=lab)
        g32.integrate(lid, pts, f.T, labels=lab)
        om.integrate(L, f.points, f.T, labels=f.labels)
    s16, s32 = g16.stats(), g32.stats()
    assert s16["error_bits"] == 0 and s16["total_blocks"] == s32["total_blocks"]
    coords = om.alloc_blocks()
    a = g16.read_blocks(coords)
    b = g32.read_blocks(coords)
    K = w.frames
    dD16, dD32, dW16, agree, checked = [], [], [], 0, 0
    for i, c in enumerate(coords):
        o = om.read_block(c)
        clean = o["taint"] == 0
        obs = clean & (o["W"] > 0)
        assert np.array_equal(a["W"][i][clean] > 0, o["W"][clean] > 0)
        dD16.append(np.abs(a["D"][i] - o["D"])[obs])
        dD32.append(np.abs(a["D"][i] - b["D"][i])[obs])
        dW16.append((np.abs(a["W"][i] - o["W"]) / (2.0 ** -11 * o["W"] + 2.0 ** -25))[obs])
        sure = obs & (o["gap"] > 2e-2)
        agree += int((a["label"][i][sure] == o["label"][sure]).sum())
        checked += int(sure.sum())
    dD16, dD32, dW16 = map(np.concatenate, (dD16, dD32, dW16))
    bound_D = K * 2.0 ** -11 * w.truncation + 1e-4 * w.voxel_size
    print(f"fp16: max|dD| vs FP64 {dD16.max():.3e} (p99 {np.percentile(dD16, 99):.3e}), vs FP32 {dD32.max():.3e}; "
          f"bound {bound_D:.3e}; max dW in units of the per-store bound {dW16.max():.2f}; "
          f"label agreement {agree}/{checked}")
    assert dD16.max() <= bound_D
    assert dW16.max() <= K
    assert agree == checked
    assert dD16.max() < 1e-3 * w.truncation * K
