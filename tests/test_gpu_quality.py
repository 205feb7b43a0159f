"""Map quality metrics (Sec. IV-B.1): CUDA path vs the FP64 oracle, on a fused map and its ground truth.

The ground truth is the noise-free scans of the same trajectory by a scanner
with 8x the beams and 4x the columns, with the true classes, in the world
frame.  Tolerances: distances are FP32 norms of
exactly representable differences (relative error ~1e-7), summed per thread
in FP64, so RE, CD and RC agree to 1e-6 relative; the labelled-vertex count
and the confusion matrix are exact except for vertices whose nearest
distance lies within 1e-6 trunc of the truncation or whose two nearest
ground-truth points tie in distance with different classes (the oracle flags
both; either side may decide them differently), and the covered count of
ground-truth points likewise.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle.quality import quality as oracle_quality  # noqa: E402
from oracle.traversability import weld  # noqa: E402


def _lib():
    import paper_2412_00291_b300 as p
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ground_truth(w, n_frames, every=1, dense=(8, 4)):
    """Noise-free points (world frame, float32) and true classes of the trajectory's scans taken by
    a denser scanner (beams x dense[0], columns x dense[1], same field of view), so that the cloud
    samples the surfaces more finely than the mesh."""
    L = w.lidar
    lid = synth.Lidar(L.H * dense[0], L.W * dense[1], L.fov_up, L.fov_down, L.r_min, L.r_max)
    wg = dataclasses.replace(w, sigma=0.0, label_mode="probs", lidar=lid)
    pts, lab = [], []
    for k, f in enumerate(synth.sequence(wg, n_frames)):
        if k % every:
            continue
        ok = np.isfinite(f.points).all(axis=1)
        p = f.points[ok].astype(np.float64)
        pts.append((p @ f.T[:3, :3].T + f.T[:3, 3]).astype(np.float32))
        lab.append(f.labels[ok].astype(np.int32))
    return np.concatenate(pts), np.concatenate(lab)


def _compare(gm, w, G, lg, trunc):
    mesh = {k: v.cpu().numpy() for k, v in gm.mesh().items()}
    q = gm.quality(_dev(G), _dev(lg), trunc)
    M, lm, _, _ = weld(mesh["positions"], mesh["colors"], mesh["vertex_keys"], mesh["triangles"])
    o = oracle_quality(M, lm, G, lg, trunc, w.n_classes)
    assert q["n_map"] == o["n_map"] and q["n_gt"] == o["n_gt"]
    for k in ("re", "cd"):
        assert abs(q[k] - o[k]) <= 1e-6 * o[k] + 1e-9, (k, q[k], o[k])
    slack_m = int(o["trunc_edge"].sum() + o["label_tie"].sum())
    slack_g = int(o["gt_edge"].sum())
    assert abs(q["rc"] - o["rc"]) * o["n_gt"] <= slack_g + 1e-9
    assert abs(q["n_labeled"] - o["n_labeled"]) <= slack_m
    assert np.abs(q["confusion"] - o["confusion"]).sum() <= 2 * slack_m
    assert abs(q["acc"] - o["acc"]) <= (2 * slack_m + 1) / max(o["n_labeled"], 1)
    return q, o, slack_m


def test_quality_line16_both_distances():
    p = _lib()
    w = synth.line16()
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    G, lg = ground_truth(w, w.frames)
    trunc = 2 * w.voxel_size
    res = {}
    for mode in ("projective", "nonprojective"):
        gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, distance=mode, max_blocks=32768,
                            hash_capacity=1 << 16, max_points=32768, max_pixels=32768,
                            mesh_vertex_capacity=1 << 22, mesh_triangle_capacity=1 << 23)
        with pytest.raises(p.MapError) as e:          # nothing extracted yet
            gm.quality(_dev(G[:10]), _dev(lg[:10]), trunc)
        assert e.value.status == 6
        for f in synth.sequence(w):
            gm.integrate(L, _dev(f.points), f.T, labels=_dev(f.labels))
        q, o, slack = _compare(gm, w, G, lg, trunc)
        res[mode] = q
        print(f"line16 {mode}: RE {q['re']:.4f} m, CD {q['cd']:.4f} m, RC {q['rc']:.4f}, mIoU {q['miou']:.4f}, "
              f"Acc {q['acc']:.4f} (oracle RE {o['re']:.4f}, flagged {slack}, vertices {q['n_map']}, "
              f"ground truth {q['n_gt']})")
        assert 0.0 < q["re"] < trunc and q["rc"] > 0.5 and q["acc"] > 0.5
        gm.close()


def test_quality_argument_errors():
    p = _lib()
    w = synth.line16()
    gm = p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=4096, hash_capacity=1 << 13,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 20,
                        mesh_triangle_capacity=1 << 21)
    G = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    lg = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(p.MapError) as e:
        gm.quality(G, lg, 0.4)
    assert e.value.status == 1
    gm.close()
