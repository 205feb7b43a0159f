"""Class update from a camera label image (Sec. III-C.3): CUDA path vs the FP64 oracle.

Both maps hold the same analytic field (values rounded to FP32 and written
into both), so only the camera arithmetic differs: the GPU traverses and
projects in FP32.  Tolerances: hit ranges within 1e-4 m of the oracle's on
pixels the oracle does not flag (a traversal step with two faces within 1e-5
relative, a decisive D near 0); the updated voxel set equal except at
voxels the oracle flags (projection within 1e-3 px of a pixel boundary,
|psi| within 1e-4 m + 1e-6 range of tau, a flagged pixel); class
log-probabilities of the updated voxels within 1e-5 (FP32 log-sum-exp).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle.camera import camera_update  # noqa: E402
from tests.fields import blocks_covering, write_field  # noqa: E402

NU, TAU, C = 0.2, 0.6, 5


def _lib():
    import paper_2412_00291_b300 as p
    return p


def _field(x):
    """Ground at z = 0.074 m and a wall at x = 6.03 m facing -x, truncated: D > 0 in free space."""
    g = x[:, 2] - 0.074
    w = 6.03 - x[:, 0]
    return np.clip(np.minimum(g, w), -TAU, TAU).astype(np.float32)


def _maps(p, w_zero=None):
    blocks = blocks_covering((-2.0, -5.0, -1.0), (8.0, 5.0, 3.0), NU)
    gm = p.SemanticTSDF(NU, TAU, C, max_blocks=16384, hash_capacity=1 << 15, max_points=4096, max_pixels=4096,
                        mesh_vertex_capacity=1 << 20, mesh_triangle_capacity=1 << 21)
    om = oracle.OracleMap(NU, TAU, C)
    write_field(om, _field, blocks, NU, dtype=np.float32)
    D = np.stack([_field(np.asarray(blocks_vox(b)) * NU) for b in blocks])
    W = np.ones_like(D)
    if w_zero is not None:
        i = [tuple(b) for b in blocks].index(tuple(w_zero))
        W[i] = 0.0
        om.write_block(w_zero, D[i].astype(np.float64), np.zeros(512))
    gm.write_blocks(blocks, D, W)
    return gm, om, blocks


def blocks_vox(b):
    lz, ly, lx = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    return np.stack([lx.ravel(), ly.ravel(), lz.ravel()], axis=1) + 8 * np.asarray(b).reshape(1, 3)


def _camera(yaw_deg, pitch_deg, pos, w=80, h=60, f=60.0):
    """World-from-camera pose: forward along yaw/pitch (pitch down positive), x right, y down."""
    yaw, pitch = math.radians(yaw_deg), math.radians(pitch_deg)
    fwd = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), -math.sin(pitch)])
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = right, down, fwd, pos
    cam = dict(width=w, height=h, fx=f, fy=f, cx=(w - 1) / 2 + 0.123, cy=(h - 1) / 2 - 0.077, r_max=20.0)
    return cam, T


@pytest.mark.parametrize("mode", ["labels", "probs"])
def test_camera_update_matches_oracle(mode):
    p = _lib()
    zero_blk = (2, 0, 0)
    gm, om, blocks = _maps(p, w_zero=zero_blk)
    cam, T = _camera(8.0, 17.0, np.array([0.31, -0.23, 1.47]))
    rng = np.random.default_rng(5)
    H, Wd = cam["height"], cam["width"]
    if mode == "labels":
        lab = rng.integers(-1, C, size=(H, Wd)).astype(np.int32)      # -1: unlabelled pixel
        rg = gm.integrate_camera(cam, T, labels=torch.from_numpy(lab).cuda())
        upd, hits, pamb, vamb = camera_update(om, cam, T, labels=lab, n_classes=C, nu=NU, tau=TAU, r_max=20.0)
    else:
        q = rng.uniform(0.0, 1.0, size=(H, Wd, C)).astype(np.float32)
        q /= q.sum(axis=2, keepdims=True)
        rg = gm.integrate_camera(cam, T, probs=torch.from_numpy(q).cuda())
        upd, hits, pamb, vamb = camera_update(om, cam, T, probs=q, n_classes=C, nu=NU, tau=TAU, r_max=20.0)
    rg = rg.cpu().numpy().astype(np.float64)
    # hit ranges
    assert np.array_equal(np.isnan(rg) & ~pamb, np.isnan(hits) & ~pamb)
    ok = ~np.isnan(hits) & ~pamb
    assert ok.sum() > 0.5 * H * Wd
    dr = np.abs(rg - hits)[ok]
    assert dr.max() <= 1e-4, dr.max()
    # updated voxels and their class log-probabilities
    coords = np.array(sorted(upd))
    g = gm.read_blocks(coords)
    n_cmp, n_upd, n_flag = 0, 0, 0
    lp0 = -math.log(C)
    for i, b in enumerate(map(tuple, coords)):
        mask, lp = upd[b]
        amb = vamb[b]
        g_upd = np.abs(g["logP"][i] - lp0).max(axis=0) > 1e-6
        bad = (g_upd != mask) & ~amb
        assert not bad.any(), (b, np.flatnonzero(bad)[:8])
        both = mask & g_upd & ~amb
        d = np.abs(g["logP"][i][:, both] - lp[:, both])
        assert d.max(initial=0) <= 1e-5, d.max()
        n_cmp += int(both.sum())
        n_upd += int(mask.sum())
        n_flag += int((amb & (mask | g_upd)).sum())
        if b == zero_blk:
            assert not g_upd.any()
    st = gm.stats()
    assert abs(st["voxels_semantic"] - n_upd) <= n_flag
    print(f"camera {mode}: {int(ok.sum())} pixels with a surface (max |dr| {dr.max():.2e} m), {n_upd} voxels "
          f"updated, {n_cmp} compared, {n_flag} flagged")
    assert n_cmp > 1000


def test_camera_argument_errors():
    p = _lib()
    gm, _, _ = _maps(p)
    cam, T = _camera(0.0, 10.0, np.array([0.0, 0.0, 1.5]))
    lab = torch.zeros((cam["height"], cam["width"]), dtype=torch.int32, device="cuda")
    with pytest.raises(p.MapError) as e:                 # neither labels nor probabilities
        gm.integrate_camera(cam, T)
    assert e.value.status == 1
    bad = T.copy()
    bad[0, 0] = 2.0
    with pytest.raises(p.MapError) as e:
        gm.integrate_camera(cam, bad, labels=lab)
    assert e.value.status == 4
    cam2 = dict(cam, fx=-1.0)
    with pytest.raises(p.MapError) as e:
        gm.integrate_camera(cam2, T, labels=lab)
    assert e.value.status == 1
