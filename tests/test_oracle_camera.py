"""Pins of the oracle's semantic update from a camera label image (Sec. III-C.3)."""
import math

import numpy as np

import oracle
from oracle.camera import camera_update, traverse
from tests.fields import blocks_covering, write_field

NU, TAU, C = 0.2, 0.6, 5


def _plane_map(z0, lo=(-2.0, -4.0, -1.0), hi=(10.0, 4.0, 3.0), w_zero_block=None):
    om = oracle.OracleMap(NU, TAU, C)
    fn = lambda x: np.clip(x[:, 2] - z0, -TAU, TAU).astype(np.float32)   # free space above z0
    blocks = blocks_covering(lo, hi, NU)
    write_field(om, fn, blocks, NU, dtype=np.float32)
    if w_zero_block is not None:
        b = om.read_block(w_zero_block)
        om.write_block(w_zero_block, b["D"], np.zeros(512))
    return om


def test_traversal_matches_dense_sampling():
    rng = np.random.default_rng(1)
    for _ in range(40):
        c = rng.uniform(-1, 1, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        vox = [v for v, _ in traverse(NU, c, d, 3.0)]
        assert len(set(vox)) == len(vox)                        # each cell once
        for a, b in zip(vox, vox[1:]):                          # face neighbours, one axis per step
            assert sum(abs(p - q) for p, q in zip(a, b)) == 1
        ts = np.arange(0.0, 3.0, 1e-4)
        pts = c[None, :] + ts[:, None] * d[None, :]
        dense = np.floor(pts / NU + 0.5).astype(int)
        seq = [tuple(dense[0])]
        for q in map(tuple, dense[1:]):
            if q != seq[-1]:
                seq.append(q)
        # the dense walk may skip a cell clipped by less than 1e-4 m; every cell it meets is traversed, in order
        it = iter(vox)
        assert all(any(q == v for v in it) for q in seq)
        assert len(vox) - len(seq) <= 3


def _down_camera(cz, w=33, h=25, f=20.0):
    """Camera at a voxel centre looking straight down (-z); the centre pixel's ray runs along voxel centres."""
    R = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0]])   # x right, y down, z forward = -z
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = [4 * NU, 0.0, cz]
    cam = dict(width=w, height=h, fx=f, fy=f, cx=(w - 1) / 2, cy=(h - 1) / 2)
    return cam, T


def test_hit_range_on_a_plane():
    z0 = 0.37 * NU
    om = _plane_map(z0)
    cam, T = _down_camera(cz=10 * NU)
    _, hits, pamb, _ = camera_update(om, cam, T, labels=np.zeros((cam["height"], cam["width"]), int),
                                     n_classes=C, nu=NU, tau=TAU)
    # centre pixel: its ray passes through voxel centres, where D is the plane distance (rounded to
    # FP32 when written, 3e-8 m), so the interpolation is exact up to that rounding
    assert abs(hits[12, 16] - (10 * NU - z0)) < 1e-7
    # every pixel: within the traversal's reach of the true ray-plane distance (|dt| <= nu sqrt(3))
    for v in range(cam["height"]):
        for u in range(cam["width"]):
            d = np.array([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], 1.0])
            d /= np.linalg.norm(d)
            dw = T[:3, :3] @ d
            t_true = (z0 - T[2, 3]) / dw[2]
            assert abs(hits[v, u] - t_true) <= NU * math.sqrt(3)


def test_update_set_and_closed_form():
    z0 = 0.37 * NU
    zero_blk = (0, 0, -1)
    om = _plane_map(z0, w_zero_block=zero_blk)
    cam, T = _down_camera(cz=10 * NU)
    lab = (np.arange(cam["height"] * cam["width"]).reshape(cam["height"], cam["width"]) % C).astype(int)
    upd, hits, pamb, vamb = camera_update(om, cam, T, labels=lab, n_classes=C, nu=NU, tau=TAU)
    n_upd = 0
    for b, (mask, lp) in upd.items():
        blk = om.read_block(b)
        if b == zero_blk:
            assert not mask.any()                        # unobserved voxels are never updated
        for li in np.flatnonzero(mask):
            lx, ly, lz = li % 8, (li // 8) % 8, li // 64
            x = np.array([8 * b[0] + lx, 8 * b[1] + ly, 8 * b[2] + lz]) * NU
            assert x[2] < T[2, 3]                         # in front of the camera
            # one update of a uniform prior: the posterior is the likelihood itself
            col = np.exp(lp[:, li])
            assert abs(col.sum() - 1.0) < 1e-12
            best = int(np.argmax(lp[:, li]))
            assert abs(lp[best, li] - math.log(0.9)) < 1e-12
            n_upd += 1
        # voxels far from the plane (|D| = tau, beyond the band) are not updated
        far = np.abs(blk["D"]) >= TAU - 1e-6
        assert not (mask & far & (np.abs(blk["D"] - 0) > TAU + NU)).any()
    assert n_upd > 100
