"""FP64 CPU oracle for the mapping path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product package never does, and
the two share no code.  The oracle itself is ``oracle.cpp`` (plain C++,
FP64, ``-O2 -ffp-contract=off``); this file compiles it and wraps its C
interface with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
BV = 512


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-o", _LIB, _SRC])
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    sig = {
        "orc_new": ([D, D, I, I, D, D, D], P),
        "orc_free": ([P], None),
        "orc_set_bands": ([P, D, D], None),
        "orc_set_track": ([P, P, I64], None),
        "orc_integrate": ([P, P, P, P, P, I64, P, I, P, P, P, I64, P], I),
        "orc_check": ([P, P], None),
        "orc_block_clearance": ([P, P, P], D),
        "orc_stats": ([P, P], None),
        "orc_num_alloc": ([P], I64),
        "orc_get_alloc": ([P, P, I64], I64),
        "orc_get_touched": ([P, P, I64], I64),
        "orc_read_block": ([P, P, P, P, P, P, P, P, P, P], I),
        "orc_write_block": ([P, P, P, P, P], I),
        "orc_mesh_build": ([P, I, P, I64, P], P),
        "orc_mesh_fetch": ([P, P, P, P, P, P, P, P, P], None),
        "orc_mesh_free": ([P], None),
        "orc_edge_key": ([I64, I64, I64, I], I64),
        "orc_query": ([P, P, I64, P, P, P], None),
        "orc_pose_terms": ([P, P, I64, P, P, P, P, P], I64),
        "orc_align": ([P, P, I64, P, I, P], I),
        "orc_se3_exp": ([P, P, P], None),
        "orc_palette": ([I, P], None),
        "orc_point_blocks": ([P, P, P, P, P, I64], I64),
        "orc_point_band": ([P, P, P, P, P], D),
        "orc_set_distance_mode": ([P, I], None),
        "orc_get_normals": ([P, P, P, I64], I64),
        "orc_read_grad": ([P, P, P], I),
        "orc_nonproj_distance": ([D, P, P, P, I], D),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


STAT_NAMES = ("valid_points", "pixel_points", "ambiguous_points", "touched_blocks", "new_blocks",
              "voxels_updated", "voxels_semantic", "voxels_seen", "taint_events", "sure_blocks",
              "ambiguous_blocks")

# Candidate-acceptance counts of a scan integrated with a decision record
# (orc_check, CK_* order): for each decision kind, how many were checked, how
# many fell in the FP64 ambiguity band (the recorded choice was accepted as
# one of the FP64 candidates and used), and how many were rejected.
CHECK_NAMES = ("points", "points_ambiguous", "points_rejected",
               "pixels", "winners_ambiguous", "winners_rejected",
               "blocks_sure", "blocks_ambiguous", "blocks_ambiguous_taken", "blocks_missing", "blocks_extra",
               "voxels", "voxel_pixels_ambiguous", "voxel_pixels_rejected", "voxel_updates_ambiguous",
               "voxel_updates_rejected", "voxel_classes_ambiguous", "voxel_classes_rejected",
               "voxels_without_record")
REJECTIONS = ("points_rejected", "winners_rejected", "blocks_missing", "blocks_extra", "voxel_pixels_rejected",
              "voxel_updates_rejected", "voxel_classes_rejected", "voxels_without_record")


class OracleMap:
    """Plain FP64 mapper: one std::unordered_map of 8^3-voxel blocks."""

    def __init__(self, voxel_size, truncation, n_classes=20, weight_mode=0, p_hit=0.9,
                 logp_floor=-30.0, lik_floor=1e-6, distance="projective"):
        self.L = _load()
        self.C = n_classes
        self.h = self.L.orc_new(voxel_size, truncation, n_classes, weight_mode, p_hit, logp_floor, lik_floor)
        self.voxel_size = voxel_size
        self.distance = distance
        if distance == "nonprojective":
            self.L.orc_set_distance_mode(self.h, 1)
        elif distance != "projective":
            raise ValueError(distance)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_free(self.h)
            self.h = None

    def set_bands(self, delta_px, eps_psi):
        self.L.orc_set_bands(self.h, delta_px, eps_psi)

    def set_track(self, coords):
        c = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
        self.L.orc_set_track(self.h, _p(c), len(c))

    def integrate(self, lidar, points, T, labels=None, probs=None, nthreads=0, decisions=None):
        """Fuse one scan.  `decisions` (optional): a single-precision implementation's choices for
        this scan, a dict with point_pix [n] int32, winner [H*W] uint64, touched [k, 3] int32 and
        vox [k, 512] int32 (see orc_integrate); ambiguous FP64 decisions then follow them when they
        are FP64 candidates, and check() reports the counts."""
        lid = np.array([lidar.H, lidar.W, lidar.fov_up, lidar.fov_down, lidar.r_min, lidar.r_max], np.float64)
        pts = np.ascontiguousarray(points, np.float32)
        lab = None if labels is None else np.ascontiguousarray(labels, np.int32)
        pr = None if probs is None else np.ascontiguousarray(probs, np.float32)
        T = np.ascontiguousarray(T, np.float64)
        d = decisions or {}
        pp = None if d.get("point_pix") is None else np.ascontiguousarray(d["point_pix"], np.int32)
        wi = None if d.get("winner") is None else np.ascontiguousarray(d["winner"], np.uint64)
        tb = None if d.get("touched") is None else np.ascontiguousarray(d["touched"], np.int32).reshape(-1, 3)
        vx = None if d.get("vox") is None else np.ascontiguousarray(d["vox"], np.int32)
        if pp is not None:
            assert len(pp) == len(pts)
        if wi is not None:
            assert len(wi) == lidar.H * lidar.W
        if vx is not None:
            assert tb is not None and vx.shape == (len(tb), BV)
        if tb is not None and len(tb) == 0:          # an empty recorded set is still a record
            tb = np.zeros((1, 3), np.int32)[:0]
            tb_p = ctypes.c_void_p(np.zeros((1, 3), np.int32).ctypes.data)
            self._keep = tb_p
        else:
            tb_p = _p(tb)
        rc = self.L.orc_integrate(self.h, _p(lid), _p(pts), _p(lab), _p(pr), len(pts), _p(T), nthreads,
                                  _p(pp), _p(wi), tb_p, 0 if tb is None else len(tb),
                                  _p(vx) if vx is not None and vx.size else None)
        assert rc == 0
        return self.stats()

    def stats(self):
        out = np.zeros(len(STAT_NAMES), np.int64)
        self.L.orc_stats(self.h, _p(out))
        return dict(zip(STAT_NAMES, out.tolist()))

    def check(self):
        """Candidate-acceptance counts of the last scan (CHECK_NAMES)."""
        out = np.zeros(24, np.int64)
        self.L.orc_check(self.h, _p(out))
        return dict(zip(CHECK_NAMES, out[:len(CHECK_NAMES)].tolist()))

    def alloc_blocks(self):
        n = self.L.orc_num_alloc(self.h)
        out = np.zeros((max(n, 1), 3), np.int32)
        self.L.orc_get_alloc(self.h, _p(out), n)
        return out[:n]

    def touched_blocks(self):
        n = self.L.orc_get_touched(self.h, None, 0)
        out = np.zeros((max(n, 1), 3), np.int32)
        self.L.orc_get_touched(self.h, _p(out), n)
        return out[:n]

    def read_block(self, coord):
        c = np.ascontiguousarray(coord, np.int32)
        D = np.zeros(BV)
        W = np.zeros(BV)
        lp = np.zeros((self.C, BV))
        taint = np.zeros(BV, np.uint8)
        lab = np.zeros(BV, np.int32)
        gap = np.zeros(BV)
        nupd = np.zeros(BV, np.int32)
        nsem = np.zeros(BV, np.int32)
        rc = self.L.orc_read_block(self.h, _p(c), _p(D), _p(W), _p(lp), _p(taint), _p(lab), _p(gap), _p(nupd),
                                   _p(nsem))
        if rc != 0:
            return None
        return dict(D=D, W=W, logP=lp, taint=taint, label=lab, gap=gap, n_upd=nupd, n_sem=nsem)

    def read_grad(self, coord):
        """Gradient g_i of one block's voxels, [3][512] (non-projective mode), or None."""
        c = np.ascontiguousarray(coord, np.int32)
        G = np.zeros((3, BV))
        return G if self.L.orc_read_grad(self.h, _p(c), _p(G)) == 0 else None

    def normals(self):
        """The last scan's normal image (world frame) [H*W][3] and its flags (bit 0 valid, bit 1 near-ambiguous)."""
        n = self.L.orc_get_normals(self.h, None, None, 0)
        N = np.zeros((max(n, 1), 3))
        f = np.zeros(max(n, 1), np.uint8)
        self.L.orc_get_normals(self.h, _p(N), _p(f), n)
        return N[:n], f[:n]

    def write_block(self, coord, D, W, logP=None):
        c = np.ascontiguousarray(coord, np.int32)
        D = np.ascontiguousarray(D, np.float64)
        W = np.ascontiguousarray(W, np.float64)
        lp = None if logP is None else np.ascontiguousarray(logP, np.float64)
        self.L.orc_write_block(self.h, _p(c), _p(D), _p(W), _p(lp))

    def mesh(self, blocks=None):
        counts = np.zeros(2, np.int64)
        if blocks is None:
            hm = self.L.orc_mesh_build(self.h, 0, None, 0, _p(counts))
        else:
            b = np.ascontiguousarray(blocks, np.int32).reshape(-1, 3)
            hm = self.L.orc_mesh_build(self.h, 1, _p(b), len(b), _p(counts))
        nv, nt = int(counts[0]), int(counts[1])
        out = dict(vkey=np.zeros(nv, np.int64), vpos=np.zeros((nv, 3)), vlab=np.zeros(nv, np.int32),
                   vgap=np.zeros(nv), vtaint=np.zeros(nv, np.uint8), tkeys=np.zeros((nt, 3), np.int64),
                   tanchor=np.zeros((nt, 3), np.int32), ttaint=np.zeros(nt, np.uint8))
        if nv or nt:
            self.L.orc_mesh_fetch(hm, *(_p(out[k]) if out[k].size else None for k in
                                       ("vkey", "vpos", "vlab", "vgap", "vtaint", "tkeys", "tanchor", "ttaint")))
        self.L.orc_mesh_free(hm)
        return out

    def query(self, xyz):
        x = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        sdf = np.zeros(len(x))
        valid = np.zeros(len(x), np.uint8)
        grad = np.zeros((len(x), 3))
        self.L.orc_query(self.h, _p(x), len(x), _p(sdf), _p(valid), _p(grad))
        return sdf, valid.astype(bool), grad

    def pose_terms(self, points, T):
        pts = np.ascontiguousarray(points, np.float32)
        T = np.ascontiguousarray(T, np.float64)
        loss = np.zeros(1)
        dL = np.zeros(6)
        H = np.zeros((6, 6))
        g = np.zeros(6)
        nv = self.L.orc_pose_terms(self.h, _p(pts), len(pts), _p(T), _p(loss), _p(dL), _p(H), _p(g))
        return dict(loss=float(loss[0]), dL=dL, H=H, g=g, n_valid=int(nv))

    def align(self, points, T0, iters=20):
        pts = np.ascontiguousarray(points, np.float32)
        T0 = np.ascontiguousarray(T0, np.float64)
        out = np.zeros((4, 4))
        rc = self.L.orc_align(self.h, _p(pts), len(pts), _p(T0), iters, _p(out))
        assert rc == 0
        return out

    def point_blocks(self, pt, T):
        """Band blocks of one point: (sure [k, 3], ambiguous [j, 3]) by the FP64 clearance test."""
        p = np.ascontiguousarray(pt, np.float32)
        T = np.ascontiguousarray(T, np.float64)
        out = np.zeros((256, 3), np.int32)
        cls = np.zeros(256, np.int8)
        n = self.L.orc_point_blocks(self.h, _p(p), _p(T), _p(out), _p(cls), 256)
        assert n <= 256
        return out[:n][cls[:n] == 1], out[:n][cls[:n] == 0]

    def point_band(self, pt, T):
        """FP64 band endpoints (voxel units + 1/2) of one point and the ambiguity margin."""
        p = np.ascontiguousarray(pt, np.float32)
        T = np.ascontiguousarray(T, np.float64)
        e0 = np.zeros(3)
        e1 = np.zeros(3)
        margin = self.L.orc_point_band(self.h, _p(p), _p(T), _p(e0), _p(e1))
        return e0, e1, float(margin)


def nonprojective_distance(psi, u, g, N=None) -> float:
    """d_i of Eq. (distance) for projective distance psi, unit ray u (voxel toward sensor), gradient g, normal N."""
    u = np.ascontiguousarray(u, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    n = np.zeros(3) if N is None else np.ascontiguousarray(N, np.float64)
    return float(_load().orc_nonproj_distance(float(psi), _p(u), _p(g), _p(n), 0 if N is None else 1))


def edge_key(x, y, z, axis) -> int:
    return int(_load().orc_edge_key(int(x), int(y), int(z), int(axis)))


def se3_exp(xi):
    xi = np.ascontiguousarray(xi, np.float64)
    R = np.zeros(9)
    t = np.zeros(3)
    _load().orc_se3_exp(_p(xi), _p(R), _p(t))
    T = np.eye(4)
    T[:3, :3] = R.reshape(3, 3)
    T[:3, 3] = t
    return T


def block_clearance(e0, e1, b) -> float:
    """Clearance (voxel units) of block b from the segment e0 -> e1 (positive: runs through it)."""
    a = np.ascontiguousarray(e0, np.float64)
    c = np.ascontiguousarray(e1, np.float64)
    bb = np.ascontiguousarray(b, np.int32)
    return float(_load().orc_block_clearance(_p(a), _p(c), _p(bb)))


def palette(C):
    out = np.zeros((C, 3), np.uint8)
    _load().orc_palette(C, _p(out))
    return out
