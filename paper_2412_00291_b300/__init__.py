"""Python binding of libsemtsdf (the C ABI in include/semtsdf.h).

Argument marshalling only: every step of the mapping path runs in the CUDA
kernels of ``_lib/libsemtsdf.so``.  PyTorch supplies device memory and
streams.  There is no CPU fallback: importing this package fails when the
library has not been built (``python paper_2412_00291_b300/build.py``).

The functions carry the C names (``map_create``, ``integrate_scan``,
``extract_mesh``, ``query_sdf`` ...); ``SemanticTSDF`` bundles them for
convenience and ``QuerySDF`` is the autograd Function of the trilinear query
(hand-written backward kernel, including the 6-DoF pose gradient).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsemtsdf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2412_00291_b300/build.py` "
                      "(there is no CPU fallback)")

import torch  # noqa: E402  (after the library check: fail fast without it)

_lib = ctypes.CDLL(LIB_PATH)

P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double

MAP_STAT_NAMES = ("valid_points", "pixel_points", "touched_blocks", "new_blocks", "voxels_updated",
                  "voxels_semantic", "dirty_blocks", "mesh_vertices", "mesh_triangles", "total_blocks",
                  "error_bits", "kernel_launches")
STATUS = {0: "MAP_OK", 1: "MAP_ERR_ARG", 2: "MAP_ERR_CUDA", 3: "MAP_ERR_CAPACITY", 4: "MAP_ERR_BAD_POSE",
          5: "MAP_ERR_TIMEOUT", 6: "MAP_ERR_STATE", 7: "MAP_ERR_NOMEM"}
MC_MAXTRI = 8
BV = 512


class MapConfig(ctypes.Structure):
    _fields_ = [("voxel_size", D), ("truncation", D), ("n_classes", I32), ("weight_mode", I32),
                ("p_hit", D), ("logp_floor", D), ("lik_floor", D), ("storage", I32), ("distance_mode", I32),
                ("max_blocks", I64), ("hash_capacity", I64), ("max_points", I64), ("max_pixels", I64),
                ("mesh_vertex_capacity", I64), ("mesh_triangle_capacity", I64)]


class LidarIntrinsics(ctypes.Structure):
    _fields_ = [("H", I32), ("W", I32), ("fov_up", D), ("fov_down", D), ("r_min", D), ("r_max", D)]


class MeshView(ctypes.Structure):
    _fields_ = [("n_vertices", I64), ("n_triangles", I64), ("positions", P), ("colors", P),
                ("vertex_keys", P), ("triangles", P), ("triangle_anchors", P)]


class ScanDesc(ctypes.Structure):
    _fields_ = [("map", P), ("lidar", LidarIntrinsics), ("points_dev", P), ("labels_dev", P), ("probs_dev", P),
                ("n", I64), ("T_world_lidar", D * 16)]


MAP_BATCH_GRAPH = 1
MAP_BATCH_AUTOTUNE = 2
MAP_BATCH_STREAMS = 4
BATCH_MAX = 48

_SIGS = {
    "map_config_default": ([P], I32),
    "map_create": ([P, P], I32),
    "map_check_scan_pose": ([P, P, P], I32),
    "map_set_decision_record": ([P, I32], I32),
    "map_set_concurrent_phases": ([P, I32], I32),
    "map_read_decision_record": ([P, P, I64, P, I64, P, I64, P, P], I32),
    "map_destroy": ([P], I32),
    "integrate_scan": ([P, P, P, P, P, I64, P, P], I32),
    "integrate_scan_host": ([P, P, P, P, P, I64, P, P], I32),
    "extract_mesh": ([P, P, P], I32),
    "map_remesh_all": ([P, P], I32),
    "map_set_incremental_mesh": ([P, I32], I32),
    "map_trav_params_default": ([P], I32),
    "map_traversability": ([P, P, P, P, P], I32),
    "map_quality": ([P, P, P, I64, D, P, P, P], I32),
    "integrate_labels_camera": ([P, P, P, P, P, P, P], I32),
    "extract_mesh_noalloc": ([P, P, P, P, P, P, I64, I64, P, P, P], I32),
    "query_sdf": ([P, P, I64, P, P, P], I32),
    "query_sdf_backward": ([P, P, P, I64, P, P, P], I32),
    "map_align_scan": ([P, P, I64, P, I32, P, P], I32),
    "map_sync": ([P, P], I32),
    "map_frame_count": ([P], I64),
    "map_frame_stats": ([P, I64, P], I32),
    "map_get_frame_stats": ([P, P, P], I32),
    "map_get_blocks": ([P, P, I64, P], I32),
    "map_read_blocks": ([P, P, I64, P, P, P, P, P], I32),
    "map_write_blocks": ([P, P, I64, P, P, P], I32),
    "map_read_gradients": ([P, P, I64, P], I32),
    "map_last_error": ([P], ctypes.c_char_p),
    "map_profile_begin": ([P, I32], I32),
    "map_profile_end": ([P, P, P, P], I32),
    "map_mc_table": ([P], I32),
    "map_palette": ([I32, P], I32),
    "map_batch_create": ([P, I32, I32, P], I32),
    "map_batch_destroy": ([P], I32),
    "map_batch_integrate": ([P, P, P], I32),
    "map_batch_sync": ([P, P], I32),
    "map_batch_config": ([P, P, P, P], I32),
    "map_batch_set_config": ([P, I32], I32),
    "map_batch_test_timeout": ([P, ctypes.c_uint64], I32),
    "map_batch_last_error": ([P], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class MapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, handle=None):
    if status != 0:
        msg = _lib.map_last_error(handle)
        raise MapError(status, msg.decode() if msg else "")


def _bcheck(status, batch=None):
    if status != 0:
        msg = _lib.map_batch_last_error(batch)
        raise MapError(status, msg.decode() if msg else "")


def _np_ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dev_ptr(t, dtype, name, shape_last=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"{name} must have shape [n, {shape_last}]")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _pose(T):
    T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(4, 4))
    return T, ctypes.c_void_p(T.ctypes.data)


def lidar_intrinsics(H, W, fov_up, fov_down, r_min=0.5, r_max=100.0) -> LidarIntrinsics:
    """Angles in radians (Sec. III-C.1 sensor model)."""
    return LidarIntrinsics(int(H), int(W), float(fov_up), float(fov_down), float(r_min), float(r_max))


# --------------------------------------------------------------------------
# C functions, one wrapper each
# --------------------------------------------------------------------------
def map_config_default(**overrides) -> MapConfig:
    cfg = MapConfig()
    _check(_lib.map_config_default(ctypes.byref(cfg)))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


def map_create(cfg: MapConfig):
    h = ctypes.c_void_p()
    _check(_lib.map_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def map_destroy(h):
    _check(_lib.map_destroy(h))


def map_check_scan_pose(cfg: MapConfig, lidar: LidarIntrinsics, T_world_lidar):
    """The pose checks integrate_scan applies, on the host without a map (MapError on failure)."""
    _, Tp = _pose(T_world_lidar)
    _check(_lib.map_check_scan_pose(ctypes.byref(cfg), ctypes.byref(lidar), Tp))


def integrate_scan(h, lidar: LidarIntrinsics, points, T_world_lidar, labels=None, probs=None, stream=None):
    n = 0 if points is None else int(points.shape[0])
    _, Tp = _pose(T_world_lidar)
    C = None if probs is None else int(probs.shape[1])
    _check(_lib.integrate_scan(h, ctypes.byref(lidar), _dev_ptr(points, torch.float32, "points", 3),
                               _dev_ptr(labels, torch.int32, "labels"),
                               _dev_ptr(probs, torch.float32, "probs", C), n, Tp, _stream(stream)), h)


def integrate_scan_host(h, lidar: LidarIntrinsics, points, T_world_lidar, labels=None, probs=None, stream=None):
    """Host (ideally pinned) buffers: numpy arrays or CPU tensors."""
    keep = []

    def hp(a, dtype):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != dtype or not a.is_contiguous():
                raise TypeError("host tensor expected")
            return ctypes.c_void_p(a.data_ptr())
        a = np.ascontiguousarray(a)
        keep.append(a)
        return _np_ptr(a)
    n = int(points.shape[0])
    _, Tp = _pose(T_world_lidar)
    _check(_lib.integrate_scan_host(h, ctypes.byref(lidar), hp(points, torch.float32), hp(labels, torch.int32),
                                    hp(probs, torch.float32), n, Tp, _stream(stream)), h)


class _CAI:
    """__cuda_array_interface__ wrapper for map-owned device arrays."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}


def _view(ptr, shape, dtype):
    typestr = {torch.float32: "<f4", torch.uint8: "|u1", torch.int64: "<i8", torch.int32: "<i4"}[dtype]
    if int(np.prod(shape)) == 0:
        return torch.zeros(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_CAI(ptr, shape, typestr), device="cuda")


def extract_mesh(h, stream=None, copy=True) -> dict:
    """Indexed mesh as CUDA tensors (copies unless copy=False; views die at the next integrate)."""
    mv = MeshView()
    _check(_lib.extract_mesh(h, ctypes.byref(mv), _stream(stream)), h)
    nv, nt = mv.n_vertices, mv.n_triangles
    out = {"positions": _view(mv.positions, (nv, 3), torch.float32),
           "colors": _view(mv.colors, (nv, 4), torch.uint8),
           "vertex_keys": _view(mv.vertex_keys, (nv,), torch.int64),
           "triangles": _view(mv.triangles, (nt, 3), torch.int32),
           "triangle_anchors": _view(mv.triangle_anchors, (nt, 3), torch.int32)}
    if copy:
        out = {k: v.clone() for k, v in out.items()}
    return out


def extract_mesh_noalloc(h, positions, colors, vertex_keys, triangles, triangle_anchors, stream=None):
    """extract_mesh into caller-owned CUDA tensors; the library allocates nothing.

    positions [V, 3] float32, colors [V, 4] uint8, vertex_keys [V] int64,
    triangles [T, 3] int32, triangle_anchors [T, 3] int32, with V and T the
    capacities.  Returns (n_vertices, n_triangles); raises MapError
    (MAP_ERR_CAPACITY, sizes in the message) when the mesh does not fit, and
    ValueError, before anything reaches the library, when the three vertex
    buffers or the two triangle buffers differ in length, or a buffer is not
    on the current CUDA device.
    """
    vbufs = dict(positions=positions, colors=colors, vertex_keys=vertex_keys)
    tbufs = dict(triangles=triangles, triangle_anchors=triangle_anchors)
    for group in (vbufs, tbufs):
        lens = {k: int(v.shape[0]) if v.dim() > 0 else -1 for k, v in group.items()}
        if len(set(lens.values())) != 1:
            raise ValueError(f"extract_mesh_noalloc: buffers of one kind must have equal lengths, got {lens}")
    cur = torch.cuda.current_device() if torch.cuda.is_available() else None
    for k, v in {**vbufs, **tbufs}.items():
        if not v.is_cuda or v.device.index != cur:
            raise ValueError(f"extract_mesh_noalloc: {k} must be on the current CUDA device (cuda:{cur}), "
                             f"not {v.device}")
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.extract_mesh_noalloc(h, _dev_ptr(positions, torch.float32, "positions", 3),
                                     _dev_ptr(colors, torch.uint8, "colors", 4),
                                     _dev_ptr(vertex_keys, torch.int64, "vertex_keys"),
                                     _dev_ptr(triangles, torch.int32, "triangles", 3),
                                     _dev_ptr(triangle_anchors, torch.int32, "triangle_anchors", 3),
                                     int(positions.shape[0]), int(triangles.shape[0]), ctypes.byref(nv),
                                     ctypes.byref(nt), _stream(stream)), h)
    return nv.value, nt.value


def map_set_decision_record(h, enable: bool):
    """Parity instrumentation: record each scan's point, pixel-winner, block and voxel decisions."""
    _check(_lib.map_set_decision_record(h, 1 if enable else 0), h)


def map_read_decision_record(h, n_points, n_pixels):
    """The last scan's recorded decisions: dict(point_pix [n], winner [H*W] uint64,
    touched [k, 3] int32, vox [k, 512] int32); synchronises the device."""
    nt = ctypes.c_int64()
    _check(_lib.map_read_decision_record(h, None, 0, None, 0, None, 0, ctypes.byref(nt), None), h)
    k = nt.value
    pp = np.zeros(max(n_points, 1), np.int32)
    wi = np.zeros(max(n_pixels, 1), np.uint64)
    tb = np.zeros((max(k, 1), 3), np.int32)
    vx = np.zeros((max(k, 1), BV), np.int32)
    _check(_lib.map_read_decision_record(h, _np_ptr(pp), n_points, _np_ptr(wi), n_pixels, _np_ptr(tb), k,
                                         ctypes.byref(nt), _np_ptr(vx)), h)
    assert nt.value == k
    return dict(point_pix=pp[:n_points], winner=wi[:n_pixels], touched=tb[:k], vox=vx[:k])


def map_set_concurrent_phases(h, concurrent: bool):
    """True (default): class update beside the re-meshing; False: after it (each phase alone)."""
    _check(_lib.map_set_concurrent_phases(h, 1 if concurrent else 0), h)


def map_remesh_all(h, stream=None):
    _check(_lib.map_remesh_all(h, _stream(stream)), h)


def map_set_incremental_mesh(h, enabled: bool):
    _check(_lib.map_set_incremental_mesh(h, 1 if enabled else 0), h)


class CameraIntrinsics(ctypes.Structure):
    _fields_ = [("width", I32), ("height", I32), ("fx", D), ("fy", D), ("cx", D), ("cy", D), ("r_max", D)]


def integrate_labels_camera(h, cam: dict, T_world_cam, labels=None, probs=None, stream=None):
    """Class update from a camera label image (CUDA tensors: labels [H, W] int32 or probs [H, W, C]
    float32).  cam: width, height, fx, fy, cx, cy, r_max.  Returns the per-pixel surface range
    ([H, W] float32 CUDA tensor, NaN where none)."""
    c = CameraIntrinsics(int(cam["width"]), int(cam["height"]), float(cam["fx"]), float(cam["fy"]),
                         float(cam["cx"]), float(cam["cy"]), float(cam.get("r_max", 50.0)))
    T = np.ascontiguousarray(T_world_cam, np.float64).reshape(16)
    rng = torch.empty((c.height, c.width), dtype=torch.float32, device="cuda")
    lp = None if labels is None else _dev_ptr(labels, torch.int32, "labels")
    pp = None if probs is None else _dev_ptr(probs, torch.float32, "probs")
    _check(_lib.integrate_labels_camera(h, ctypes.byref(c), lp, pp, _np_ptr(T), ctypes.c_void_p(rng.data_ptr()),
                                        _stream(stream)), h)
    return rng


class QualityReport(ctypes.Structure):
    _fields_ = [("re", D), ("cd", D), ("rc", D), ("miou", D), ("acc", D), ("n_map", I64), ("n_gt", I64),
                ("n_labeled", I64), ("n_correct", I64)]


def map_quality(h, n_classes, gt_points, gt_labels, trunc, stream=None) -> dict:
    """Quality of the last extracted mesh against a ground-truth cloud (CUDA tensors [n, 3] float32,
    [n] int32): dict of re, cd, rc, miou, acc, counts and the confusion matrix [gt class][vertex class]."""
    rep = QualityReport()
    conf = np.zeros((n_classes, n_classes), np.int64)
    n = int(gt_points.shape[0])
    _check(_lib.map_quality(h, _dev_ptr(gt_points, torch.float32, "gt_points", 3),
                            _dev_ptr(gt_labels, torch.int32, "gt_labels"), n, float(trunc), ctypes.byref(rep),
                            _np_ptr(conf), _stream(stream)), h)
    out = {k: getattr(rep, k) for k, _ in QualityReport._fields_}
    out["confusion"] = conf
    return out


class TravParams(ctypes.Structure):
    _fields_ = [("radius", D), ("max_height_diff", D), ("max_steepness", D), ("max_roughness", D),
                ("class_mask", ctypes.c_uint64)]


def map_traversability(h, n_vertices, radius=None, max_height_diff=None, max_steepness=None, max_roughness=None,
                       allowed_classes=None, stream=None):
    """Traversability of the last extracted mesh: (props [nv, 4] float32 CUDA tensor = height
    difference, steepness, roughness, ball size; traversable [nv] uint8).  Angles in radians;
    allowed_classes: iterable of classes (None: all)."""
    p = TravParams()
    _check(_lib.map_trav_params_default(ctypes.byref(p)))
    for k, v in (("radius", radius), ("max_height_diff", max_height_diff), ("max_steepness", max_steepness),
                 ("max_roughness", max_roughness)):
        if v is not None:
            setattr(p, k, float(v))
    if allowed_classes is not None:
        m = 0
        for c in allowed_classes:
            if 0 <= int(c) < 64:
                m |= 1 << int(c)
        p.class_mask = m
    props = torch.empty((max(n_vertices, 1), 4), dtype=torch.float32, device="cuda")
    trav = torch.empty(max(n_vertices, 1), dtype=torch.uint8, device="cuda")
    _check(_lib.map_traversability(h, ctypes.byref(p), ctypes.c_void_p(props.data_ptr()),
                                   ctypes.c_void_p(trav.data_ptr()), _stream(stream)), h)
    return props[:n_vertices], trav[:n_vertices]


def query_sdf(h, xyz, stream=None):
    xyz = xyz.contiguous()
    m = int(xyz.shape[0])
    sdf = torch.empty(m, dtype=torch.float32, device=xyz.device)
    valid = torch.empty(m, dtype=torch.uint8, device=xyz.device)
    _check(_lib.query_sdf(h, _dev_ptr(xyz, torch.float32, "xyz", 3), m, ctypes.c_void_p(sdf.data_ptr()),
                          ctypes.c_void_p(valid.data_ptr()), _stream(stream)), h)
    return sdf, valid.bool()


def query_sdf_backward(h, xyz, grad_sdf, pose_grad=None, stream=None):
    """grad_xyz [m, 3]; adds the (rho, phi) pose gradient into pose_grad (float64 [6]) when given."""
    xyz = xyz.contiguous()
    grad_sdf = grad_sdf.contiguous().float()
    m = int(xyz.shape[0])
    gx = torch.empty((m, 3), dtype=torch.float32, device=xyz.device)
    pg = None if pose_grad is None else _dev_ptr(pose_grad, torch.float64, "pose_grad")
    _check(_lib.query_sdf_backward(h, _dev_ptr(xyz, torch.float32, "xyz", 3),
                                   _dev_ptr(grad_sdf, torch.float32, "grad_sdf"), m,
                                   ctypes.c_void_p(gx.data_ptr()), pg, _stream(stream)), h)
    return gx


def map_align_scan(h, points, T0, iters=20, stream=None):
    _, T0p = _pose(T0)
    out = np.zeros((4, 4))
    _check(_lib.map_align_scan(h, _dev_ptr(points, torch.float32, "points", 3), int(points.shape[0]), T0p,
                               int(iters), _np_ptr(out), _stream(stream)), h)
    out[3] = [0.0, 0.0, 0.0, 1.0]
    return out


def map_frame_count(h) -> int:
    return int(_lib.map_frame_count(h))


def map_frame_stats(h, frame, check=True) -> dict:
    """Counters of one of the last 8 scans (waits for that scan only)."""
    out = np.zeros(16, np.int64)
    st = _lib.map_frame_stats(h, int(frame), _np_ptr(out))
    if check:
        _check(st, h)
    return dict(zip(MAP_STAT_NAMES, out[:len(MAP_STAT_NAMES)].tolist()))


def map_sync(h, stream=None):
    _check(_lib.map_sync(h, _stream(stream)), h)


def map_get_frame_stats(h, stream=None, check=True) -> dict:
    out = np.zeros(16, np.int64)
    st = _lib.map_get_frame_stats(h, _np_ptr(out), _stream(stream))
    if check:
        _check(st, h)
    return dict(zip(MAP_STAT_NAMES, out[:len(MAP_STAT_NAMES)].tolist()))


def map_get_blocks(h) -> np.ndarray:
    cnt = ctypes.c_int64()
    _check(_lib.map_get_blocks(h, None, 0, ctypes.byref(cnt)), h)
    n = cnt.value
    out = np.zeros((max(n, 1), 3), np.int32)
    _check(_lib.map_get_blocks(h, _np_ptr(out), n, ctypes.byref(cnt)), h)
    return out[:n]


def map_read_blocks(h, coords, n_classes, want_logp=True) -> dict:
    c = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
    n = len(c)
    out = dict(D=np.zeros((n, BV), np.float32), W=np.zeros((n, BV), np.float32),
               label=np.zeros((n, BV), np.uint8), found=np.zeros(n, np.uint8))
    lp = np.zeros((n, n_classes, BV), np.float32) if want_logp else None
    _check(_lib.map_read_blocks(h, _np_ptr(c), n, _np_ptr(out["D"]), _np_ptr(out["W"]), _np_ptr(lp),
                                _np_ptr(out["label"]), _np_ptr(out["found"])), h)
    out["logP"] = lp
    out["found"] = out["found"].astype(bool)
    return out


def map_read_gradients(h, coords) -> np.ndarray:
    """Gradients g_i [n][3][512] of the listed blocks (non-projective maps)."""
    c = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
    G = np.zeros((len(c), 3, BV), np.float32)
    _check(_lib.map_read_gradients(h, _np_ptr(c), len(c), _np_ptr(G)), h)
    return G


def map_write_blocks(h, coords, D, W, logP=None):
    c = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
    D = np.ascontiguousarray(D, np.float32)
    W = np.ascontiguousarray(W, np.float32)
    lp = None if logP is None else np.ascontiguousarray(logP, np.float32)
    _check(_lib.map_write_blocks(h, _np_ptr(c), len(c), _np_ptr(D), _np_ptr(W), _np_ptr(lp)), h)


PHASES = ("reset", "points", "tsdf", "semantic", "mesh")


def map_profile_begin(h, max_frames):
    _check(_lib.map_profile_begin(h, int(max_frames)), h)


def map_profile_end(h, max_frames):
    """Phase durations [frames, 5] (ms, see PHASES) and per-frame counters [frames, 16]."""
    out = np.zeros((max(int(max_frames), 1), len(PHASES)), np.float32)
    st = np.zeros((max(int(max_frames), 1), 16), np.int64)
    n = ctypes.c_int32()
    _check(_lib.map_profile_end(h, _np_ptr(out), _np_ptr(st), ctypes.byref(n)), h)
    return out[:n.value], st[:n.value]


def map_batch_create(handles, flags=MAP_BATCH_GRAPH | MAP_BATCH_AUTOTUNE):
    arr = (P * len(handles))(*[hh.value if isinstance(hh, ctypes.c_void_p) else hh for hh in handles])
    b = ctypes.c_void_p()
    _bcheck(_lib.map_batch_create(arr, len(handles), int(flags), ctypes.byref(b)))
    return b


def map_batch_destroy(b):
    _bcheck(_lib.map_batch_destroy(b))


def map_batch_integrate(b, handles, lidars, points, poses, labels=None, probs=None, stream=None):
    """One cooperative launch fuses points[i] (pose poses[i]) into handles[i] for every i."""
    n = len(handles)
    descs = (ScanDesc * n)()
    for i in range(n):
        pts = points[i]
        lab = None if labels is None else labels[i]
        pr = None if probs is None else probs[i]
        C = None if pr is None else int(pr.shape[1])
        d = descs[i]
        d.map = handles[i].value if isinstance(handles[i], ctypes.c_void_p) else handles[i]
        d.lidar = lidars[i]
        d.points_dev = _dev_ptr(pts, torch.float32, "points", 3)
        d.labels_dev = _dev_ptr(lab, torch.int32, "labels")
        d.probs_dev = _dev_ptr(pr, torch.float32, "probs", C)
        d.n = 0 if pts is None else int(pts.shape[0])
        T = np.asarray(poses[i], dtype=np.float64).reshape(16)
        for k in range(16):
            d.T_world_lidar[k] = float(T[k])
    _bcheck(_lib.map_batch_integrate(b, descs, _stream(stream)), b)


def map_batch_sync(b, stream=None):
    _bcheck(_lib.map_batch_sync(b, _stream(stream)), b)


def map_batch_config(b) -> dict:
    t, v, tuned = I32(), I32(), I32()
    _bcheck(_lib.map_batch_config(b, ctypes.byref(t), ctypes.byref(v), ctypes.byref(tuned)), b)
    return {"threads_per_block": t.value, "items_per_thread": v.value, "tuned": bool(tuned.value)}


def map_batch_set_config(b, index):
    _bcheck(_lib.map_batch_set_config(b, int(index)), b)


def map_batch_test_timeout(b, spin_limit):
    _bcheck(_lib.map_batch_test_timeout(b, int(spin_limit)), b)


def map_last_error(h=None) -> str:
    s = _lib.map_last_error(h)
    return s.decode() if s else ""


def map_mc_table() -> np.ndarray:
    t = np.full((256, MC_MAXTRI, 3), -1, np.int8)
    if _lib.map_mc_table(_np_ptr(t)) != 0:
        raise MapError(6, "marching-cubes table generation failed")
    return t


def map_palette(n_classes) -> np.ndarray:
    out = np.zeros((n_classes, 3), np.uint8)
    if _lib.map_palette(int(n_classes), _np_ptr(out)) != 0:
        raise MapError(1, "bad class count")
    return out


# --------------------------------------------------------------------------
# convenience object + autograd
# --------------------------------------------------------------------------
class SemanticTSDF:
    """A map: ``SemanticTSDF(voxel_size, truncation, n_classes, **config)``."""

    def __init__(self, voxel_size=0.1, truncation=0.3, n_classes=20, distance="projective", **cfg):
        modes = {"projective": 0, "nonprojective": 1}
        if distance not in modes:
            raise ValueError(f"distance must be one of {sorted(modes)}")
        cfg.setdefault("distance_mode", modes[distance])
        self.cfg = map_config_default(voxel_size=voxel_size, truncation=truncation, n_classes=n_classes, **cfg)
        self.h = map_create(self.cfg)
        self.n_classes = n_classes

    def close(self):
        if getattr(self, "h", None):
            map_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, lidar, points, T, labels=None, probs=None, stream=None):
        integrate_scan(self.h, lidar, points, T, labels=labels, probs=probs, stream=stream)

    def integrate_host(self, lidar, points, T, labels=None, probs=None, stream=None):
        integrate_scan_host(self.h, lidar, points, T, labels=labels, probs=probs, stream=stream)

    def frame_count(self):
        return map_frame_count(self.h)

    def frame_stats(self, frame, check=True):
        return map_frame_stats(self.h, frame, check)

    def stats(self, stream=None, check=True):
        return map_get_frame_stats(self.h, stream, check)

    def sync(self, stream=None):
        map_sync(self.h, stream)

    def blocks(self):
        return map_get_blocks(self.h)

    def read_blocks(self, coords, want_logp=True):
        return map_read_blocks(self.h, coords, self.n_classes, want_logp)

    def read_gradients(self, coords):
        return map_read_gradients(self.h, coords)

    def write_block(self, coord, D, W, logP=None):
        map_write_blocks(self.h, np.asarray(coord).reshape(1, 3), np.asarray(D).reshape(1, BV),
                         np.asarray(W).reshape(1, BV), None if logP is None else np.asarray(logP)[None])

    def write_blocks(self, coords, D, W, logP=None):
        map_write_blocks(self.h, coords, D, W, logP)

    def mesh(self, stream=None):
        return extract_mesh(self.h, stream)

    def set_concurrent_phases(self, concurrent=True):
        map_set_concurrent_phases(self.h, concurrent)

    def record_decisions(self, enable=True):
        map_set_decision_record(self.h, enable)

    def decisions(self, n_points, n_pixels):
        return map_read_decision_record(self.h, n_points, n_pixels)

    def remesh_all(self, stream=None):
        map_remesh_all(self.h, stream)

    def set_incremental_mesh(self, enabled: bool):
        map_set_incremental_mesh(self.h, enabled)

    def integrate_camera(self, cam, T_world_cam, labels=None, probs=None, stream=None):
        """Class update from a camera label image; returns the per-pixel surface range."""
        return integrate_labels_camera(self.h, cam, T_world_cam, labels=labels, probs=probs, stream=stream)

    def quality(self, gt_points, gt_labels, trunc, stream=None):
        """After mesh(): RE, Chamfer-L1, coverage, mIoU, accuracy against a ground-truth cloud."""
        return map_quality(self.h, self.n_classes, gt_points, gt_labels, trunc, stream)

    def traversability(self, n_vertices, **params):
        """After mesh(): per-vertex (props, traversable) of that mesh (see map_traversability)."""
        return map_traversability(self.h, n_vertices, **params)

    def query(self, xyz, stream=None):
        return query_sdf(self.h, xyz, stream)

    def align(self, points, T0, iters=20, stream=None):
        return map_align_scan(self.h, points, T0, iters, stream)


class QuerySDF(torch.autograd.Function):
    """sdf = D(xyz) by trilinear interpolation; backward through the CUDA kernel.

    ``QuerySDF.apply(xyz, tsdf_map)``; invalid queries return NaN with zero
    gradient.  ``pose_gradient(map, xyz, grad_sdf)`` gives the (rho, phi)
    left-perturbation gradient of the same backward.
    """

    @staticmethod
    def forward(ctx, xyz, tsdf_map):
        sdf, valid = query_sdf(tsdf_map.h, xyz)
        ctx.save_for_backward(xyz)
        ctx.tsdf_map = tsdf_map
        ctx.mark_non_differentiable(valid)
        return sdf, valid

    @staticmethod
    def backward(ctx, grad_sdf, grad_valid):
        (xyz,) = ctx.saved_tensors
        g = torch.nan_to_num(grad_sdf, nan=0.0)
        return query_sdf_backward(ctx.tsdf_map.h, xyz, g), None


def pose_gradient(tsdf_map, xyz, grad_sdf):
    pg = torch.zeros(6, dtype=torch.float64, device=xyz.device)
    query_sdf_backward(tsdf_map.h, xyz, grad_sdf, pose_grad=pg)
    return pg
