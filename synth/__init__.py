"""Seeded synthetic LiDAR workloads (scenes, trajectories, scans, labels).

Input generation only: nothing here computes any step of the mapping
method.  The FP64 oracle tests, the CUDA parity tests and ``bench.py`` all
draw their inputs from this module, so both sides see the same scans.

The paper evaluates on public LiDAR datasets (SemanticKITTI, SemanticUSL,
FusionPortable; Sec. IV-B) which are not available here.  The scenes below
stand in for them with the same sensor geometry: a spinning multi-beam LiDAR
whose points sit on a regular (beam, column) grid (Sec. III-C.1, the range
image equation), driven through a seeded scene of ground, boxes, cylinders and
sloped ground patches, with per-point labels or class-probability vectors.

Sensor model (shared by generator and mapper, restating the range-image
equation of Sec. III-C.1): pixel (v, u) has polar angle
``theta0 + v * dtheta`` with ``theta0 = pi/2 - fov_up`` and
``dtheta = (fov_up - fov_down) / (H - 1)``, and azimuth ``pi - u * dphi`` with
``dphi = 2 pi / W``.  Generated points lie on their own pixel's centre ray,
perturbed along the ray by Gaussian range noise; a workload with ``jitter``
> 0 also turns each ray by normal angular offsets (``jitter`` pixels std in
both angles), so that points fall off their pixel's centre ray, some near
pixel boundaries, some pixels receive two points and some none.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raycast.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the ray caster (gcc, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.synth_raycast.argtypes = [P, P, ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int,
                                      ctypes.c_int, P, P, ctypes.c_long, ctypes.c_double,
                                      ctypes.c_double, P, P, ctypes.c_int]
        lib.synth_raycast.restype = ctypes.c_int
        lib.synth_scan.argtypes = [P, P, ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                   P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                   P, P, P, P, P, ctypes.c_int, ctypes.c_double]
        lib.synth_scan.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


# --------------------------------------------------------------------------
# sensor
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Lidar:
    H: int
    W: int
    fov_up: float          # radians, elevation of beam 0
    fov_down: float        # radians, elevation of beam H-1
    r_min: float = 0.5
    r_max: float = 100.0

    @property
    def dphi(self) -> float:
        return 2.0 * math.pi / self.W

    @property
    def dtheta(self) -> float:
        return (self.fov_up - self.fov_down) / (self.H - 1)

    @property
    def theta0(self) -> float:
        return math.pi / 2.0 - self.fov_up

    def ray_dirs(self) -> np.ndarray:
        """Unit centre-ray directions in the LiDAR frame, [H*W, 3] float64, row-major (v, u)."""
        v = np.arange(self.H, dtype=np.float64)[:, None]
        u = np.arange(self.W, dtype=np.float64)[None, :]
        th = self.theta0 + v * self.dtheta
        ph = math.pi - u * self.dphi
        st = np.sin(th)
        d = np.stack(np.broadcast_arrays(st * np.cos(ph), st * np.sin(ph), np.cos(th)), axis=-1)
        return np.ascontiguousarray(d.reshape(-1, 3))


def lidar_deg(H, W, fov_up_deg, fov_down_deg, r_max, r_min=0.5) -> Lidar:
    return Lidar(H, W, math.radians(fov_up_deg), math.radians(fov_down_deg), r_min, r_max)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------
@dataclass
class Scene:
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))   # lo xyz, hi xyz
    box_cls: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cyls: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))    # cx, cy, r, h
    cyl_cls: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ramps: np.ndarray = field(default_factory=lambda: np.zeros((0, 7)))   # cx, cy, hx, hy, z0, gx, gy
    ramp_cls: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ground_cls: int = 0

    def cast(self, origin, dirs_world: np.ndarray, t_max: float, nthreads: int = 0):
        """Nearest-hit distance (inf = no hit) and class (-1 = no hit) for each ray."""
        lib = _load()
        n = dirs_world.shape[0]
        dirs_world = np.ascontiguousarray(dirs_world, dtype=np.float64)
        t = np.empty(n, np.float64)
        c = np.empty(n, np.int32)
        b = np.ascontiguousarray(self.boxes, np.float64)
        bc = np.ascontiguousarray(self.box_cls, np.int32)
        cy = np.ascontiguousarray(self.cyls, np.float64)
        cc = np.ascontiguousarray(self.cyl_cls, np.int32)
        r = np.ascontiguousarray(self.ramps, np.float64)
        rc = np.ascontiguousarray(self.ramp_cls, np.int32)
        o = np.ascontiguousarray(origin, np.float64)
        lib.synth_raycast(_ptr(b), _ptr(bc), len(b), _ptr(cy), _ptr(cc), len(cy), _ptr(r), _ptr(rc), len(r),
                          int(self.ground_cls), _ptr(o), _ptr(dirs_world), n, float(t_max), 4.0,
                          _ptr(t), _ptr(c), int(nthreads))
        return t, c


def _footprint_clear(kind, p, path_dist, corridor):
    """True when the primitive's xy footprint stays `corridor` metres away from the path."""
    if kind == 0:
        cx, cy = (p[0] + p[3]) / 2, (p[1] + p[4]) / 2
        rad = math.hypot(p[3] - p[0], p[4] - p[1]) / 2
    elif kind == 1:
        cx, cy, rad = p[0], p[1], p[2]
    else:
        cx, cy = p[0], p[1]
        rad = math.hypot(p[2], p[3])
    return path_dist(cx, cy) - rad >= corridor


def _random_prims(rng, n_box, n_cyl, xr, yr, n_cls, path_dist, corridor, n_ramp=0, mixed=None):
    boxes, bcls, cyls, ccls, ramps, rcls = [], [], [], [], [], []
    kinds = [0] * n_box + [1] * n_cyl
    if mixed is not None:   # n primitives, each a box or a cylinder with p = 1/2
        kinds = [int(k) for k in (rng.random(mixed) < 0.5)]
    for kind in kinds:
        while True:
            cx, cy = rng.uniform(*xr), rng.uniform(*yr)
            if kind == 0:
                sx, sy, sz = rng.uniform(1.0, 5.0, size=3)
                p = [cx - sx / 2, cy - sy / 2, 0.0, cx + sx / 2, cy + sy / 2, sz]
            else:
                p = [cx, cy, rng.uniform(0.3, 1.0), rng.uniform(2.0, 8.0)]
            if _footprint_clear(kind, p, path_dist, corridor):
                break
        cls = int(rng.integers(1, n_cls))
        (boxes if kind == 0 else cyls).append(p)
        (bcls if kind == 0 else ccls).append(cls)
    for _ in range(n_ramp):
        while True:
            cx, cy = rng.uniform(*xr), rng.uniform(*yr)
            hx, hy = rng.uniform(2.5, 10.0, size=2)
            slope = math.radians(rng.uniform(0.0, 10.0))
            az = rng.uniform(0.0, 2 * math.pi)
            g = math.tan(slope)
            p = [cx, cy, hx, hy, rng.uniform(0.0, 1.0), g * math.cos(az), g * math.sin(az)]
            if _footprint_clear(2, p, path_dist, corridor):
                break
        ramps.append(p)
        rcls.append(0)
    return Scene(np.array(boxes, np.float64).reshape(-1, 6), np.array(bcls, np.int32),
                 np.array(cyls, np.float64).reshape(-1, 4), np.array(ccls, np.int32),
                 np.array(ramps, np.float64).reshape(-1, 7), np.array(rcls, np.int32), 0)


def rot_rpy(roll, pitch, yaw) -> np.ndarray:
    cr, sr, cp, sp, cyw, syw = (math.cos(roll), math.sin(roll), math.cos(pitch), math.sin(pitch),
                                math.cos(yaw), math.sin(yaw))
    Rz = np.array([[cyw, -syw, 0], [syw, cyw, 0], [0, 0, 1.0]])
    Ry = np.array([[cp, 0, sp], [0, 1.0, 0], [-sp, 0, cp]])
    Rx = np.array([[1.0, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return Rz @ Ry @ Rx


def pose(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    lidar: Lidar
    sigma: float
    frames: int
    voxel_size: float
    truncation: float
    n_classes: int
    label_mode: str        # "hard" or "probs"
    scene_kind: str        # "line", "loop", "drive"
    seed: int
    n_prims: int = 0
    extent: float = 0.0
    jitter: float = 0.0    # angular offset of each ray, std in pixels (0: points on the centre rays)


def line16() -> Workload:
    """10 scans, 16 x 1024, +-15 deg, 50 m, sigma 2 cm, straight drive, hard labels, 0.2 m voxels."""
    return Workload("scan16x1024_line10_v0.2", lidar_deg(16, 1024, 15.0, -15.0, 50.0), 0.02, 10,
                    0.2, 0.6, 20, "hard", "line", 1)


def line16_jitter() -> Workload:
    """line16 with each ray turned by N(0, 0.35 px) in both angles (points off the pixel centres)."""
    from dataclasses import replace
    return replace(line16(), name="scan16x1024_line10_v0.2_jitter", jitter=0.35)


def loop64() -> Workload:
    """200 scans, 64 x 2048, +-22.5 deg, 100 m, sigma 3 cm, 400 m loop, 20-way probabilities, 0.1 m voxels."""
    return Workload("scan64x2048_loop200_v0.1", lidar_deg(64, 2048, 22.5, -22.5, 100.0), 0.03, 200,
                    0.1, 0.3, 20, "probs", "loop", 2, n_prims=2000, extent=200.0)


def drive1km(seed: int = 5) -> Workload:
    """Large map for scan-to-map alignment: the 64 x 2048 scanner (+-22.5 deg, 100 m, sigma 3 cm)
    on a gently winding 960 m drive through a seeded 1 km x 1 km scene of 50,000 boxes/cylinders
    (the density of the 200 m loop scene) and 1,000 sloped patches; 480 poses 2 m apart, hard
    labels, 0.1 m voxels, 0.3 m truncation."""
    return Workload("scan64x2048_drive1km_v0.1", lidar_deg(64, 2048, 22.5, -22.5, 100.0), 0.03, 480,
                    0.1, 0.3, 20, "hard", "drive", seed, n_prims=50000, extent=1000.0)


def streams32(seed: int = 3, n_streams: int = 32) -> list[Workload]:
    """Independent map streams of uneven size for the batched form (50 frames of each are used).

    Per stream: beams from {16, 32, 64, 128}, columns from {512, 1024, 2048},
    voxel size from {0.05, 0.1, 0.2, 0.4} m (uniform draws), truncation 3 x
    voxel, +-22.5 deg, 100 m, sigma 3 cm, 20-way class-probability vectors,
    its own seeded 200 m x 200 m scene of 2,000 primitives on the 400 m loop
    (200 poses per lap, 2 m apart, as in the 64 x 2048 workload).
    """
    rng = np.random.default_rng([seed, 13])
    out = []
    for i in range(n_streams):
        H = int(rng.choice([16, 32, 64, 128]))
        W = int(rng.choice([512, 1024, 2048]))
        v = float(rng.choice([0.05, 0.1, 0.2, 0.4]))
        out.append(Workload(f"stream{i}_{H}x{W}_v{v}", lidar_deg(H, W, 22.5, -22.5, 100.0), 0.03, 200,
                            v, 3.0 * v, 20, "probs", "loop", 1000 * seed + i, n_prims=2000, extent=200.0))
    return out


LOOP_RADIUS = 400.0 / (2.0 * math.pi)


def make_scene(w: Workload) -> Scene:
    rng = np.random.default_rng([w.seed, 7])
    if w.scene_kind == "line":
        def dist(x, y):
            xc = min(max(x, 0.0), float(w.frames - 1))
            return math.hypot(x - xc, y)
        return _random_prims(rng, 20, 10, (-20.0, 40.0), (-25.0, 25.0), w.n_classes, dist, 3.0)
    if w.scene_kind == "loop":
        half = w.extent / 2

        def dist(x, y):
            return abs(math.hypot(x, y) - LOOP_RADIUS)
        return _random_prims(rng, 0, 0, (-half, half), (-half, half), w.n_classes, dist, 4.0,
                             n_ramp=40, mixed=w.n_prims)
    if w.scene_kind == "drive":
        half = w.extent / 2

        def dist(x, y):
            return abs(y - drive_y(x, w.seed))
        return _random_prims(rng, 0, 0, (-half, half), (-half, half), w.n_classes, dist, 4.0,
                             n_ramp=w.n_prims // 50, mixed=w.n_prims)
    raise ValueError(w.scene_kind)


def drive_y(x, seed):
    """Lateral offset of the gently winding drive used by the large-map workload."""
    a = 0.5 + 0.25 * ((seed * 2654435761) % 1000) / 1000.0
    return 20.0 * math.sin(a * x / 100.0)


def trajectory(w: Workload, n_frames: int | None = None) -> list[np.ndarray]:
    """World-from-LiDAR poses (4x4 float64), one per frame; small seeded roll/pitch."""
    n = w.frames if n_frames is None else n_frames
    rng = np.random.default_rng([w.seed, 11])
    out = []
    for k in range(n):
        roll, pitch = np.radians(rng.uniform(-2.0, 2.0, size=2))
        if w.scene_kind == "line":
            R = rot_rpy(roll, pitch, 0.0)
            t = np.array([k * 1.0, 0.0, 1.8])
        elif w.scene_kind == "loop":
            a = 2.0 * math.pi * (k % w.frames) / w.frames
            R = rot_rpy(roll, pitch, a + math.pi / 2)
            t = np.array([LOOP_RADIUS * math.cos(a), LOOP_RADIUS * math.sin(a), 1.8])
        else:
            x = -w.extent / 2 + 20.0 + 2.0 * k
            dy = (drive_y(x + 0.01, w.seed) - drive_y(x - 0.01, w.seed)) / 0.02
            R = rot_rpy(roll, pitch, math.atan(dy))
            t = np.array([x, drive_y(x, w.seed), 1.8])
        out.append(pose(R, t))
    return out


@dataclass
class Frame:
    points: np.ndarray     # [N, 3] float32, LiDAR frame, NaN = no return
    labels: np.ndarray     # [N] int32: per-point label (hard mode) or true class (probs mode); -1 = no return
    probs: np.ndarray | None   # [N, C] float32 or None
    T: np.ndarray          # [4, 4] float64 world-from-LiDAR
    true_range: np.ndarray  # [N] float64 analytic hit distance (inf = none)
    true_cls: np.ndarray    # [N] int32


def make_frame(w: Workload, scene: Scene, T: np.ndarray, k: int, dirs_l=None, nthreads: int = 0,
               out: Frame | None = None) -> Frame:
    """Ray-cast scan k and draw its noise and labels from counter-based streams keyed by (seed, k, pixel).

    `out` lets a caller reuse the arrays of an earlier frame.
    """
    lib = _load()
    L = w.lidar
    n, C = L.H * L.W, w.n_classes
    if out is None:
        out = Frame(np.empty((n, 3), np.float32), np.empty(n, np.int32),
                    np.empty((n, C), np.float32) if w.label_mode == "probs" else None,
                    T, np.empty(n, np.float64), np.empty(n, np.int32))
    out.T = np.array(T, np.float64)
    R = np.ascontiguousarray(T[:3, :3], np.float64)
    t = np.ascontiguousarray(T[:3, 3], np.float64)
    sc = scene
    b = np.ascontiguousarray(sc.boxes, np.float64)
    bc = np.ascontiguousarray(sc.box_cls, np.int32)
    cy = np.ascontiguousarray(sc.cyls, np.float64)
    cc = np.ascontiguousarray(sc.cyl_cls, np.int32)
    r = np.ascontiguousarray(sc.ramps, np.float64)
    rc = np.ascontiguousarray(sc.ramp_cls, np.int32)
    lib.synth_scan(_ptr(b), _ptr(bc), len(b), _ptr(cy), _ptr(cc), len(cy), _ptr(r), _ptr(rc), len(r),
                   int(sc.ground_cls), _ptr(R), _ptr(t), L.H, L.W, L.theta0, L.dtheta, L.dphi, L.r_max,
                   w.sigma, C, 0 if w.label_mode == "hard" else 1, 0.1, w.seed, k,
                   _ptr(out.points), _ptr(out.labels), _ptr(out.probs) if out.probs is not None else None,
                   _ptr(out.true_range), _ptr(out.true_cls), int(nthreads), float(w.jitter))
    return out


def sequence(w: Workload, n_frames: int | None = None, nthreads: int = 0):
    """Yield the workload's frames in order (frame k >= w.frames repeats the loop)."""
    scene = make_scene(w)
    for k, T in enumerate(trajectory(w, n_frames)):
        yield make_frame(w, scene, T, k, nthreads=nthreads)
