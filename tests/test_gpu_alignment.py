"""Scan-to-map alignment on the 1 km drive map: the slow-converging scan explained.

From a 0.5 m / 5 deg perturbation most of a scan's points start outside the
truncation band (|D| <= tau = 0.3 m around surfaces), where the fused distance
gives no gradient, so Gauss-Newton on sum D(T p)^2 is driven by the near
points only and some scans need more than 20 iterations.  This test takes
the scan the alignment benchmark reports as its worst (scan 60 of the drive,
the eleventh of its 21 scans, with the fewest points inside the band at the
start) and checks that (1) after 20 iterations it is still ~0.5 deg off,
(2) after 50 it reaches the optimum the other scans reach (within 0.05 deg),
and (3) the FP64 oracle's Gauss-Newton, on a copy of the same map and the
scan's points within 55 m, from the same start, follows the same path: after
20 iterations both poses agree to 1 mm and 0.05 deg.  The residual after 20
iterations is therefore the method's (a start outside the truncation basin),
not the arithmetic's.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import oracle  # noqa: E402
import synth  # noqa: E402


def _axis_angle(a, theta):
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(theta) * K + (1.0 - math.cos(theta)) * (K @ K)


def _rot_deg(Ra, Rb):
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return math.degrees(math.acos(min(1.0, max(-1.0, c))))


def test_slow_scan_converges_and_matches_fp64_path():
    import paper_2412_00291_b300 as P
    dev = torch.device("cuda", 0)
    w = synth.drive1km(seed=5)
    L = w.lidar
    lid = P.lidar_intrinsics(L.H, L.W, L.fov_up, L.fov_down, L.r_min, L.r_max)
    nb = 1 << 18
    m = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, storage=1, max_blocks=nb, hash_capacity=4 * nb,
                       mesh_vertex_capacity=32 << 20, mesh_triangle_capacity=64 << 20)
    scene = synth.make_scene(w)
    Ts = synth.trajectory(w, w.frames)
    K_SCAN, I_PICK = 60, 10
    pts = T = None
    for k in range(w.frames):
        f = synth.make_frame(w, scene, Ts[k], k)
        m.integrate(lid, torch.from_numpy(f.points).to(dev), f.T, labels=torch.from_numpy(f.labels).to(dev))
        if k == K_SCAN:
            ok = np.isfinite(f.points).all(axis=1)
            pts, T = f.points[ok].copy(), f.T.copy()
        if m.stats()["total_blocks"] >= 78125:
            break
    assert k == 110 and pts is not None           # the benchmark's map: 111 scans, ~40 M voxels
    # the benchmark's perturbation of its eleventh scan (random direction and axis, same stream)
    rng = np.random.default_rng([w.seed, 17])
    for _ in range(I_PICK + 1):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
    dT = np.eye(4)
    dT[:3, :3] = _axis_angle(a, math.radians(5.0))
    dT[:3, 3] = 0.5 * d
    T0 = T @ dT
    pd = torch.from_numpy(pts).to(dev)
    T20 = m.align(pd, T0, iters=20)
    T50 = m.align(pd, T0, iters=50)
    r20, r50 = _rot_deg(T20[:3, :3], T[:3, :3]), _rot_deg(T50[:3, :3], T[:3, :3])
    t50 = float(np.linalg.norm(T50[:3, 3] - T[:3, 3]))
    print(f"scan {K_SCAN}: 20 iterations {r20:.3f} deg, 50 iterations {r50:.3f} deg / {t50:.3f} m")
    assert r20 > 0.3                      # still converging after 20 iterations
    assert r50 < 0.05 and t50 < 0.06      # the optimum the other scans reach (~4 cm map offset)
    # the same start, the scan's points within 55 m, on an FP64 copy of the map around the sensor
    coords = m.blocks()
    c = (coords.astype(np.float64) + 0.5) * 8 * w.voxel_size
    near = coords[np.linalg.norm(c - T[:3, 3], axis=1) < 60.0]
    g = m.read_blocks(near, want_logp=False)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    for j, b in enumerate(near):
        om.write_block(b, g["D"][j].astype(np.float64), g["W"][j].astype(np.float64))
    near_pts = pts[np.linalg.norm(pts.astype(np.float64), axis=1) < 55.0]
    To = om.align(near_pts, T0, iters=20)
    Tg = m.align(torch.from_numpy(near_pts).to(dev), T0, iters=20)
    dt = float(np.linalg.norm(To[:3, 3] - Tg[:3, 3]))
    dr = _rot_deg(To[:3, :3], Tg[:3, :3])
    ro = _rot_deg(To[:3, :3], T[:3, :3])
    print(f"FP64 oracle after 20 iterations: {ro:.3f} deg from the truth; GPU - oracle {dt:.2e} m, {dr:.3f} deg")
    assert ro > 0.2                       # the FP64 path is just as far from converged
    assert dt < 1e-3 and dr < 0.05        # and the GPU follows it
    m.close()
