"""The synthetic input generator: analytic hits against ray marching, determinism."""
import math

import numpy as np

import synth


def _occupied(scene, p):
    """Inside any solid primitive or below the ground (for points p [n, 3])."""
    occ = p[:, 2] < 0.0
    for b in scene.boxes:
        occ |= np.all((p >= b[:3]) & (p <= b[3:]), axis=1)
    for c in scene.cyls:
        occ |= ((p[:, 0] - c[0]) ** 2 + (p[:, 1] - c[1]) ** 2 <= c[2] ** 2) & (p[:, 2] >= 0) & (p[:, 2] <= c[3])
    return occ


def _ramp_side(scene, p):
    """Per ramp: sign of height above its surface inside its footprint (0 outside)."""
    out = []
    for r in scene.ramps:
        inside = (np.abs(p[:, 0] - r[0]) <= r[2]) & (np.abs(p[:, 1] - r[1]) <= r[3])
        zs = r[4] + r[5] * (p[:, 0] - r[0]) + r[6] * (p[:, 1] - r[1])
        out.append(np.where(inside & (zs >= 0), np.sign(p[:, 2] - zs), 0.0))
    return np.array(out)


def _march(scene, o, d, t_max, step=1e-3):
    ts = np.arange(0.0, t_max, step)
    p = o[None, :] + ts[:, None] * d[None, :]
    hit = _occupied(scene, p)
    side = _ramp_side(scene, p)
    flips = np.zeros(len(ts), bool)
    if len(side):
        flips[1:] = np.any((side[:, 1:] != side[:, :-1]) & (side[:, 1:] != 0) & (side[:, :-1] != 0), axis=0)
    first = np.flatnonzero(hit | flips)
    return ts[first[0]] if len(first) else math.inf


def test_analytic_hits_match_ray_marching():
    rng = np.random.default_rng(21)
    sc = synth.Scene(
        boxes=np.array([[3, -1, 0, 5, 1, 2.5], [-6, 2, 0, -4, 5, 1.5], [1, 4, 0, 3, 7, 4.0]], float),
        box_cls=np.array([1, 2, 3], np.int32),
        cyls=np.array([[0, -5, 0.8, 3.0], [-3, -3, 0.4, 6.0]], float),
        cyl_cls=np.array([4, 5], np.int32),
        ramps=np.array([[8, 6, 3, 2, 0.5, 0.1, -0.05]], float),
        ramp_cls=np.array([6], np.int32))
    o = np.array([0.2, 0.3, 1.8])
    d = rng.normal(size=(300, 3))
    d[:, 2] = -np.abs(d[:, 2]) * 0.3
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t, cls = sc.cast(o, d, 20.0)
    hits = 0
    for i in range(len(d)):
        tm = _march(sc, o, d[i], 20.0)
        if math.isinf(tm):
            assert math.isinf(t[i]) and cls[i] == -1
        else:
            assert abs(tm - t[i]) <= 1.5e-3, (i, tm, t[i])
            hits += 1
    assert hits > 200


def test_points_sit_on_pixel_centre_rays_and_are_deterministic():
    w = synth.line16()
    sc = synth.make_scene(w)
    T = synth.trajectory(w, 2)[1]
    f1 = synth.make_frame(w, sc, T, 1)
    f2 = synth.make_frame(w, sc, T, 1, nthreads=1)
    assert f1.points.tobytes() == f2.points.tobytes()
    assert f1.labels.tobytes() == f2.labels.tobytes()
    ok = np.isfinite(f1.points[:, 0])
    d = w.lidar.ray_dirs()
    p = f1.points[ok].astype(np.float64)
    r = np.linalg.norm(p, axis=1)
    cosang = np.einsum("ij,ij->i", p / r[:, None], d[ok])
    assert np.all(cosang > 1 - 1e-12)
    # noise: r - true range ~ N(0, sigma)
    res = r - f1.true_range[ok]
    assert abs(res.mean()) < 3 * w.sigma / math.sqrt(len(res)) + 1e-4
    assert abs(res.std() / w.sigma - 1) < 0.05
    # hard labels: flipped with p = 0.1 to a different class
    flips = f1.labels[ok] != f1.true_cls[ok]
    assert abs(flips.mean() - 0.1) < 0.02


def test_probability_rows():
    w = synth.loop64()
    sc = synth.make_scene(w)
    T = synth.trajectory(w, 1)[0]
    f = synth.make_frame(w, sc, T, 0)
    ok = f.labels >= 0
    q = f.probs[ok].astype(np.float64)
    np.testing.assert_allclose(q.sum(axis=1), 1.0, atol=1e-5)
    assert np.all(q >= 0)
    assert (q.argmax(axis=1) == f.true_cls[ok]).mean() > 0.8
    assert np.all(f.probs[~ok] == 0)
    assert 0.5 < ok.mean() < 0.95


def test_angular_jitter_moves_points_off_their_pixel_centres():
    """jitter = 0.35 px: the FP64 projection (u_c, v_c) of each point sits N(0, 0.35) pixels from
    its generating pixel in both angles, so about 15 % of the points land nearer another pixel;
    ranges keep their noise model; the jitter draws leave the un-jittered streams unchanged."""
    wj = synth.line16_jitter()
    w0 = synth.line16()
    sc = synth.make_scene(w0)
    T = synth.trajectory(w0, 2)[1]
    f = synth.make_frame(wj, sc, T, 1)
    f0 = synth.make_frame(w0, sc, T, 1)
    L = wj.lidar
    ok = np.isfinite(f.points[:, 0])
    p = f.points[ok].astype(np.float64)
    r = np.linalg.norm(p, axis=1)
    uc = (math.pi - np.arctan2(p[:, 1], p[:, 0])) / L.dphi
    vc = (np.arccos(p[:, 2] / r) - L.theta0) / L.dtheta
    idx = np.flatnonzero(ok)
    u0, v0 = idx % L.W, idx // L.W
    du = (uc - u0 + L.W / 2) % L.W - L.W / 2
    dv = vc - v0
    assert abs(du.std() - 0.35) < 0.02 and abs(dv.std() - 0.35) < 0.02
    # (which rays hit something depends a little on the jitter, so allow a small selection bias)
    assert abs(du.mean()) < 0.02 and abs(dv.mean()) < 0.02
    moved = (np.floor(uc + 0.5) % L.W != u0) | (np.floor(vc + 0.5) != v0)
    assert 0.2 < moved.mean() < 0.35          # 1 - (1 - 0.153)^2 = 0.28 expected
    res = r - f.true_range[ok]
    assert abs(res.std() / wj.sigma - 1) < 0.05
    # the same seeds without jitter give the centre-ray scan, bit for bit the un-jittered workload's
    assert np.isfinite(f0.points[:, 0]).sum() > 0
    f0b = synth.make_frame(w0, sc, T, 1)
    assert f0.points.tobytes() == f0b.points.tobytes()
