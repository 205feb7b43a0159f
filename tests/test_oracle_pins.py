"""Pins of the FP64 oracle against closed forms, brute force and invariants.

None of these retypes an oracle formula: each expected value comes from the
scene geometry (sphere, plane, per-pixel ranges), from a closed-form
solution of the update rules of the paper (Sec. III-C.2 running average,
Eq. bayesian_filter), or from brute-force enumeration, so a dropped term, a
wrong sign, a wrong index or a transposed operand in the oracle fails one of
them.  All run on the CPU in a few seconds.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.fields import (block_voxels, blocks_covering, points_on_rays, random_rotation, write_field)

BV = 512


def _pose(R, t):
    return synth.pose(R, np.asarray(t, np.float64))


def _all_voxels(m):
    """(coords, D, W, logP, taint) over every allocated block of an oracle map."""
    out = []
    for b in m.alloc_blocks():
        blk = m.read_block(b)
        if blk is None:
            continue
        out.append((block_voxels(b), blk))
    return out


# ---------------------------------------------------------------------------
# projective TSDF (Sec. III-C.2) on a hollow sphere seen from its centre
# ---------------------------------------------------------------------------
def _sphere_scan(R_s=3.0, H=64, W=256):
    lid = synth.lidar_deg(H, W, 89.0, -89.0, r_max=20.0)
    pts = points_on_rays(lid, np.full(H * W, R_s))
    return lid, pts


@pytest.mark.parametrize("weight_mode", [0, 1])
def test_sphere_tsdf_closed_form(weight_mode):
    """Every pixel range equals the sphere radius, so psi = R - rho exactly."""
    rng = np.random.default_rng(3)
    R_s, nu, tau = 3.0, 0.2, 0.6
    lid, pts = _sphere_scan(R_s)
    Rw = random_rotation(rng)
    t0 = np.array([0.31, -0.17, 0.12])
    T = _pose(Rw, t0)
    m = oracle.OracleMap(nu, tau, n_classes=2, weight_mode=weight_mode)
    n_frames = 3
    for _ in range(n_frames):
        st = m.integrate(lid, pts, T, labels=np.zeros(len(pts), np.int32))
    assert st["ambiguous_points"] == 0 and st["valid_points"] == len(pts)
    r_pix = np.linalg.norm(pts.astype(np.float64), axis=1)
    assert np.ptp(r_pix) < 1e-6
    checked = 0
    for v, blk in _all_voxels(m):
        rho = np.linalg.norm(v * nu - t0, axis=1)
        psi = R_s - rho
        far = psi < -tau - 1e-5
        near_edge = np.abs(psi + tau) <= 1e-5
        upd = ~far & ~near_edge
        assert np.all(blk["W"][far] == 0.0) and np.all(blk["D"][far] == 0.0)
        sdf = np.minimum(psi, tau)
        w = np.clip((psi + tau) / (2 * tau), 0.0, 1.0) if weight_mode == 0 else np.ones_like(psi)
        np.testing.assert_allclose(blk["D"][upd], sdf[upd], atol=2e-6, rtol=0)
        # k identical observations: D unchanged by the running average, W = k * w
        np.testing.assert_allclose(blk["W"][upd], n_frames * w[upd], atol=1e-5, rtol=0)
        checked += int(upd.sum())
    assert checked > 10000


def test_sphere_band_coverage_and_extent():
    """Allocated blocks cover the +-tau shell and nothing farther than tau from it."""
    rng = np.random.default_rng(4)
    R_s, nu, tau = 3.0, 0.2, 0.6
    lid, pts = _sphere_scan(R_s)
    t0 = np.array([0.05, 0.11, -0.07])
    T = _pose(random_rotation(rng), t0)
    m = oracle.OracleMap(nu, tau, n_classes=2)
    m.integrate(lid, pts, T, labels=np.zeros(len(pts), np.int32))
    alloc = {tuple(b) for b in m.alloc_blocks()}
    # every voxel well inside the shell lies in an allocated block
    vox = blocks_covering(t0 - (R_s + tau), t0 + (R_s + tau), nu)
    shell = 0
    for b in vox:
        v = block_voxels(b)
        rho = np.linalg.norm(v * nu - t0, axis=1)
        inshell = np.abs(rho - R_s) <= tau - 0.05
        if inshell.any():
            shell += 1
            assert tuple(b) in alloc
    assert shell > 50
    # every allocated block's cell box meets the shell R +- tau
    for b in alloc:
        lo = nu * (8 * np.array(b) - 0.5)
        hi = lo + 8 * nu
        nearest = np.clip(t0, lo, hi)
        dmin = np.linalg.norm(nearest - t0)
        far = np.where(np.abs(lo - t0) > np.abs(hi - t0), lo, hi)
        dmax = np.linalg.norm(far - t0)
        assert dmin <= R_s + tau + 1e-4 and dmax >= R_s - tau - 1e-4


# ---------------------------------------------------------------------------
# range image + pixel choice, by brute-force containment in the sensor's ray grid
# ---------------------------------------------------------------------------
def _brute_pixel(lid, d):
    """Pixel whose angular cell contains unit LiDAR-frame direction d (or None / 'edge').

    Cells are half-open in the index direction, as rounding u_c + 1/2 down
    makes them; directions within 1e-9 of a cell edge are reported as 'edge'.
    """
    H, W = lid.H, lid.W
    z = d[2]
    row = None
    for v in range(H):
        th = lid.theta0 + v * lid.dtheta
        lo, hi = math.cos(th + lid.dtheta / 2), math.cos(th - lid.dtheta / 2)
        if min(abs(z - lo), abs(z - hi)) < 1e-9:
            return "edge"
        if lo < z <= hi:
            row = v
    if row is None:
        return None
    hxy = math.hypot(d[0], d[1])
    if hxy < 1e-9:
        return "edge"
    h = (d[0] / hxy, d[1] / hxy)
    col = None
    c_half = math.cos(lid.dphi / 2)
    for u in range(W):
        ph = math.pi - u * lid.dphi
        c = h[0] * math.cos(ph) + h[1] * math.sin(ph)
        if abs(c - c_half) < 1e-9:
            return "edge"
        if c > c_half:
            col = u
    assert col is not None
    return row * W + col


def test_pixel_choice_brute_force():
    rng = np.random.default_rng(5)
    lid = synth.lidar_deg(5, 16, 20.0, -20.0, r_max=30.0)
    nu, tau = 0.25, 0.75
    ranges = rng.uniform(3.0, 8.0, size=lid.H * lid.W)
    pts = points_on_rays(lid, ranges)
    Rw = random_rotation(rng)
    t0 = np.array([0.05, 0.02, -0.03])
    T = _pose(Rw, t0)
    m = oracle.OracleMap(nu, tau, n_classes=2)
    st = m.integrate(lid, pts, T, labels=np.zeros(len(pts), np.int32))
    assert st["pixel_points"] == lid.H * lid.W and st["ambiguous_points"] == 0
    r_pix = np.linalg.norm(pts.astype(np.float64), axis=1)
    checked = skipped = 0
    for v, blk in _all_voxels(m):
        rel = v * nu - t0
        rho = np.linalg.norm(rel, axis=1)
        dl = (rel @ Rw) / rho[:, None]          # R^T rel, row-wise
        for i in range(BV):
            pix = _brute_pixel(lid, dl[i])
            if pix == "edge":
                skipped += 1
                continue
            if pix is None:
                assert blk["W"][i] == 0.0
                continue
            psi = r_pix[pix] - rho[i]
            if abs(psi + tau) < 1e-6:
                skipped += 1
                continue
            if psi < -tau:
                assert blk["W"][i] == 0.0
            else:
                assert blk["D"][i] == pytest.approx(min(psi, tau), abs=1e-9)
                assert blk["W"][i] == pytest.approx(min((psi + tau) / (2 * tau), 1.0), abs=1e-9)
            checked += 1
    assert checked > 5000 and skipped < checked // 100


def test_nearest_point_wins_pixel():
    """Two returns in one pixel: the voxel sees the nearer range."""
    lid = synth.lidar_deg(3, 8, 10.0, -10.0, r_max=30.0)
    nu, tau = 0.2, 0.6
    d = lid.ray_dirs()
    n = lid.H * lid.W
    near = np.full(n, 5.0)
    far = np.full(n, 9.0)
    pts = np.concatenate([d * far[:, None], d * near[:, None]]).astype(np.float32)
    m = oracle.OracleMap(nu, tau, n_classes=2, weight_mode=1)
    m.integrate(lid, pts, np.eye(4), labels=np.zeros(len(pts), np.int32))
    # voxel straight ahead along +x (column W/2, middle row) at 5.2 m: behind the
    # near return by 0.2 m -> D = -0.2; with the far return it would be +0.6
    v = np.array([26, 0, 0])
    b = np.floor_divide(v, 8)
    blk = m.read_block(b)
    i = int((v - 8 * b) @ np.array([1, 8, 64]))
    assert blk["W"][i] == 1.0
    assert blk["D"][i] == pytest.approx(5.0 - 26 * nu, abs=1e-6)


# ---------------------------------------------------------------------------
# semantic fusion (Eq. bayesian_filter): closed forms and invariants
# ---------------------------------------------------------------------------
def _sem_voxels(m, nu, t0, R_s, tau, margin=1e-5):
    """Voxels inside the semantic gate |psi| <= tau with a margin, every frame."""
    out = []
    for v, blk in _all_voxels(m):
        psi = R_s - np.linalg.norm(v * nu - t0, axis=1)
        gate = (np.abs(psi) < tau - margin) & (blk["W"] > 0)
        free = (psi > tau + margin) & (blk["W"] > 0)
        out.append((blk, gate, free))
    return out


def test_hard_label_count_closed_form():
    C, p_hit = 20, 0.9
    R_s, nu, tau = 3.0, 0.2, 0.6
    lid, pts = _sphere_scan(R_s)
    t0 = np.array([0.2, 0.1, -0.05])
    T = _pose(random_rotation(np.random.default_rng(6)), t0)
    m = oracle.OracleMap(nu, tau, n_classes=C, p_hit=p_hit)
    seq = [3, 3, 7, 3, 7]
    for lab in seq:
        m.integrate(lid, pts, T, labels=np.full(len(pts), lab, np.int32))
    # posterior proportional to kappa^{n_c}, kappa = p_hit (C-1) / (1 - p_hit)
    n_c = np.bincount(seq, minlength=C).astype(float)
    lk = math.log(p_hit * (C - 1) / (1 - p_hit))
    a = n_c * lk
    expect = a - (a.max() + math.log(np.exp(a - a.max()).sum()))
    n_gate = 0
    for blk, gate, free in _sem_voxels(m, nu, t0, R_s, tau):
        if gate.any():
            np.testing.assert_allclose(blk["logP"][:, gate], expect[:, None] * np.ones((1, gate.sum())),
                                       atol=1e-12, rtol=0)
            assert np.all(blk["label"][gate] == 3)   # most frequent label wins
            n_gate += int(gate.sum())
        if free.any():   # observed only as free space: prior untouched (uniform)
            np.testing.assert_allclose(blk["logP"][:, free], -math.log(C), atol=1e-15)
    assert n_gate > 1000


def test_identical_labels_convergence():
    C, p_hit, k = 20, 0.9, 4
    R_s, nu, tau = 3.0, 0.2, 0.6
    lid, pts = _sphere_scan(R_s)
    t0 = np.array([0.0, 0.0, 0.05])
    m = oracle.OracleMap(nu, tau, n_classes=C, p_hit=p_hit)
    for _ in range(k):
        m.integrate(lid, pts, _pose(np.eye(3), t0), labels=np.full(len(pts), 11, np.int32))
    rho_ = (1 - p_hit) / ((C - 1) * p_hit)
    p_l = 1.0 / (1.0 + (C - 1) * rho_ ** k)
    p_o = rho_ ** k / (1.0 + (C - 1) * rho_ ** k)
    seen = 0
    for blk, gate, _ in _sem_voxels(m, nu, t0, R_s, tau):
        if not gate.any():
            continue
        P = np.exp(blk["logP"][:, gate])
        np.testing.assert_allclose(P[11], p_l, rtol=1e-12)
        np.testing.assert_allclose(np.delete(P, 11, axis=0), p_o, rtol=1e-9)
        seen += int(gate.sum())
    assert seen > 1000


def test_probability_vector_closed_form_and_invariants():
    C = 20
    R_s, nu, tau = 3.0, 0.2, 0.6
    lid, pts = _sphere_scan(R_s, H=48, W=192)
    t0 = np.array([0.1, -0.1, 0.0])
    T = _pose(random_rotation(np.random.default_rng(7)), t0)
    rng = np.random.default_rng(8)
    qs = [rng.dirichlet(np.ones(C)) * 0.98 + 0.001 for _ in range(4)]
    maps = []
    for order in ([0, 1, 2, 3], [3, 1, 0, 2]):
        m = oracle.OracleMap(nu, tau, n_classes=C)
        for k in order:
            probs = np.tile(qs[k].astype(np.float32), (len(pts), 1))
            m.integrate(lid, pts, T, probs=probs)
        maps.append(m)
    # closed form: log P_c = sum_k log q_c^(k) - logsumexp (q passes through float32)
    a = sum(np.log(q.astype(np.float32).astype(np.float64)) for q in qs)
    expect = a - (a.max() + math.log(np.exp(a - a.max()).sum()))
    checked = 0
    for (blk, gate, _), (blk2, gate2, _) in zip(_sem_voxels(maps[0], nu, t0, R_s, tau),
                                                 _sem_voxels(maps[1], nu, t0, R_s, tau)):
        if not gate.any():
            continue
        lp = blk["logP"][:, gate]
        np.testing.assert_allclose(lp, expect[:, None] * np.ones((1, gate.sum())), atol=1e-12)
        np.testing.assert_allclose(np.exp(lp).sum(axis=0), 1.0, atol=1e-12)     # sums to one
        np.testing.assert_allclose(blk2["logP"][:, gate], lp, atol=1e-12)       # order-independent
        checked += int(gate.sum())
    assert checked > 500
    # a uniform likelihood leaves the posterior unchanged
    m = maps[0]
    before = [blk["logP"].copy() for _, blk in _all_voxels(m)]
    m.integrate(lid, pts, T, probs=np.full((len(pts), C), 1.0 / C, np.float32))
    for b0, (_, blk) in zip(before, _all_voxels(m)):
        np.testing.assert_allclose(blk["logP"], b0, atol=1e-12)


def test_probability_floors():
    """The two floors of the class update.  A likelihood entry below lik_floor counts as lik_floor
    (one update from the uniform prior gives log max(q, lik_floor) renormalised); a class whose
    likelihood stays at the floor falls by ~ln(1e6) per scan until its log-probability sits at
    logp_floor exactly, while the other classes keep the closed form of their product (the floored
    class carries < e^-30 of the mass, far below the 1e-12 tolerance)."""
    C, R_s, nu, tau = 6, 3.0, 0.2, 0.6
    lik_floor, logp_floor = 1e-6, -30.0
    lid, pts = _sphere_scan(R_s, H=48, W=192)
    t0 = np.array([0.05, 0.1, -0.05])
    T = _pose(random_rotation(np.random.default_rng(9)), t0)
    q = np.array([0.0, 0.4, 0.3, 0.2, 0.1, 0.0], np.float32)       # classes 0 and 5 below the floor
    m = oracle.OracleMap(nu, tau, n_classes=C, logp_floor=logp_floor, lik_floor=lik_floor)
    probs = np.tile(q, (len(pts), 1))
    lq = np.log(np.maximum(q.astype(np.float64), lik_floor))
    for k in range(1, 5):
        m.integrate(lid, pts, T, probs=probs)
        a = k * lq
        checked = 0
        for blk, gate, _ in _sem_voxels(m, nu, t0, R_s, tau):
            if not gate.any():
                continue
            lp = blk["logP"][:, gate]
            expect = a - (a.max() + math.log(np.exp(a - a.max()).sum()))
            if expect.min() > logp_floor:
                # no log-probability floor binds yet: the closed form with the likelihood floor
                np.testing.assert_allclose(lp, expect[:, None] * np.ones((1, gate.sum())), atol=1e-12)
            else:
                # classes 0 and 5 sit at the floor; the others keep the closed form of their product
                assert np.all(lp[[0, 5]] == logp_floor)
                live = np.array([1, 2, 3, 4])
                al = a[live] - (a[live].max() + math.log(np.exp(a[live] - a[live].max()).sum()))
                np.testing.assert_allclose(lp[live], al[:, None] * np.ones((1, gate.sum())), atol=1e-12)
            checked += int(gate.sum())
        assert checked > 500
    assert 3 * (math.log(lik_floor) - math.log(0.4)) < logp_floor   # the floor binds from the third scan


# ---------------------------------------------------------------------------
# block allocation along the band: brute-force segment sampling
# ---------------------------------------------------------------------------
def _seg_box_dist(e0, e1, b):
    """Min distance (voxel units) between a sampled segment and block b's box."""
    t = np.linspace(0.0, 1.0, 40001)[:, None]
    p = e0[None, :] + t * (e1 - e0)[None, :]
    lo, hi = 8.0 * b, 8.0 * b + 8.0
    q = np.clip(p, lo, hi)
    return np.linalg.norm(p - q, axis=1).min()


def _segment64(p, T, nu, tau):
    """The band segment of point p (LiDAR frame) written out independently, in FP64: the world
    point, the unit ray from the sensor, [p - tau d, p + tau d] (start at the sensor when
    |p| < tau), in voxel units + 1/2."""
    pw = T[:3, :3] @ p.astype(np.float64) + T[:3, 3]
    ray = pw - T[:3, 3]
    ray /= np.linalg.norm(ray)
    start = T[:3, 3] if np.linalg.norm(p.astype(np.float64)) < tau else pw - tau * ray
    return start / nu + 0.5, (pw + tau * ray) / nu + 0.5


def test_block_clearance_closed_forms():
    """Clearance = the deepest L-infinity penetration of the segment into the block's box."""
    b = np.array([0, 0, 0])
    # along x through the middle, ending 3 voxels inside: limited by the end point (x = 3)
    assert oracle.block_clearance([-2, 4, 4], [3, 4, 4], b) == pytest.approx(3.0)
    # through the whole block along x: limited by the y/z half widths (4)
    assert oracle.block_clearance([-2, 4, 4], [12, 4, 4], b) == pytest.approx(4.0)
    # off-centre in y (y = 6.5): 1.5 from the upper y face
    assert oracle.block_clearance([-2, 6.5, 4], [12, 6.5, 4], b) == pytest.approx(1.5)
    # parallel outside (y = 9): -1
    assert oracle.block_clearance([-2, 9, 4], [12, 9, 4], b) == pytest.approx(-1.0)
    # diagonal through the corner (8, 8, z) in the xy plane: touches the block's edge only -> 0
    assert oracle.block_clearance([7, 9, 4], [9, 7, 4], b) == pytest.approx(0.0, abs=1e-12)
    # the same diagonal moved inward by 0.1 in x and y: depth 0.1 at the crossing point
    assert oracle.block_clearance([6.9, 8.9, 4], [8.9, 6.9, 4], b) == pytest.approx(0.1)
    # ... and outward: the nearest approach is 0.1 beyond the edge on both axes -> -0.1
    assert oracle.block_clearance([7.1, 9.1, 4], [9.1, 7.1, 4], b) == pytest.approx(-0.1)
    # a point-like segment inside
    assert oracle.block_clearance([1, 2, 3], [1, 2, 3], b) == pytest.approx(1.0)
    # other blocks: translation by 8 b
    assert oracle.block_clearance([-2 + 8, 4 - 16, 4 + 24], [3 + 8, 4 - 16, 4 + 24], [1, -2, 3]) == \
        pytest.approx(3.0)


@pytest.mark.parametrize("nu,tau", [(0.1, 0.3), (0.25, 1.25)])
def test_band_blocks_brute_force(nu, tau):
    """tau = 3 nu (one crossing per axis at most) and tau = 5 nu (Table II: several).

    The oracle's FP64 endpoints equal the segment written out here; dense sampling of that
    segment (1/40000 of its length per step) finds every sure block and only blocks in
    sure + ambiguous; every ambiguous block lies within the margin of the segment."""
    rng = np.random.default_rng(9)
    m = oracle.OracleMap(nu, tau, n_classes=2)
    n_amb = 0
    for trial in range(200):
        T = _pose(random_rotation(rng), rng.uniform(-30, 30, size=3))
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p = (d * rng.uniform(0.2, 60.0)).astype(np.float32)
        if trial % 25 == 0:       # exact block-plane hits on purpose
            p = np.array([8 * nu * 3, 0.0, 0.0], np.float32)
            T = np.eye(4)
        e0, e1, margin = m.point_band(p, T)
        w0, w1 = _segment64(p, T, nu, tau)
        np.testing.assert_allclose(e0, w0, rtol=0, atol=1e-9)
        np.testing.assert_allclose(e1, w1, rtol=0, atol=1e-9)
        assert 0 < margin < 1e-2
        sure, amb = m.point_blocks(p, T)
        sure = {tuple(b) for b in sure.tolist()}
        amb = {tuple(b) for b in amb.tolist()}
        assert not (sure & amb)
        ts = np.linspace(0.0, 1.0, 40001)[:, None]
        samp = np.floor((w0[None, :] + ts * (w1 - w0)[None, :]) / 8.0).astype(np.int64)
        brute = {tuple(b) for b in np.unique(samp, axis=0).tolist()}
        assert sure <= brute, (trial, sure - brute)
        assert brute <= sure | amb, (trial, brute - sure - amb)
        for b in amb:
            assert _seg_box_dist(w0, w1, np.array(b, float)) <= 2 * margin, (trial, b)
            n_amb += 1
        assert len(sure) <= 1 + 3 * (int(2 * tau / nu) // 8 + 1)
    assert n_amb <= 20


def test_band_blocks_margin_classes():
    """A band ending just inside, on, or just outside a block plane: sure / ambiguous / absent."""
    nu, tau = 0.1, 0.3
    m = oracle.OracleMap(nu, tau, n_classes=2)
    # a point on +x at range r: e1_x = (r + tau) / nu + 1/2; put it at 8 * 5 + delta voxels
    for delta, want in ((0.05, "sure"), (1e-7, "ambiguous"), (-1e-7, "ambiguous"), (-0.05, "absent")):
        r = ((8 * 5 + delta) - 0.5) * nu - tau
        p = np.array([r, 0.0, 0.0], np.float32)
        e0, e1, margin = m.point_band(p, np.eye(4))
        assert abs(e1[0] - (40 + delta)) < 1e-5
        sure, amb = m.point_blocks(p, np.eye(4))
        blk = (5, 0, 0)
        got = "sure" if blk in {tuple(b) for b in sure.tolist()} else \
            ("ambiguous" if blk in {tuple(b) for b in amb.tolist()} else "absent")
        if abs(e1[0] - 40) > margin:
            assert got == ("sure" if e1[0] > 40 else "absent"), (delta, got)
        else:
            assert got == "ambiguous", (delta, got)
        assert got == want, (delta, got, e1[0] - 40, margin)


# ---------------------------------------------------------------------------
# marching cubes (Sec. III-C.3): closed forms, topology, orientation
# ---------------------------------------------------------------------------
def _mesh_edges(tk):
    """Directed triangle edges (as key pairs) with their multiplicity."""
    e = np.concatenate([tk[:, [0, 1]], tk[:, [1, 2]], tk[:, [2, 0]]])
    keys, cnt = np.unique(e, axis=0, return_counts=True)
    return {tuple(k): c for k, c in zip(keys.tolist(), cnt.tolist())}


def _tri_normals(me, keys_tri):
    idx = {k: i for i, k in enumerate(me["vkey"].tolist())}
    P = me["vpos"]
    a = P[[idx[k] for k in keys_tri[:, 0]]]
    b = P[[idx[k] for k in keys_tri[:, 1]]]
    c = P[[idx[k] for k in keys_tri[:, 2]]]
    return np.cross(b - a, c - a), a, b, c


def test_mc_linear_field_exact_and_oriented():
    rng = np.random.default_rng(10)
    nu = 0.1
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    c = 0.05
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    blocks = blocks_covering([-1.0] * 3, [1.0] * 3, nu)
    write_field(m, lambda x: x @ n - c, blocks, nu)
    me = m.mesh()
    assert len(me["tkeys"]) > 500
    np.testing.assert_allclose(me["vpos"] @ n - c, 0.0, atol=1e-12)
    nrm, *_ = _tri_normals(me, me["tkeys"])
    # normals point toward +D (free space); no degenerate triangles
    assert np.all(nrm @ n > 0)
    # every interior edge is used once in each direction
    E = _mesh_edges(me["tkeys"])
    for (a, b), cnt in E.items():
        assert cnt == 1
    interior = sum(1 for (a, b) in E if (b, a) in E)
    assert interior > 0.9 * len(E)


def test_mc_axis_plane_two_triangles_per_cube():
    nu = 0.1
    k = 5                     # plane between voxel layers z = 5 and z = 6
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    blocks = np.array([[bx, by, 0] for bx in range(2) for by in range(2)])
    write_field(m, lambda x: x[:, 2] - nu * (k + 0.37), blocks, nu)
    me = m.mesh()
    nx = ny = 16              # voxels per side of the written region
    assert len(me["tkeys"]) == 2 * (nx - 1) * (ny - 1)
    assert len(me["vkey"]) == nx * ny
    np.testing.assert_allclose(me["vpos"][:, 2], nu * (k + 0.37), atol=1e-12)


def test_mc_sphere_watertight_area_euler():
    nu, Rs = 0.1, 5.0
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    cand = blocks_covering([-Rs - 0.5] * 3, [Rs + 0.5] * 3, nu)
    keep = []
    for b in cand:
        lo = nu * (8 * b - 0.5)
        hi = lo + 8 * nu
        dmin = np.linalg.norm(np.clip(0.0, lo, hi))
        dmax = np.linalg.norm(np.maximum(np.abs(lo), np.abs(hi)))
        if dmin <= Rs + 0.3 and dmax >= Rs - 0.3:
            keep.append(b)
    write_field(m, lambda x: Rs - np.linalg.norm(x, axis=1), np.array(keep), nu)
    me = m.mesh()
    tk = me["tkeys"]
    E = _mesh_edges(tk)
    # closed, consistently oriented 2-manifold: each directed edge once, its reverse once
    assert all(cnt == 1 for cnt in E.values())
    assert all((b, a) in E for (a, b) in E)
    V, F = len(me["vkey"]), len(tk)
    n_edges = len(E) // 2
    assert V - n_edges + F == 2
    nrm, a, b, c = _tri_normals(me, tk)
    area = 0.5 * np.linalg.norm(nrm, axis=1).sum()
    assert abs(area / (4 * math.pi * Rs ** 2) - 1.0) < 0.01
    # hollow sphere seen from inside: +D is toward the centre
    centroid = (a + b + c) / 3
    dots = np.einsum("ij,ij->i", nrm, -centroid)
    # zero-area triangles appear where a voxel centre lies exactly on the sphere
    assert np.all(dots > -1e-15) and (dots > 0).mean() > 0.99


def test_mc_random_field_closed_chain():
    """Random signs exercise every case, including faces with four crossings.

    Each cube's triangles bound that cube's loops, and every face segment is
    walked once in each direction by the two cubes sharing the face, so away
    from the outer faces of the meshed region the triangles form a closed
    oriented 2-chain: every edge a->b is matched by as many b->a.
    """
    rng = np.random.default_rng(11)
    nu = 0.1
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    blocks = np.array([[x, y, z] for x in range(2) for y in range(2) for z in range(2)])
    vals = {}

    def field(x):
        v = np.round(x / nu).astype(int)
        return np.array([vals.setdefault(tuple(q), rng.normal()) for q in v])
    write_field(m, field, blocks, nu)
    me = m.mesh()
    E = _mesh_edges(me["tkeys"])
    idx = {k: i for i, k in enumerate(me["vkey"].tolist())}
    P = me["vpos"] / nu
    n_matched = 0
    for (a, b), cnt in E.items():
        if E.get((b, a), 0) == cnt:
            n_matched += 1
            continue
        # unmatched edges lie on the outer faces of the meshed region [0, 15]^3
        pa, pb = P[idx[a]], P[idx[b]]
        on = [(abs(pa[k] - s) < 1e-6 and abs(pb[k] - s) < 1e-6) for k in range(3) for s in (0.0, 15.0)]
        assert any(on)
    assert n_matched > 0.8 * len(E)
    # every vertex lies strictly inside its lattice edge
    key = me["vkey"]
    axis = key & 3
    lo = np.stack([((key >> s) & ((1 << 20) - 1)) - (1 << 19) for s in (2, 22, 42)], axis=1)
    frac = P[np.arange(len(P)), axis] - lo[np.arange(len(P)), axis]
    assert np.all((frac > 0) & (frac < 1))
    other = [k for k in range(3)]
    for k in other:
        sel = axis != k
        np.testing.assert_allclose(P[sel, k], lo[sel, k], atol=1e-9)


def test_mc_vertex_label_from_nearer_endpoint():
    nu, C = 0.1, 5
    m = oracle.OracleMap(nu, 0.3, n_classes=C)
    blocks = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]])

    def logp(v):
        cls = (v[:, 0] + 2 * v[:, 1] + 3 * v[:, 2]) % C
        lp = np.full((C, len(v)), -5.0)
        lp[cls, np.arange(len(v))] = -0.01
        return lp
    write_field(m, lambda x: x[:, 2] - nu * 6.3, blocks, nu, logp_fn=logp)
    me = m.mesh()
    # plane z = 6.3 voxels: the z-edge (6 -> 7) has its nearer endpoint at z = 6
    for key, lab in zip(me["vkey"].tolist(), me["vlab"].tolist()):
        x = ((key >> 2) & ((1 << 20) - 1)) - (1 << 19)
        y = ((key >> 22) & ((1 << 20) - 1)) - (1 << 19)
        z = ((key >> 42) & ((1 << 20) - 1)) - (1 << 19)
        assert key & 3 == 2 and z == 6
        assert lab == (x + 2 * y + 3 * z) % C


# ---------------------------------------------------------------------------
# trilinear query_sdf, its gradients and Gauss-Newton alignment
# ---------------------------------------------------------------------------
def test_query_linear_field_exact():
    rng = np.random.default_rng(12)
    nu = 0.1
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    write_field(m, lambda x: x @ n - 0.02, blocks_covering([-1.0] * 3, [1.0] * 3, nu), nu)
    x = rng.uniform(-0.8, 0.8, size=(500, 3))
    sdf, valid, grad = m.query(x)
    assert valid.all()
    np.testing.assert_allclose(sdf, x @ n - 0.02, atol=1e-12)
    np.testing.assert_allclose(grad, np.tile(n, (len(x), 1)), atol=1e-10)
    s2, v2, g2 = m.query(np.array([[50.0, 0.0, 0.0]]))
    assert not v2[0] and np.isnan(s2[0]) and np.all(g2 == 0)


def test_query_gradient_central_differences():
    rng = np.random.default_rng(13)
    nu, Rs = 0.1, 1.0
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    write_field(m, lambda x: Rs - np.linalg.norm(x, axis=1), blocks_covering([-1.5] * 3, [1.5] * 3, nu), nu)
    x = rng.uniform(-1.2, 1.2, size=(400, 3))
    f = x / nu - np.floor(x / nu)
    h = 1e-6
    keep = np.all((f > 2e-4) & (f < 1 - 2e-4), axis=1)      # away from cell faces (C0 kinks)
    x = x[keep]
    _, valid, grad = m.query(x)
    for k in range(3):
        dx = np.zeros(3)
        dx[k] = h
        sp, _, _ = m.query(x + dx)
        sm, _, _ = m.query(x - dx)
        np.testing.assert_allclose(grad[valid, k], ((sp - sm) / (2 * h))[valid], atol=1e-6)


def test_pose_gradient_central_differences():
    rng = np.random.default_rng(14)
    nu = 0.1
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    write_field(m, lambda x: x @ n + 0.1 * x[:, 0] ** 0, blocks_covering([-1.5] * 3, [1.5] * 3, nu), nu)
    pts = rng.uniform(-0.6, 0.6, size=(300, 3)).astype(np.float32)
    T = _pose(random_rotation(rng) @ np.eye(3), [0.05, -0.02, 0.03])
    T[:3, :3] = synth.rot_rpy(0.1, -0.05, 0.2)
    base = m.pose_terms(pts, T)
    assert base["n_valid"] == len(pts)
    h = 1e-6
    for j in range(6):
        xi = np.zeros(6)
        xi[j] = h
        lp = m.pose_terms(pts, oracle.se3_exp(xi) @ T)["loss"]
        lm = m.pose_terms(pts, oracle.se3_exp(-xi) @ T)["loss"]
        assert base["dL"][j] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-8)
    np.testing.assert_allclose(base["g"], 0.5 * base["dL"], rtol=1e-12, atol=1e-14)


def test_se3_exp_closed_form():
    # rotation about z by a: Exp((0,0,0, 0,0,a)) = Rz(a); translation along a pure rho is rho
    a = 0.7
    T = oracle.se3_exp([0.0, 0.0, 0.0, 0.0, 0.0, a])
    np.testing.assert_allclose(T[:3, :3], synth.rot_rpy(0.0, 0.0, a), atol=1e-15)
    T = oracle.se3_exp([0.3, -0.2, 0.1, 0.0, 0.0, 0.0])
    np.testing.assert_allclose(T[:3, 3], [0.3, -0.2, 0.1], atol=1e-15)
    # screw motion: rotating by pi about z with rho = (0, 0, 1) advances 1 along z
    T = oracle.se3_exp([0.0, 0.0, 1.0, 0.0, 0.0, math.pi])
    np.testing.assert_allclose(T[:3, 3], [0.0, 0.0, 1.0], atol=1e-12)


def _room_points(rng, size, o, n=4000):
    """Points where rays from o hit the inside walls of the box [0, size]."""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    with np.errstate(divide="ignore"):
        t = np.where(d > 0, (np.asarray(size) - o) / d, -o / d)
    return o + d * t.min(axis=1, keepdims=True)


def test_gauss_newton_recovers_pose():
    rng = np.random.default_rng(15)
    nu = 0.1
    size = np.array([6.0, 5.0, 4.0])

    def room(x):
        return np.minimum(x, size - x).min(axis=1)
    m = oracle.OracleMap(nu, 0.3, n_classes=2)
    blocks = blocks_covering([-0.6] * 3, size + 0.6, nu)
    write_field(m, room, blocks, nu)
    T_true = _pose(synth.rot_rpy(0.02, -0.03, 0.4), [2.8, 2.2, 1.6])
    pw = _room_points(rng, size, T_true[:3, 3])
    pl = ((pw - T_true[:3, 3]) @ T_true[:3, :3]).astype(np.float32)
    xi = np.concatenate([rng.normal(size=3), rng.normal(size=3)])
    xi[:3] *= 0.1 / np.linalg.norm(xi[:3])
    xi[3:] *= math.radians(2.0) / np.linalg.norm(xi[3:])
    T0 = oracle.se3_exp(xi) @ T_true
    T = m.align(pl, T0, iters=20)
    assert np.abs(T[:3, 3] - T_true[:3, 3]).max() < 2e-3
    assert np.abs(T[:3, :3] - T_true[:3, :3]).max() < 2e-3
    assert m.pose_terms(pl, T)["loss"] < 1e-2 * m.pose_terms(pl, T0)["loss"]


def test_palette_hsv():
    pal = oracle.palette(20)
    assert pal.shape == (20, 3) and len({tuple(p) for p in pal}) == 20
    assert tuple(pal[0]) == (255, 0, 0)
