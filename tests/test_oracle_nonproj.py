"""Pins of the oracle's non-projective distance (Sec. III-C.2, Eq. distance).

The expected values come from geometry the formula has to reproduce, not
from the formula retyped:
  - a sphere seen from outside (convex) and from inside (concave): the exact
    signed distance |x - O| - R (resp. R - |x - O|) of a voxel on the ray
    through the surface point p_j, with g the true gradient at the voxel and
    N the true normal at p_j;
  - a plane: the perpendicular distance;
  - the normal image of a scanned plane: the plane's normal, facing the
    sensor, with no normal exactly where a neighbour pixel has no return;
  - an oblique plane fused over several scans: D equals the true distance
    up to the projective sampling error of the pixel grid, while the
    projective distance overestimates it by psi (1 - cos theta).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.fields import block_voxels, points_on_rays


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def _sphere_cases(rng, concave, n=3000):
    """(psi, u, g, N, exact distance) for voxels on rays through a sphere of radius R at the origin."""
    out = []
    while len(out) < n:
        R = rng.uniform(0.5, 5.0)
        if concave:
            S = _unit(rng.normal(size=3)) * rng.uniform(0.0, 0.9) * R
            dirn = _unit(rng.normal(size=3))
            b = S @ dirn
            s = -b + math.sqrt(b * b - (S @ S - R * R))        # forward hit from inside
            q = S + s * dirn
            N = -q / R                                           # faces the interior (the sensor)
        else:
            S = _unit(rng.normal(size=3)) * rng.uniform(1.5, 10.0) * R
            q = _unit(rng.normal(size=3)) * R
            N = q / R
            if N @ (S - q) <= 0.0:                               # hidden side: not the first hit
                continue
        u = _unit(S - q)
        span = np.linalg.norm(S - q)
        psi = rng.uniform(-0.4, 0.4) * min(R, span)
        x = q + psi * u
        rx = np.linalg.norm(x)
        if rx < 1e-3 * R:
            continue
        if concave:
            d_true, g = R - rx, -x / rx
        else:
            d_true, g = rx - R, x / rx
        out.append((psi, u, g, N, d_true))
    return out


@pytest.mark.parametrize("concave", [False, True])
def test_distance_exact_on_a_sphere(concave):
    """On a circle through p_j the formula is the exact distance, both sides of the surface."""
    rng = np.random.default_rng(11 + concave)
    checked = 0
    for psi, u, g, N, d_true in _sphere_cases(rng, concave):
        if g @ N <= 0.0 or g @ u <= 0.0:
            continue          # the flat case applies there (cos alpha <= 0) or |cos theta| folds the sign
        d = oracle.nonprojective_distance(psi, u, g, N)
        assert abs(d - d_true) <= 1e-10 * max(1.0, abs(psi)), (psi, d, d_true)
        checked += 1
    assert checked > 2000


def test_sphere_distance_differs_from_the_projective_and_flat_forms():
    """The curvature term matters: the flat form |cos theta| psi misses the sphere distance."""
    rng = np.random.default_rng(5)
    worst_flat = 0.0
    for psi, u, g, N, d_true in _sphere_cases(rng, False, 500):
        if g @ N <= 0.0 or g @ u <= 0.0:
            continue
        worst_flat = max(worst_flat, abs(abs(g @ u) * psi - d_true) / max(abs(psi), 1e-9))
    assert worst_flat > 0.05


def test_distance_flat_cases():
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = _unit(rng.normal(size=3))
        u = _unit(rng.normal(size=3))
        if n @ u < 0:
            u = -u
        psi = rng.uniform(-1.0, 1.0)
        # plane: g = N = n, the perpendicular distance of p_j + psi u
        assert abs(oracle.nonprojective_distance(psi, u, n, n) - psi * (n @ u)) < 1e-12
        # no normal at the pixel: flat with the stored gradient
        assert abs(oracle.nonprojective_distance(psi, u, n, None) - psi * (n @ u)) < 1e-12
        # gradient and normal more than 90 degrees apart: flat
        assert abs(oracle.nonprojective_distance(psi, u, n, -n) - psi * (n @ u)) < 1e-12
        # no gradient yet: the projective distance
        assert oracle.nonprojective_distance(psi, u, np.zeros(3), n) == psi


# ---------------------------------------------------------------------------
# scans of planes
# ---------------------------------------------------------------------------
def _plane_scan(lid, T, n, c):
    """Noise-free points on the plane n . x = c (world), LiDAR frame; NaN where a ray misses or exceeds r_max."""
    d_l = lid.ray_dirs()
    R, t = T[:3, :3], T[:3, 3]
    d_w = d_l @ R.T
    den = d_w @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (c - n @ t) / den
    ok = (den != 0) & (s > 0) & (s <= lid.r_max)
    ranges = np.where(ok, s, np.nan)
    return points_on_rays(lid, ranges), ok.reshape(lid.H, lid.W)


@pytest.mark.parametrize("which", ["ground", "wall"])
def test_normal_image_of_a_plane(which):
    rng = np.random.default_rng(2)
    lid = synth.lidar_deg(32, 512, 15.0, -25.0, r_max=40.0)
    Rw = synth.rot_rpy(math.radians(3.0), math.radians(-2.0), math.radians(40.0))
    t0 = np.array([1.3, -0.7, 1.8])
    T = synth.pose(Rw, t0)
    if which == "ground":
        n, c = np.array([0.0, 0.0, 1.0]), 0.037
    else:
        n = _unit([-1.0, 0.2, 0.0])
        c = n @ (t0 + 7.0 * _unit(Rw[:, 0]))
    pts, hit = _plane_scan(lid, T, n, c)
    m = oracle.OracleMap(0.2, 0.6, n_classes=2, distance="nonprojective")
    m.integrate(lid, pts, T, labels=np.zeros(len(pts), np.int32))
    N, f = m.normals()
    valid = np.zeros_like(hit)
    valid[1:] = hit[1:] & hit[:-1] & np.roll(hit, 1, axis=1)[1:]
    assert np.array_equal((f & 1).astype(bool).reshape(hit.shape), valid)
    assert valid.sum() > 1000
    Nv = N[valid.ravel()]
    # the plane's normal, on the sensor's side of the plane (n . t0 > c)
    assert np.max(np.abs(Nv - n)) < 1e-4
    assert not np.any(f & 2)


def _voxels_with(m, fn):
    for b in m.alloc_blocks():
        blk = m.read_block(b)
        if blk is not None:
            yield block_voxels(b), blk, fn(b)


def test_oblique_plane_true_distance():
    """Several scans of a plane seen at ~50 degrees: D is the perpendicular distance.

    The only error left in the non-projective mode is the pixel grid's: a voxel
    takes the range of its pixel's centre ray, not of its own ray, which on a
    plane at incidence i differs by up to about r tan(i) times the angle to the
    pixel centre.  The projective mode is off by psi (1 - cos theta) on top.
    """
    lid = synth.lidar_deg(128, 2048, 20.0, -20.0, r_max=30.0)
    n = _unit([-1.0, 1.2, 0.1])
    c = -4.0
    nu, tau = 0.1, 0.3
    maps = {k: oracle.OracleMap(nu, tau, n_classes=2, weight_mode=1, distance=k)
            for k in ("projective", "nonprojective")}
    poses = [synth.pose(synth.rot_rpy(0.01 * k, -0.02 * k, 0.3 + 0.05 * k), np.array([0.2 * k, 0.1 * k, 0.0]))
             for k in range(4)]
    for T in poses:
        pts, _ = _plane_scan(lid, T, n, c)
        for m in maps.values():
            m.integrate(lid, pts, T, labels=np.zeros(len(pts), np.int32))
    half_pix = 0.5 * math.hypot(lid.dphi, lid.dtheta)
    err = {}
    for k, m in maps.items():
        e_all = []
        for v, blk, G in _voxels_with(m, lambda b, m=m: m.read_grad(b)):
            x = v * nu
            dist = x @ n - c                                        # > 0 on the sensors' side
            r_all = np.array([np.linalg.norm(x - T[:3, 3], axis=1) for T in poses])
            elev = np.array([np.arcsin(((x - T[:3, 3]) @ T[:3, :3])[:, 2] / np.linalg.norm(x - T[:3, 3], axis=1))
                             for T in poses])
            # seen by every scan, well inside the returns (r_max 30 m) and below the top beam (no
            # normal there): every pixel the voxel projected to had a normal
            sel = ((blk["W"] == len(poses)) & (np.abs(dist) < 0.5 * tau) & (blk["taint"] == 0)
                   & (r_all.max(axis=0) < 20.0) & (elev.max(axis=0) < lid.fov_up - 2.0 * lid.dtheta))
            if k == "nonprojective":
                # gradient: the plane's normal; unit length once a normal was seen (zero before,
                # e.g. for voxels that only ever projected to pixels at the edge of the returns)
                np.testing.assert_allclose(G[:, sel].T, np.broadcast_to(n, (int(sel.sum()), 3)), atol=1e-4)
                gl = np.linalg.norm(G, axis=0)
                assert np.all((np.abs(gl - 1.0) < 1e-12) | (gl == 0.0))
                assert np.all(G[:, blk["W"] == 0] == 0.0)
            r = r_all[:, sel].max(axis=0)
            cos_i = np.min([np.abs((x[sel] - T[:3, 3]) @ n) / np.linalg.norm(x[sel] - T[:3, 3], axis=1)
                            for T in poses], axis=0)
            bound = 1.2 * (r + tau) * np.sqrt(1.0 - cos_i ** 2) / cos_i * half_pix + 1e-6
            e = np.abs(blk["D"][sel] - dist[sel])
            if k == "nonprojective":
                assert np.all(e <= bound), float(np.max(e - bound))
            e_all.append(e)
        err[k] = np.concatenate(e_all)
    assert len(err["nonprojective"]) > 5000
    assert np.mean(err["projective"]) > 5.0 * np.mean(err["nonprojective"])
