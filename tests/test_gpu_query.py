"""query_sdf forward/backward, pose gradient and Gauss-Newton alignment vs the oracle.

Both maps hold the same seeded field (written through the C ABI and the
oracle's block writer, values exactly representable in FP32 or FP16), so
any difference comes from the query arithmetic alone.

Tolerances: sdf |d| <= 2e-6 m (FP32 interpolation of |D| <= 1 m fields near
the origin); dD/dx relative 1e-4; pose gradient relative 1e-4 (acceptance
rule); aligned pose within 1e-4 m / 1e-4 rad of the oracle's FP64 run.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.fields import block_voxels, blocks_covering, random_rotation  # noqa: E402


def _P():
    import paper_2412_00291_b300 as P
    return P


def _twin(field, blocks, nu, storage=0, n_classes=2):
    P = _P()
    g = P.SemanticTSDF(nu, 3 * nu, n_classes, storage=storage, max_blocks=max(4096, 2 * len(blocks)),
                       hash_capacity=1 << 16, max_points=1 << 18, max_pixels=1 << 12, mesh_vertex_capacity=1 << 20,
                       mesh_triangle_capacity=1 << 20)
    o = oracle.OracleMap(nu, 3 * nu, n_classes)
    cast = np.float16 if storage else np.float32
    D = np.stack([field(block_voxels(b) * nu) for b in blocks]).astype(cast).astype(np.float32)
    W = np.ones_like(D)
    g.write_blocks(blocks, D, W)
    for b, d in zip(blocks, D):
        o.write_block(b, d.astype(np.float64), np.ones(512))
    return g, o


def _sphere(c, R):
    return lambda x: R - np.linalg.norm(x - c, axis=1)


@pytest.mark.parametrize("storage", [0, 1])
def test_query_forward_backward(storage):
    rng = np.random.default_rng(31)
    nu = 0.1
    blocks = blocks_covering([-1.6] * 3, [1.6] * 3, nu)
    g, o = _twin(_sphere(np.zeros(3), 1.0), blocks, nu, storage)
    x = rng.uniform(-1.7, 1.7, size=(20000, 3)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    sdf, valid = g.query(xd)
    osdf, ovalid, ograd = o.query(x.astype(np.float64))
    np.testing.assert_array_equal(valid.cpu().numpy(), ovalid)
    assert ovalid.mean() > 0.5 and (~ovalid).sum() > 100
    s = sdf.cpu().numpy()
    assert np.all(np.isnan(s[~ovalid]))
    np.testing.assert_allclose(s[ovalid], osdf[ovalid], atol=2e-6, rtol=0)
    P = _P()
    gs = torch.from_numpy(rng.normal(size=len(x)).astype(np.float32)).cuda()
    gx = P.query_sdf_backward(g.h, xd, gs).cpu().numpy()
    want = ograd * gs.cpu().numpy()[:, None]
    np.testing.assert_allclose(gx[ovalid], want[ovalid], atol=1e-4 * np.abs(want).max(), rtol=1e-4)
    assert np.all(gx[~ovalid] == 0)
    # autograd Function gives the same gradient
    xr = xd.clone().requires_grad_(True)
    sd, vd = P.QuerySDF.apply(xr, g)
    (torch.nan_to_num(sd) * gs).sum().backward()
    np.testing.assert_allclose(xr.grad.cpu().numpy(), gx, rtol=0, atol=0)


def test_pose_gradient_matches_oracle_and_fd():
    rng = np.random.default_rng(32)
    nu = 0.1
    blocks = blocks_covering([-2.0] * 3, [2.0] * 3, nu)
    g, o = _twin(_sphere(np.array([0.1, -0.2, 0.05]), 1.2), blocks, nu)
    P = _P()
    pts = (rng.normal(size=(5000, 3)) * 0.3 + rng.normal(size=(5000, 3)) / 1.0).astype(np.float32)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    pts *= rng.uniform(0.9, 1.5, size=(len(pts), 1)).astype(np.float32)
    T = synth.pose(random_rotation(rng), [0.03, -0.02, 0.01])
    # world points of the scan under T (FP32, as a user would pass them)
    xw = (pts.astype(np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)
    xd = torch.from_numpy(xw).cuda()
    sdf, valid = g.query(xd)
    grad_sdf = torch.where(valid, 2.0 * torch.nan_to_num(sdf), torch.zeros_like(sdf))
    pg = P.pose_gradient(g, xd, grad_sdf).cpu().numpy()
    ref = o.pose_terms(xw.astype(np.float64).astype(np.float32), np.eye(4))
    np.testing.assert_allclose(pg, ref["dL"], rtol=1e-4, atol=1e-6 * np.abs(ref["dL"]).max())
    # and against FP64 central differences of the oracle loss (h = 1e-4)
    h = 1e-4
    for j in range(6):
        xi = np.zeros(6)
        xi[j] = h
        lp = o.pose_terms(xw, oracle.se3_exp(xi))["loss"]
        lm = o.pose_terms(xw, oracle.se3_exp(-xi))["loss"]
        fd = (lp - lm) / (2 * h)
        assert pg[j] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(ref["dL"]).max())


@pytest.mark.parametrize("name,storage", [("line16", 0), ("drive1km", 1)])
def test_pose_gradient_on_a_fused_map(name, storage):
    """The pose gradient on a map fused from scans rather than an analytic field: the oracle fuses
    the first four scans of the workload (16 x 1024 at 0.2 m voxels near the origin, FP32 storage;
    64 x 2048 at 0.1 m voxels 480 m from it, FP16 storage), its blocks (rounded to the storage
    type) are written into both maps, and the device
    gradient of sum sdf^2 over the last scan's points at a perturbed pose is compared with the
    oracle's FP64 analytic gradient and with FP64 central differences (h = 1e-4) of its loss.
    Rotations are taken about the points' centroid c (the gradient about the origin converts as
    g_phi(c) = g_phi - c x g_rho).  Only points valid and inside the same interpolation cell at the
    pose and all 12 perturbed poses enter the loss: the trilinear field's gradient jumps across
    cell faces, so the loss is smooth only there."""
    w = getattr(synth, name)()
    L = w.lidar
    frames = list(synth.sequence(w, 4))
    cast = np.float16 if storage else np.float32
    ob = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    for f in frames:
        ob.integrate(L, f.points, f.T, labels=f.labels)
    blocks = ob.alloc_blocks()
    D, W = [], []
    for b in blocks:
        r = ob.read_block(b)
        D.append(r["D"].astype(cast).astype(np.float32))
        W.append(r["W"].astype(cast).astype(np.float32))
    D, W = np.stack(D), np.stack(W)
    P = _P()
    g = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, storage=storage, max_blocks=2 * len(blocks),
                       hash_capacity=1 << 17, max_points=1 << 18, max_pixels=1 << 18, mesh_vertex_capacity=1 << 20,
                       mesh_triangle_capacity=1 << 20)
    g.write_blocks(blocks, D, W)
    o = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    for b, d, wt in zip(blocks, D, W):
        o.write_block(b, d.astype(np.float64), wt.astype(np.float64))
    f = frames[-1]
    p = f.points[np.isfinite(f.points).all(axis=1)]
    T = f.T @ synth.pose(synth.rot_rpy(0.004, -0.003, 0.006), [0.04, -0.03, 0.02])
    xw = (p.astype(np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)
    x = xw.astype(np.float64)
    c = x.mean(axis=0)
    nu, h = w.voxel_size, 1e-4

    def moved(j, sgn):
        if j < 3:
            y = x.copy()
            y[:, j] += sgn * h
            return y
        e = np.zeros(6)
        e[j] = sgn * h
        return (x - c) @ oracle.se3_exp(e)[:3, :3].T + c

    base_sdf, ok, base_grad = o.query(x)
    cell = np.floor(x / nu)
    sides = {}
    for j in range(6):
        for sgn in (1, -1):
            y = moved(j, sgn)
            sd, vv, _ = o.query(y)
            sides[(j, sgn)] = sd
            ok &= vv & np.all(np.floor(y / nu) == cell, axis=1)
    assert ok.sum() > 2000
    fd = np.array([(np.sum(sides[(j, 1)][ok] ** 2) - np.sum(sides[(j, -1)][ok] ** 2)) / (2 * h) for j in range(6)])
    gx = 2.0 * base_sdf[ok, None] * base_grad[ok]
    ref = np.concatenate([gx.sum(axis=0), np.cross(x[ok] - c, gx).sum(axis=0)])
    xd = torch.from_numpy(xw).cuda()
    sdf, valid = g.query(xd)
    okd = torch.from_numpy(ok).cuda()
    assert bool(valid[okd].all())
    gs = torch.where(okd & valid, 2.0 * torch.nan_to_num(sdf), torch.zeros_like(sdf))
    pg = P.pose_gradient(g, xd, gs).cpu().numpy().astype(np.float64)
    pg_c = np.concatenate([pg[:3], pg[3:] - np.cross(c, pg[:3])])
    scale = float(np.abs(ref).max())
    e_ref = float(np.max(np.abs(pg_c - ref)) / scale)
    e_fd = float(np.max(np.abs(pg_c - fd)) / scale)
    print(f"fused-map pose gradient ({name}): {int(ok.sum())} of {len(p)} points in the loss, relative error "
          f"{e_ref:.2e} vs the oracle's analytic gradient, {e_fd:.2e} vs central differences")
    assert e_ref <= 1e-4, e_ref
    assert e_fd <= 1e-4, e_fd


def _room_points(rng, size, o, n):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    with np.errstate(divide="ignore"):
        t = np.where(d > 0, (np.asarray(size) - o) / d, -o / d)
    return o + d * t.min(axis=1, keepdims=True)


@pytest.mark.parametrize("storage", [0, 1])
def test_gauss_newton_alignment(storage):
    rng = np.random.default_rng(33)
    nu = 0.1
    size = np.array([6.0, 5.0, 4.0])
    blocks = blocks_covering([-0.6] * 3, size + 0.6, nu)
    g, o = _twin(lambda x: np.minimum(x, size - x).min(axis=1), blocks, nu, storage)
    T_true = synth.pose(synth.rot_rpy(0.02, -0.03, 0.4), [2.8, 2.2, 1.6])
    pw = _room_points(rng, size, T_true[:3, 3], 20000)
    pl = ((pw - T_true[:3, 3]) @ T_true[:3, :3]).astype(np.float32)
    xi = np.concatenate([rng.normal(size=3), rng.normal(size=3)])
    xi[:3] *= 0.1 / np.linalg.norm(xi[:3])
    xi[3:] *= math.radians(2.0) / np.linalg.norm(xi[3:])
    T0 = oracle.se3_exp(xi) @ T_true
    Tg = g.align(torch.from_numpy(pl).cuda(), T0, iters=20)
    To = o.align(pl, T0, iters=20)
    assert np.abs(Tg[:3, 3] - To[:3, 3]).max() < (1e-4 if storage == 0 else 1e-3)
    assert np.abs(Tg[:3, :3] - To[:3, :3]).max() < (1e-4 if storage == 0 else 1e-3)
    assert np.abs(Tg[:3, 3] - T_true[:3, 3]).max() < 3e-3
