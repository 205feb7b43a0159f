"""Batched persistent integration (one cooperative launch for many maps).

map_batch_integrate must give, map by map, what integrate_scan gives: the
same block sets, the same voxel contents bit for bit, the same per-frame
counters (dirty-block count aside, see COUNTERS) and the same mesh.  The maps in one batch differ in voxel size,
storage precision, class input (hard labels or probability vectors) and
scan size (including an empty scan), and the autotuner rotates the launch
configuration every step, so every configuration is checked.  One batched
map is also compared with the FP64 oracle.  The barrier's bounded wait is
exercised by letting one CTA leave before the first barrier: the step must
report MAP_ERR_TIMEOUT and the next step must run normally.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.gpu_compare import Lockstep, compare_blocks, compare_meshes  # noqa: E402

# dirty_blocks is left out: a block allocated in this scan links itself to its neighbours while
# other warps read those links to queue lower neighbours for re-meshing, so a new block none of
# whose voxels was observed may or may not be queued.  Such a block has no valid cube and emits
# nothing either way (the mesh counters and meshes are compared exactly).
COUNTERS = ("valid_points", "pixel_points", "touched_blocks", "new_blocks", "voxels_updated", "voxels_semantic",
            "mesh_vertices", "mesh_triangles", "total_blocks", "error_bits")


def _lib():
    import paper_2412_00291_b300 as p
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sorted(c):
    c = np.asarray(c).reshape(-1, 3)
    return c[np.lexsort((c[:, 2], c[:, 1], c[:, 0]))]


def _probs(labels, C, seed):
    """Soft class vectors peaked at the label (rows sum to 1)."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.0, 1.0, size=(labels.size, C)).astype(np.float32)
    q[np.arange(labels.size), np.clip(labels, 0, C - 1)] += 6.0
    return (q / q.sum(axis=1, keepdims=True)).astype(np.float32)


def _new_map(p, w, nu, tau, storage):
    return p.SemanticTSDF(nu, tau, w.n_classes, storage=storage, max_blocks=32768, hash_capacity=1 << 16,
                          max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                          mesh_triangle_capacity=1 << 23)


# (voxel size, truncation, storage, class input, points kept per frame)
SPECS = [(None, None, 0, "labels", None),
         (0.2, 0.6, 0, "probs", None),
         (None, None, 1, "labels", None),
         (0.15, 0.45, 0, "labels", "ragged")]


def _inputs(w, frames, spec, k, f):
    nu, tau, storage, cls, keep = spec
    pts, lab = f.points, f.labels
    if keep == "ragged":
        n = [0, 4097, 13, len(pts)][k % 4]     # empty scan, ragged sizes, full scan
        pts, lab = pts[:n], lab[:n]
    probs = _probs(lab, w.n_classes, 100 + k) if cls == "probs" else None
    return pts, (None if cls == "probs" else lab), probs


@pytest.fixture(scope="module")
def batch_run():
    p = _lib()
    w = synth.line16()
    frames = list(synth.sequence(w, 8))
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    seq, bat = [], []
    for s in SPECS:
        nu = s[0] or w.voxel_size
        tau = s[1] or w.truncation
        seq.append(_new_map(p, w, nu, tau, s[2]))
        bat.append(_new_map(p, w, nu, tau, s[2]))
    b = p.map_batch_create([m.h for m in bat], p.MAP_BATCH_GRAPH | p.MAP_BATCH_AUTOTUNE)
    om = oracle.OracleMap(w.voxel_size, w.truncation, w.n_classes)
    assert SPECS[0][0] is None and SPECS[0][1] is None
    ls = Lockstep(seq[0], om)
    stats_seq, stats_bat, configs = [], [], []
    for k, f in enumerate(frames):
        ins = [_inputs(w, frames, s, k, f) for s in SPECS]
        dev = [(_dev(pt), None if lb is None else _dev(lb), None if pr is None else _dev(pr)) for pt, lb, pr in ins]
        for i, (m, (pt, lb, pr)) in enumerate(zip(seq, dev)):
            if i == 0:        # map 0 in lockstep with the oracle (recorded decisions accepted)
                ls.scan(L, w.lidar, ins[0][0], f.T, labels=ins[0][1], probs=ins[0][2])
            else:
                m.integrate(L, pt, f.T, labels=lb, probs=pr)
        p.map_batch_integrate(b, [m.h for m in bat], [L] * len(bat), [d[0] for d in dev], [f.T] * len(bat),
                              labels=[d[1] for d in dev], probs=[d[2] for d in dev])
        p.map_batch_sync(b)
        configs.append(p.map_batch_config(b))
        stats_seq.append([m.stats() for m in seq])
        stats_bat.append([m.stats() for m in bat])
    yield dict(p=p, w=w, seq=seq, bat=bat, b=b, om=om, stats_seq=stats_seq, stats_bat=stats_bat, configs=configs,
               n_frames=len(frames))
    p.map_batch_destroy(b)
    for m in seq + bat:
        m.close()


def test_batch_counters_match_sequential(batch_run):
    for k, (ss, sb) in enumerate(zip(batch_run["stats_seq"], batch_run["stats_bat"])):
        for i, (a, c) in enumerate(zip(ss, sb)):
            for name in COUNTERS:
                assert a[name] == c[name], (k, i, name, a[name], c[name])
    # every map did real work except the empty-scan frames of the ragged one
    assert all(s[0]["voxels_updated"] > 10000 for s in batch_run["stats_bat"])
    assert batch_run["stats_bat"][0][3]["valid_points"] == 0


def test_batch_voxels_bit_identical(batch_run):
    for m_s, m_b in zip(batch_run["seq"], batch_run["bat"]):
        cs, cb = _sorted(m_s.blocks()), _sorted(m_b.blocks())
        assert np.array_equal(cs, cb)
        gs, gb = m_s.read_blocks(cs), m_b.read_blocks(cs)
        for key in ("D", "W", "label", "logP"):
            if gs[key] is None:
                continue
            assert np.array_equal(gs[key].view(np.uint8), gb[key].view(np.uint8)), key


def test_batch_mesh_identical(batch_run):
    for m_s, m_b in zip(batch_run["seq"], batch_run["bat"]):
        a = {k: v.cpu().numpy() for k, v in m_s.mesh().items()}
        c = {k: v.cpu().numpy() for k, v in m_b.mesh().items()}
        assert a["positions"].shape == c["positions"].shape and a["triangles"].shape == c["triangles"].shape
        ta = {tuple(t) for t in a["vertex_keys"][a["triangles"]].tolist()}
        tc = {tuple(t) for t in c["vertex_keys"][c["triangles"]].tolist()}
        assert ta == tc
        oa, oc = np.argsort(a["vertex_keys"], kind="stable"), np.argsort(c["vertex_keys"], kind="stable")
        assert np.array_equal(a["vertex_keys"][oa], c["vertex_keys"][oc])
        assert np.array_equal(a["positions"][oa], c["positions"][oc])
        assert np.array_equal(a["colors"][oa], c["colors"][oc])


def test_batch_map_against_oracle(batch_run):
    w, om, gm = batch_run["w"], batch_run["om"], batch_run["bat"][0]
    coords = _sorted(gm.blocks())
    assert np.array_equal(coords, _sorted(om.alloc_blocks()))
    compare_blocks(gm, om, coords, w.voxel_size, batch_run["n_frames"], w.n_classes)
    g = {k: v.cpu().numpy() for k, v in gm.mesh().items()}
    compare_meshes(g, om.mesh(), om, w.voxel_size)


def test_batch_and_single_calls_on_one_map():
    """Batched steps and single integrate_scan calls mixed on the same map: each call leaves the
    range image and counters for the next one (the batch kernel resets the set it uses itself, a
    single call's per-point kernel resets the other set), so the result must equal, bit for bit,
    a map that took every scan through integrate_scan, and so must every per-scan counter."""
    p = _lib()
    w = synth.line16()
    frames = list(synth.sequence(w, 8))
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    ref = _new_map(p, w, w.voxel_size, w.truncation, 0)
    mix = _new_map(p, w, w.voxel_size, w.truncation, 0)
    b = p.map_batch_create([mix.h], p.MAP_BATCH_GRAPH)
    for k, f in enumerate(frames):
        pt, lb = _dev(f.points), _dev(f.labels)
        ref.integrate(L, pt, f.T, labels=lb)
        if k in (0, 1, 4, 7):
            p.map_batch_integrate(b, [mix.h], [L], [pt], [f.T], labels=[lb])
            p.map_batch_sync(b)
        else:
            mix.integrate(L, pt, f.T, labels=lb)
        sr, sm = ref.stats(), mix.stats()
        for key in COUNTERS:
            assert sr[key] == sm[key], (k, key, sr[key], sm[key])
    cr = _sorted(ref.blocks())
    assert np.array_equal(cr, _sorted(mix.blocks()))
    gr, gm = ref.read_blocks(cr), mix.read_blocks(cr)
    for key in ("D", "W", "label", "logP"):
        assert np.array_equal(gr[key].view(np.uint8), gm[key].view(np.uint8)), key
    p.map_batch_destroy(b)
    ref.close()
    mix.close()


@pytest.mark.parametrize("graph", [False, True], ids=["streams", "streams-graph"])
def test_streams_batch_matches_single_calls(graph):
    """MAP_BATCH_STREAMS: every map's scan runs on a stream of the batch, all maps concurrently (with
    MAP_BATCH_GRAPH: the step captured and replayed as one graph launch).  The maps (different voxel
    sizes, storage precisions and class inputs, ragged and empty scans, one in the non-projective
    distance mode, which the batch kernel does not take) must equal maps fed single integrate_scan
    calls, bit for bit, with the same counters (the download ring's too)."""
    p = _lib()
    w = synth.line16()
    frames = list(synth.sequence(w, 5))
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)

    def maps():
        out = [_new_map(p, w, s[0] or w.voxel_size, s[1] or w.truncation, s[2]) for s in SPECS]
        out.append(p.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, distance="nonprojective",
                                  max_blocks=32768, hash_capacity=1 << 16, max_points=32768, max_pixels=32768,
                                  mesh_vertex_capacity=1 << 22, mesh_triangle_capacity=1 << 23))
        return out
    specs = SPECS + [(None, None, 0, "labels", None)]
    seq, con = maps(), maps()
    b = p.map_batch_create([m.h for m in con], p.MAP_BATCH_STREAMS | (p.MAP_BATCH_GRAPH if graph else 0))
    for k, f in enumerate(frames):
        ins = [_inputs(w, frames, s_, k, f) for s_ in specs]
        dev = [(_dev(pt), None if lb is None else _dev(lb), None if pr is None else _dev(pr)) for pt, lb, pr in ins]
        for m, (pt, lb, pr) in zip(seq, dev):
            m.integrate(L, pt, f.T, labels=lb, probs=pr)
        p.map_batch_integrate(b, [m.h for m in con], [L] * len(con), [d[0] for d in dev], [f.T] * len(con),
                              labels=[d[1] for d in dev], probs=[d[2] for d in dev])
        p.map_batch_sync(b)
        for i, (ms, mc) in enumerate(zip(seq, con)):
            a, c = ms.stats(), mc.stats()
            for name in COUNTERS + ("dirty_blocks",):
                assert a[name] == c[name], (k, i, name, a[name], c[name])
            assert mc.frame_stats(k)["voxels_updated"] == a["voxels_updated"]
    for ms, mc in zip(seq, con):
        cs = _sorted(ms.blocks())
        assert np.array_equal(cs, _sorted(mc.blocks()))
        gs, gc = ms.read_blocks(cs), mc.read_blocks(cs)
        for key in ("D", "W", "label", "logP"):
            assert np.array_equal(gs[key].view(np.uint8), gc[key].view(np.uint8)), key
    p.map_batch_destroy(b)
    for m in seq + con:
        m.close()


def test_streams_batch_refusal_leaves_that_map_alone():
    """Streams mode: a map whose scan is refused (a pose that is not a rotation) keeps its state, the
    other map of the step is fused, and the refusal is returned."""
    p = _lib()
    w = synth.line16()
    f = next(iter(synth.sequence(w, 1)))
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    a, c = _new_map(p, w, w.voxel_size, w.truncation, 0), _new_map(p, w, w.voxel_size, w.truncation, 0)
    b = p.map_batch_create([a.h, c.h], p.MAP_BATCH_STREAMS)
    bad = f.T.copy()
    bad[0, 0] *= 1.01
    pt, lb = _dev(f.points), _dev(f.labels)
    with pytest.raises(p.MapError) as e:
        p.map_batch_integrate(b, [a.h, c.h], [L, L], [pt, pt], [f.T, bad], labels=[lb, lb])
    assert e.value.status == 4
    p.map_batch_sync(b)
    assert a.stats()["valid_points"] > 0 and a.stats()["total_blocks"] > 0
    assert c.stats()["total_blocks"] == 0 and c.frame_count() == 0
    p.map_batch_destroy(b)
    a.close()
    c.close()


def test_autotuner_visits_every_configuration(batch_run):
    p = batch_run["p"]
    # 8 steps: the tuner is still timing (3 steps per configuration)
    assert all(not c["tuned"] for c in batch_run["configs"])
    b = batch_run["b"]
    for i in range(6):
        p.map_batch_set_config(b, i)
        c = p.map_batch_config(b)
        assert c["threads_per_block"] in (128, 256) and c["items_per_thread"] in (1, 2, 4)
    p.map_batch_set_config(b, -1)


def test_autotuner_settles_on_a_configuration():
    p = _lib()
    w = synth.line16()
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    m = _new_map(p, w, w.voxel_size, w.truncation, 1)
    b = p.map_batch_create([m.h], p.MAP_BATCH_GRAPH | p.MAP_BATCH_AUTOTUNE)
    frames = list(synth.sequence(w, 10))
    for k in range(20):                       # 6 configurations x 3 timed steps, then the choice
        f = frames[k % 10]
        p.map_batch_integrate(b, [m.h], [L], [_dev(f.points)], [f.T], labels=[_dev(f.labels)])
    p.map_batch_sync(b)
    c = p.map_batch_config(b)
    assert c["tuned"] and c["threads_per_block"] in (128, 256) and c["items_per_thread"] in (1, 2, 4)
    p.map_batch_destroy(b)
    m.close()


def test_batch_barrier_timeout_reports_and_recovers():
    p = _lib()
    w = synth.line16()
    frames = list(synth.sequence(w, 3))
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    ref = _new_map(p, w, w.voxel_size, w.truncation, 0)
    m = _new_map(p, w, w.voxel_size, w.truncation, 0)
    b = p.map_batch_create([m.h], p.MAP_BATCH_GRAPH)
    p.map_batch_set_config(b, 4)

    def step(f):
        p.map_batch_integrate(b, [m.h], [L], [_dev(f.points)], [f.T], labels=[_dev(f.labels)])

    ref.integrate(L, _dev(frames[0].points), frames[0].T, labels=_dev(frames[0].labels))
    step(frames[0])
    p.map_batch_sync(b)
    p.map_batch_test_timeout(b, 2000)
    step(frames[1])
    with pytest.raises(p.MapError) as e:
        p.map_batch_sync(b)
    assert e.value.status == 5
    # the failed step fused nothing; the next one runs normally
    ref.integrate(L, _dev(frames[2].points), frames[2].T, labels=_dev(frames[2].labels))
    step(frames[2])
    p.map_batch_sync(b)
    a, c = ref.stats(), m.stats()
    for name in COUNTERS:
        assert a[name] == c[name], name
    p.map_batch_destroy(b)
    ref.close()
    m.close()


def test_batch_argument_errors():
    p = _lib()
    with pytest.raises(p.MapError):
        p.map_batch_create([])
    w = synth.line16()
    m1 = _new_map(p, w, w.voxel_size, w.truncation, 0)
    m2 = _new_map(p, w, w.voxel_size, w.truncation, 0)
    b = p.map_batch_create([m1.h])
    f = next(iter(synth.sequence(w, 1)))
    L = p.lidar_intrinsics(w.lidar.H, w.lidar.W, w.lidar.fov_up, w.lidar.fov_down, w.lidar.r_min, w.lidar.r_max)
    with pytest.raises(p.MapError) as e:       # descriptor names a map outside the batch
        p.map_batch_integrate(b, [m2.h], [L], [_dev(f.points)], [f.T], labels=[_dev(f.labels)])
    assert e.value.status == 1
    with pytest.raises(p.MapError):            # bad configuration index
        p.map_batch_set_config(b, 6)
    p.map_batch_destroy(b)
    m1.close()
    m2.close()
