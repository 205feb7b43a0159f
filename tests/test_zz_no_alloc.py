"""extract_mesh_noalloc, the mesh extraction that allocates nothing.

Some callers cannot allocate device memory: a real-time loop that must not
block on cudaMalloc, or a host framework that reserved all of the GPU's
memory up front and hands the library only buffers it owns.  For them the
library offers extract_mesh_noalloc, which writes into the caller's buffers
and keeps its scratch in one static device array shared by all calls.  This
test checks, through the C ABI, that it returns exactly what extract_mesh
returns, on two calls in a row with the map changing in between (the shared
scratch still holds the previous call's contents), that the second call
leaves the device's free memory and torch's allocator untouched, that a
too-small buffer is refused with the needed sizes, and that a pool larger
than the static scratch, or a host buffer, is refused before any launch.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


def _buffers(nv, nt):
    return dict(positions=torch.empty((nv, 3), dtype=torch.float32, device="cuda"),
                colors=torch.empty((nv, 4), dtype=torch.uint8, device="cuda"),
                vertex_keys=torch.empty(nv, dtype=torch.int64, device="cuda"),
                triangles=torch.empty((nt, 3), dtype=torch.int32, device="cuda"),
                triangle_anchors=torch.empty((nt, 3), dtype=torch.int32, device="cuda"))


def test_extract_mesh_noalloc_matches_extract_mesh():
    import paper_2412_00291_b300 as P
    w = synth.line16()
    L = w.lidar
    lid = P.lidar_intrinsics(L.H, L.W, L.fov_up, L.fov_down, L.r_min, L.r_max)
    gm = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=32768, hash_capacity=1 << 16,
                        max_points=32768, max_pixels=32768, mesh_vertex_capacity=1 << 22,
                        mesh_triangle_capacity=1 << 23)
    frames = list(synth.sequence(w, 4))

    def fuse(f):
        gm.integrate(lid, torch.from_numpy(f.points).cuda(), f.T, labels=torch.from_numpy(f.labels).cuda())

    fuse(frames[0])
    fuse(frames[1])
    bufs = _buffers(1 << 20, 1 << 21)
    sizes = []
    for call in range(2):
        fuse(frames[2 + call])
        ref = P.extract_mesh(gm.h)
        torch.cuda.synchronize()
        free0, alloc0, resv0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), \
            torch.cuda.memory_reserved()
        nv, nt = P.extract_mesh_noalloc(gm.h, **bufs)
        torch.cuda.synchronize()
        if call == 1:      # nothing allocated by the call itself (device or torch caching allocator)
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == resv0
        assert nv == ref["positions"].shape[0] and nt == ref["triangles"].shape[0]
        assert nt > 1000
        for name in ("positions", "colors", "vertex_keys", "triangles", "triangle_anchors"):
            n = nv if name in ("positions", "colors", "vertex_keys") else nt
            assert torch.equal(bufs[name][:n], ref[name]), (call, name)
        sizes.append((nv, nt))
    assert sizes[1] != sizes[0]          # the map changed between the two calls
    small = _buffers(16, 16)
    with pytest.raises(P.MapError) as e:
        P.extract_mesh_noalloc(gm.h, **small)
    assert e.value.status == 3
    assert f"{sizes[1][0]} vertices" in str(e.value) and f"{sizes[1][1]} triangles" in str(e.value)
    gm.close()


def test_extract_mesh_noalloc_refusals():
    """A pool beyond the scratch's 2^19 blocks and host buffers are refused with MAP_ERR_ARG
    before any kernel runs (the output counts stay untouched)."""
    import paper_2412_00291_b300 as P
    big = P.SemanticTSDF(0.2, 0.6, 2, max_blocks=(1 << 19) + 1, hash_capacity=1 << 21, max_points=1024,
                         max_pixels=1024, mesh_vertex_capacity=1024, mesh_triangle_capacity=1024, storage=1)
    bufs = _buffers(64, 64)
    with pytest.raises(P.MapError) as e:
        P.extract_mesh_noalloc(big.h, **bufs)
    assert e.value.status == 1 and "524288" in str(e.value)
    big.close()
    w = synth.line16()
    gm = P.SemanticTSDF(w.voxel_size, w.truncation, w.n_classes, max_blocks=4096, hash_capacity=1 << 13,
                        max_points=16384, max_pixels=16384, mesh_vertex_capacity=1 << 16,
                        mesh_triangle_capacity=1 << 17)
    host = np.zeros(64 * 4, np.float32)
    nv, nt = ctypes.c_int64(-7), ctypes.c_int64(-7)
    d = {k: ctypes.c_void_p(v.data_ptr()) for k, v in bufs.items()}
    st = P._lib.extract_mesh_noalloc(gm.h, ctypes.c_void_p(host.ctypes.data), d["colors"], d["vertex_keys"],
                                     d["triangles"], d["triangle_anchors"], 64, 64, ctypes.byref(nv),
                                     ctypes.byref(nt), P._stream(None))
    assert st == 1 and nv.value == -7 and nt.value == -7
    assert "not device memory" in P._lib.map_last_error(gm.h).decode()
    gm.close()
