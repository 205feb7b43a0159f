"""Host-side checks of libsemtsdf that need no GPU.

- the shared library loads and exports every function declared in
  include/semtsdf.h;
- the marching-cubes case table it generates at load time agrees, case by
  case, with the oracle's runtime face walk (independent code, same rule);
- its class palette agrees with the oracle's.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "semtsdf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    import paper_2412_00291_b300 as p
    names = _header_functions()
    assert {"map_create", "integrate_scan", "extract_mesh", "query_sdf"} <= set(names)
    lib = ctypes.CDLL(p.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_mc_table_matches_oracle_face_walk():
    import paper_2412_00291_b300 as p
    table = p.map_mc_table()
    nu = 0.1
    for cs in range(256):
        m = oracle.OracleMap(nu, 0.3, n_classes=2)
        D = np.full(512, 1.0)
        W = np.zeros(512)
        for c in range(8):
            dx, dy, dz = c & 1, (c >> 1) & 1, c >> 2
            vi = dx + 8 * dy + 64 * dz
            D[vi] = -1.0 - 0.1 * c if (cs >> c) & 1 else 1.0 + 0.1 * c
            W[vi] = 1.0
        m.write_block([0, 0, 0], D, W)
        me = m.mesh()
        want = {tuple(t) for t in me["tkeys"].tolist()}
        got = set()
        for j in range(p.MC_MAXTRI):
            tri = table[cs, j]
            if tri[0] < 0:
                break
            keys = []
            for ce in tri:
                axis, d1, d2 = ce >> 2, ce & 1, (ce >> 1) & 1
                off = [0, 0, 0]
                off[(axis + 1) % 3] = d1
                off[(axis + 2) % 3] = d2
                keys.append(oracle.edge_key(off[0], off[1], off[2], axis))
            got.add(tuple(keys))
        assert got == want, cs


def test_mc_table_uses_exactly_the_crossing_edges():
    """Every case with corners on both sides emits triangles, and its triangles use exactly the
    cube edges whose endpoints differ in sign (the mesh kernel marks vertex edges by sign
    changes next to fully observed cubes and relies on this)."""
    import paper_2412_00291_b300 as p
    table = p.map_mc_table()
    for cs in range(256):
        crossing = set()
        for ce in range(12):
            axis, d1, d2 = ce >> 2, ce & 1, (ce >> 1) & 1
            off = [0, 0, 0]
            off[(axis + 1) % 3] = d1
            off[(axis + 2) % 3] = d2
            c0 = off[0] + 2 * off[1] + 4 * off[2]
            c1 = c0 + (1 << axis)
            if ((cs >> c0) ^ (cs >> c1)) & 1:
                crossing.add(ce)
        used = {int(ce) for j in range(p.MC_MAXTRI) if table[cs, j, 0] >= 0 for ce in table[cs, j]}
        assert used == crossing, cs
        assert (len(used) > 0) == (cs not in (0, 255))


def test_mc_table_cases_fit_the_device_copy():
    """The device copy of the table keeps 5 triangle slots per case (map_create refuses a table with a
    larger case): every case has at most 5 triangles, the slots after a case's last triangle are -1,
    and the largest case does use 5 (the classic marching-cubes maximum)."""
    import paper_2412_00291_b300 as p
    table = p.map_mc_table()
    used = table[:, :, 0] >= 0
    n = used.sum(axis=1)
    assert n.max() == 5
    for cs in range(256):
        assert used[cs, :n[cs]].all() and not used[cs, n[cs]:].any(), cs
        assert (table[cs, n[cs]:] == -1).all(), cs


def test_palette_matches_oracle():
    import paper_2412_00291_b300 as p
    for C in (2, 7, 20, 64):
        np.testing.assert_array_equal(p.map_palette(C), oracle.palette(C))


def test_config_defaults():
    import paper_2412_00291_b300 as p
    cfg = p.map_config_default()
    assert cfg.voxel_size == pytest.approx(0.1) and cfg.truncation == pytest.approx(0.3)
    assert cfg.n_classes == 20 and cfg.weight_mode == 0 and cfg.storage == 0 and cfg.distance_mode == 0
    assert ctypes.sizeof(cfg) == 104


def _table_ii():
    """The traversability parameters of Table II, from the golden fixture (SI units, radians)."""
    import math
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table_ii_traversability.txt")):
        if line.strip() and not line.startswith("#"):
            name, value, unit = line.split()
            out[name] = math.radians(float(value)) if unit == "deg" else float(value)
    return out


def test_traversability_defaults_are_table_ii():
    """The library's and the oracle's defaults are Table II's (radius, height difference, steepness,
    roughness), every class allowed."""
    import inspect
    import math
    import paper_2412_00291_b300 as p
    from oracle.traversability import traversability
    g = _table_ii()
    t = p.TravParams()
    assert p._lib.map_trav_params_default(ctypes.byref(t)) == 0
    assert t.radius == pytest.approx(g["radius"]) and t.max_height_diff == pytest.approx(g["max_height_difference"])
    assert t.max_steepness == pytest.approx(g["max_steepness"]) and t.max_roughness == pytest.approx(g["max_roughness"])
    assert t.class_mask == (1 << 64) - 1
    assert p._lib.map_trav_params_default(None) != 0
    d = inspect.signature(traversability).parameters
    assert d["r"].default == pytest.approx(g["radius"]) and d["t_hd"].default == pytest.approx(g["max_height_difference"])
    assert math.radians(d["t_s_deg"].default) == pytest.approx(g["max_steepness"])
    assert math.radians(d["t_r_deg"].default) == pytest.approx(g["max_roughness"])


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror of a C struct of the header has the C compiler's size and field offsets."""
    import shutil
    import subprocess
    import paper_2412_00291_b300 as p
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    mirrors = {"map_config": p.MapConfig, "lidar_intrinsics": p.LidarIntrinsics, "mesh_view": p.MeshView,
               "scan_desc": p.ScanDesc, "trav_params": p.TravParams, "camera_intrinsics": p.CameraIntrinsics,
               "quality_report": p.QualityReport}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "semtsdf.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def _poly_coeffs(name):
    """Coefficients of atan_p / asin_q from the generated header (highest degree first)."""
    import re
    txt = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2412_00291_b300", "csrc", "poly_approx.h")).read()
    body = txt[txt.index(name + "(float s)"):]
    body = body[:body.index("return")]
    return [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]


def _horner_fma32(coeffs, s):
    # float32 Horner with a single rounding per step (as fmaf)
    r = np.full_like(s, coeffs[0], dtype=np.float64)
    for c in coeffs[1:]:
        r = (r * s.astype(np.float64) + np.float32(c)).astype(np.float32).astype(np.float64)
    return r


def test_projection_polynomials_meet_their_bounds():
    """The voxel-projection polynomials (atan on [0, 1], asin on [0, 1/2]) against numpy's
    double-precision arctan / arcsin: below 2e-7 rad, far inside the 1e-3-pixel margin
    (3e-6 rad for 2048 columns, 1.2e-5 rad for 64 beams over 45 deg)."""
    t = np.linspace(0.0, 1.0, 400001).astype(np.float32)
    a = t.astype(np.float64) * _horner_fma32(_poly_coeffs("atan_p"), (t * t).astype(np.float32))
    assert np.abs(a - np.arctan(t.astype(np.float64))).max() < 2e-7
    c = np.linspace(0.0, 0.5, 400001).astype(np.float32)
    b = c.astype(np.float64) * _horner_fma32(_poly_coeffs("asin_q"), (c * c).astype(np.float32))
    assert np.abs(b - np.arcsin(c.astype(np.float64))).max() < 2e-7


def test_extract_mesh_noalloc_wrapper_rejects_bad_buffers_before_any_call():
    """The Python binding checks buffer lengths and devices before calling the library: a
    mismatch raises ValueError (CPU tensors here, so nothing could be launched anyway)."""
    import torch

    import paper_2412_00291_b300 as p
    ok = dict(positions=torch.zeros((8, 3)), colors=torch.zeros((8, 4), dtype=torch.uint8),
              vertex_keys=torch.zeros(8, dtype=torch.int64), triangles=torch.zeros((5, 3), dtype=torch.int32),
              triangle_anchors=torch.zeros((5, 3), dtype=torch.int32))
    for name, short in (("colors", torch.zeros((7, 4), dtype=torch.uint8)),
                        ("vertex_keys", torch.zeros(4, dtype=torch.int64)),
                        ("triangle_anchors", torch.zeros((4, 3), dtype=torch.int32))):
        bad = dict(ok, **{name: short})
        with pytest.raises(ValueError, match="equal lengths"):
            p.extract_mesh_noalloc(None, **bad)
    with pytest.raises(ValueError, match="current CUDA device"):
        p.extract_mesh_noalloc(None, **ok)


def test_scan_pose_range_check_through_the_c_abi():
    """Voxel coordinates must stay within |v| < 2^19 - 16 (block and mesh-vertex keys): the
    host-side pose check refuses a scan that could reach beyond, before any map is touched."""
    import paper_2412_00291_b300 as p
    cfg = p.map_config_default(voxel_size=0.1, truncation=0.3, n_classes=20)
    lid = p.lidar_intrinsics(64, 2048, np.radians(22.5), np.radians(-22.5), 0.5, 100.0)
    lim = (2 ** 19 - 16) * 0.1           # metres of the coordinate range at 0.1 m voxels
    T = np.eye(4)
    p.map_check_scan_pose(cfg, lid, T)
    for axis in range(3):
        for sign in (1.0, -1.0):
            T = np.eye(4)
            T[axis, 3] = sign * (lim - 100.0 - 0.3 - 0.2)      # just inside
            p.map_check_scan_pose(cfg, lid, T)
            T[axis, 3] = sign * (lim - 100.0 - 0.3 + 0.2)      # just beyond
            with pytest.raises(p.MapError) as e:
                p.map_check_scan_pose(cfg, lid, T)
            assert e.value.status == 4 and "coordinate range" in str(e.value)
    # the other pose checks come through the same call
    T = np.eye(4)
    T[0, 0] = 1.01
    with pytest.raises(p.MapError) as e:
        p.map_check_scan_pose(cfg, lid, T)
    assert e.value.status == 4
    T = np.eye(4)
    T[1, 3] = np.nan
    with pytest.raises(p.MapError):
        p.map_check_scan_pose(cfg, lid, T)
