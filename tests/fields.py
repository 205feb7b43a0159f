"""Test fixtures: seeded scans on pixel-centre rays and analytic voxel fields.

Nothing here computes a step of the mapping method; these build inputs
(points at chosen ranges, block contents from closed-form fields) that the
tests feed to the oracle and to the CUDA path alike.
"""
import math

import numpy as np

import synth

BV = 512


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def points_on_rays(lidar, ranges):
    """One float32 point per pixel at the given ranges (NaN range -> no return)."""
    d = lidar.ray_dirs()
    return (d * np.asarray(ranges, np.float64).reshape(-1, 1)).astype(np.float32)


def block_voxels(coord):
    """Integer voxel coordinates of a block, local index = x + 8 y + 64 z."""
    lz, ly, lx = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    v = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], axis=1)
    return v + 8 * np.asarray(coord, np.int64).reshape(1, 3)


def blocks_covering(lo, hi, nu):
    """Block coordinates whose voxel centres span the world box [lo, hi]."""
    vlo = np.floor(np.asarray(lo) / nu).astype(int)
    vhi = np.ceil(np.asarray(hi) / nu).astype(int)
    blo, bhi = np.floor_divide(vlo, 8), np.floor_divide(vhi, 8)
    g = np.meshgrid(*[np.arange(blo[k], bhi[k] + 1) for k in range(3)], indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1)


def write_field(target, fn, blocks, nu, n_classes=None, logp_fn=None, dtype=np.float64):
    """Write D = fn(x) (world metres), W = 1 into every listed block of `target`.

    `target` has write_block(coord, D, W, logP) (oracle map or CUDA map binding).
    """
    for b in blocks:
        v = block_voxels(b)
        x = v * nu
        D = np.asarray(fn(x), np.float64)
        W = np.ones(BV)
        lp = None if logp_fn is None else logp_fn(v)
        target.write_block(b, D.astype(dtype), W.astype(dtype), lp)
