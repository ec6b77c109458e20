"""Small shared helpers for the tests (no smearing arithmetic here)."""

import numpy as np


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 (the absolute norm if b is zero)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    nd = np.linalg.norm((a - b).ravel())
    return float(nd if nb == 0 else nd / nb)


def per_vector_rel_l2(a, b):
    """Relative L2 error of each vector along axis 0."""
    return [rel_l2(a[v], b[v]) for v in range(np.asarray(b).shape[0])]


def sublattice_mask(dims, c):
    """Boolean [Lz, Ly, Lx] mask of the sites with (x&1, y&1, z&1) = bits of c."""
    Lx, Ly, Lz, _ = dims
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x & 1) == (c & 1)) & ((y & 1) == ((c >> 1) & 1)) & ((z & 1) == ((c >> 2) & 1))
