"""Node coordinates of structured meshes, i fastest: shape (nz+1, ny+1, nx+1, dim)."""
import math

import numpy as np


def uniform_nodes(n, lo, hi):
    """Uniform box; n = cells per axis (2 or 3 entries)."""
    dim = len(n)
    axes = [lo[d] + (hi[d] - lo[d]) * np.arange(n[d] + 1) / n[d] for d in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return np.stack(grids, axis=-1).astype(np.float64)


def perturbed_nodes_3d(n, amp=0.1, length=2.0 * math.pi):
    """x_i = xi_i + amp sin(xi_1) sin(xi_2) sin(xi_3) on [0, length]^3 (periodic-compatible)."""
    nodes = uniform_nodes(n, (0.0, 0.0, 0.0), (length,) * 3)
    s = np.sin(nodes[..., 0]) * np.sin(nodes[..., 1]) * np.sin(nodes[..., 2])
    return nodes + amp * s[..., None]


def perturbed_nodes_xy(n, amp=0.1, length=2.0 * math.pi):
    """The paper's curvilinear TGV mesh: x += amp sin x sin y, y += amp sin x sin y, z unchanged."""
    nodes = uniform_nodes(n, (0.0, 0.0, 0.0), (length,) * 3)
    s = np.sin(nodes[..., 0]) * np.sin(nodes[..., 1])
    out = nodes.copy()
    out[..., 0] += amp * s
    out[..., 1] += amp * s
    return out
