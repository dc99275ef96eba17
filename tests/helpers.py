"""Shared test helpers: layout conversion between the oracle (full 2x2 tensors on the
last axes) and the C ABI (3 planes xx, yy, xy), and error measures."""
import numpy as np


def to3(t):
    """(ny, nx, 2, 2) -> (3, ny, nx) with planes xx, yy, xy."""
    return np.stack([t[..., 0, 0], t[..., 1, 1], t[..., 0, 1]])


def from3(a):
    """(3, ny, nx) -> (ny, nx, 2, 2)."""
    t = np.empty(a.shape[1:] + (2, 2))
    t[..., 0, 0] = a[0]
    t[..., 1, 1] = a[1]
    t[..., 0, 1] = a[2]
    t[..., 1, 0] = a[2]
    return t


def bar3(eps_bar):
    return (float(eps_bar[0, 0]), float(eps_bar[1, 1]), float(eps_bar[0, 1]))


def bar22(b3):
    return np.array([[b3[0], b3[2]], [b3[2], b3[1]]], dtype=float)


def rel_l2(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def tensor_rel_l2(a3, b3):
    """Relative L2 with the Frobenius weight (xy counted twice)."""
    w = np.array([1.0, 1.0, 2.0])[:, None, None]
    d = np.sum(w * (a3 - b3) ** 2)
    nb = np.sum(w * b3 ** 2)
    return float(np.sqrt(d / (nb if nb > 0 else 1.0)))
