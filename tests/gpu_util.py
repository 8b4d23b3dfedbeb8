"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def entry_rel_max(a, b, floor):
    """Largest per-entry relative error |a - b| / |b| over the entries with
    |b| >= floor * max |b| (below that floor an entry's error is judged
    against the matrix's scale by rel_max)."""
    mag = np.abs(b)
    big = mag >= floor * mag.max()
    return float((np.abs(a - b)[big] / mag[big]).max())
