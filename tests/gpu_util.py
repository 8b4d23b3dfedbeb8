"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())
