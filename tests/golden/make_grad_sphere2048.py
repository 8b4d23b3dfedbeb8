"""Writes grad_sphere2048.txt: the FP64 oracle's gradient of L = Re(a^H Z b)
for the 2048-triangle sphere (octasphere level 4, radius 1 lambda, vertices
jittered by U[+-2 %] of the mean edge length, seed 20190115; 6-point rule,
k = 2 pi; a, b seeded complex Gaussian vectors, seeds 7 and 8), computed by
the oracle's dual-number differentiation of its direct (sincos) fill. Calls
only oracle/ and the seeded workloads.

Format: line 1 'L dL/dk', then one line per vertex 'dL/dx dL/dy dL/dz'.
Run from the repository root: python tests/golden/make_grad_sphere2048.py
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    wl = W.sphere_3072()
    om = O.Mesh(wl.xyz, wl.tri)
    a = W.complex_gaussian(om.ne, 7)
    b = W.complex_gaussian(om.ne, 8)
    L, g, dk = om.loss_grad(2 * math.pi, 6, a, b)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grad_sphere2048.txt")
    with open(out, "w") as f:
        f.write(f"{L!r} {dk!r}\n")
        for row in np.asarray(g):
            f.write(" ".join(repr(float(x)) for x in row) + "\n")


if __name__ == "__main__":
    main()
