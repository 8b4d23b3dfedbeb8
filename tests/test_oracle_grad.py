"""Pin of the oracle's reference gradient (forward-mode dual numbers) against
central finite differences of the direct FP64 oracle."""
import math

import numpy as np

import oracle as O
import workloads as W


def loss(xyz, tri, k, rule, a, b):
    Z = O.Mesh(xyz, tri).z_full(k, rule)
    return float(np.real(np.conj(a) @ Z @ b))


def test_dual_gradient_vs_central_differences():
    xyz, tri = W.octasphere(1, 0.4)
    xyz = W.jitter(xyz, tri, 0.03, 2)
    k = 2 * math.pi
    m = O.Mesh(xyz, tri)
    a = W.complex_gaussian(m.ne, 1)
    b = W.complex_gaussian(m.ne, 2)
    L, g, gk = m.loss_grad(k, 4, a, b)
    assert abs(L - loss(xyz, tri, k, 4, a, b)) <= 1e-12 * abs(L)
    h = 1e-5
    rng = np.random.default_rng(0)
    for v, c in [tuple(x) for x in rng.integers(0, [len(xyz), 3], size=(8, 2))]:
        xp = xyz.copy(); xp[v, c] += h
        xm = xyz.copy(); xm[v, c] -= h
        fd = (loss(xp, tri, k, 4, a, b) - loss(xm, tri, k, 4, a, b)) / (2 * h)
        assert abs(fd - g[v, c]) <= 1e-6 * np.abs(g).max(), (v, c, fd, g[v, c])
    fdk = (loss(xyz, tri, k + h, 4, a, b) - loss(xyz, tri, k - h, 4, a, b)) / (2 * h)
    assert abs(fdk - gk) <= 1e-6 * abs(gk)
