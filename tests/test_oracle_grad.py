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


def test_masked_gradient_and_dk_agree_with_full():
    xyz, tri = W.octasphere(1, 0.5)
    xyz = W.jitter(xyz, tri, 0.03, 4)
    k = 2 * math.pi
    m = O.Mesh(xyz, tri)
    a = W.complex_gaussian(m.ne, 5)
    b = W.complex_gaussian(m.ne, 6)
    L, g, gk = m.loss_grad(k, 3, a, b)
    v = 4
    mask = np.isin(np.arange(len(tri)), np.where((tri == v).any(axis=1))[0]).astype(np.int32)
    _, gm, _ = m.loss_grad(k, 3, a, b, tri_mask=mask)
    np.testing.assert_allclose(gm[v], g[v], rtol=1e-12, atol=1e-12 * np.abs(g).max())
    L2, gk2 = m.loss_dk(k, 3, a, b)
    assert abs(L2 - L) <= 1e-12 * abs(L) and abs(gk2 - gk) <= 1e-12 * abs(gk)
