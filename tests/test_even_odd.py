"""The even-odd form of the 1D kernels (Sec. 4.1), on the CPU.

The binary64 apply kernel evaluates the basis change S (Gauss-Lobatto
Lagrange polynomials at the Gauss points), the collocation derivative D on
the Gauss points and their transposes in even-odd form.  That rests on two
facts checked here with matrices built independently in numpy (product-form
Lagrange polynomials, numpy's Gauss-Legendre points): S is centrosymmetric
and D anti-centrosymmetric; and on the splitting algebra, restated here from
its definition and compared with the direct matrix-vector products.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

import ref1d


def _matrices(k):
    gl = ref1d.gl_nodes(k)
    g = 0.5 * (L.leggauss(k)[0] + 1.0)
    S = np.array([[ref1d._lagrange_eval(gl, i, np.array(gq))[0] for i in range(k)] for gq in g])
    D = np.array([[ref1d._lagrange_eval(g, j, np.array(gq))[1] for j in range(k)] for gq in g])
    return S, D


def _halves(M):
    """ME[q][i] = (M[q][i] + M[q][k-1-i]) / 2 (i < h), ME[q][h] = M[q][h] for
    odd k, MO[q][i] = (M[q][i] - M[q][k-1-i]) / 2, rows q < (k+1)/2."""
    k = M.shape[0]
    h, h2 = k // 2, (k + 1) // 2
    ME = np.zeros((h2, h2))
    MO = np.zeros((h2, max(h, 1)))
    for q in range(h2):
        for i in range(h):
            ME[q, i] = 0.5 * (M[q, i] + M[q, k - 1 - i])
            MO[q, i] = 0.5 * (M[q, i] - M[q, k - 1 - i])
        if k % 2:
            ME[q, h] = M[q, h]
    return ME, MO


def _even_odd_apply(ME, MO, u, anti):
    k = len(u)
    h, h2 = k // 2, (k + 1) // 2
    e = np.array([u[i] + u[k - 1 - i] for i in range(h)] + ([u[h]] if k % 2 else []))
    o = np.array([u[i] - u[k - 1 - i] for i in range(h)])
    out = np.zeros(k)
    for q in range(h):
        ev = ME[q, :h2] @ e
        od = MO[q, :h] @ o
        out[q] = ev + od
        out[k - 1 - q] = od - ev if anti else ev - od
    if k % 2:
        out[h] = MO[h, :h] @ o if anti else ME[h, :h2] @ e
    return out


@pytest.mark.parametrize("k", range(2, 10))
def test_symmetry_of_the_1d_matrices(k):
    S, D = _matrices(k)
    R = np.eye(k)[::-1]  # reversal
    assert np.allclose(R @ S @ R, S, atol=1e-13)
    assert np.allclose(R @ D @ R, -D, atol=1e-11 * max(1.0, np.abs(D).max()))
    # S reproduces polynomials: rows sum to one; D annihilates constants
    assert np.allclose(S.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-11 * max(1.0, np.abs(D).max()))


@pytest.mark.parametrize("k", range(2, 10))
def test_even_odd_apply_equals_direct_product(k):
    S, D = _matrices(k)
    rng = np.random.default_rng(k)
    for M, anti in ((S, False), (S.T, False), (D, True), (D.T, True)):
        ME, MO = _halves(M)
        for _ in range(3):
            u = rng.uniform(-1, 1, k)
            got = _even_odd_apply(ME, MO, u, anti)
            want = M @ u
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(M).sum()), (k, anti)


def test_even_odd_operation_count():
    """k - (k mod 2) sums, h pairs of (k+1)/2 + h products and a sum and a
    difference, plus the middle output: fewer operations than k^2 from k = 5."""
    import bench
    for k in range(2, 10):
        centro, anti = bench.even_odd_ops(k, False), bench.even_odd_ops(k, True)
        assert anti <= centro
        if k >= 5:
            assert centro < k * k
    assert bench.even_odd_ops(5, False) == 21 and bench.even_odd_ops(5, True) == 20


def test_flop_models_of_the_two_face_modes():
    """The face loop's flop count (bench roofline) is below the
    element-centric one at every degree: it drops the neighbour's
    re-interpolation and evaluates each side's flux once; the even-odd form
    lowers both from k = 5 on."""
    import bench
    for k in range(2, 10):
        for op in ("sipg", "advection"):
            for geom in ("full", "merged", "cartesian"):
                for eo in (False, True):
                    loop = bench.kernel_flops_per_cell_loop(k, op, geom, even_odd=eo)
                    elem = bench.kernel_flops_per_cell(k, op, geom, even_odd=eo)
                    assert 0 < loop < elem, (k, op, geom, eo)
                if k >= 5:
                    assert (bench.kernel_flops_per_cell_loop(k, op, geom, even_odd=True)
                            < bench.kernel_flops_per_cell_loop(k, op, geom, even_odd=False))
    # p = 4, G3 SIPG: 264 flop/dof with the even-odd sweeps (the x faces'
    # value traces are the x lines' end layers, without arithmetic)
    assert round(bench.kernel_flops_per_cell_loop(5, "sipg", "full", even_odd=True) / 125) == 264
