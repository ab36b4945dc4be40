"""Pins of the oracle's transfer operators (Section 3.2: "standard full
weighting and linear interpolation", read for cell-centred grids).

For nested grids (n_f = 2 n_c) the reading reduces to the textbook
cell-centred operators: interpolation 3/4 of the nearer coarse cell and 1/4
of the other one; full weighting (1, 3, 3, 1)/8 in the interior and, as the
row-normalised transpose of the interpolation with a constant ghost,
(4, 3, 1)/8 at the ends; a Dirichlet face's ghost is the negated end value
(zero correction on the face), so the end fine cell takes 3/4 - 1/4 = 1/2.
For odd sizes the reading is defined, not textbook: interpolation is
linear in the cell-centre coordinate, so it reproduces linear data away from
the ends; restriction rows sum to one and are the columns of the
interpolation scaled.  In several dimensions both are tensor products.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2606_04292_gb300 import workloads as W


def _oracle(n, kinds=None, dim=None):
    dim = dim or (len(n) if hasattr(n, "__len__") else 1)
    kinds = kinds or [W.NOFLUX] * (2 * dim - 2) + [W.FREE_DRAINAGE, W.DIRICHLET]
    p = W.random_problem(dim, n, W.GARDNER, 3, bc_kinds=kinds)
    return Oracle(p), p


def _matrices(o, lev=0):
    nf, nc = o.ncell(lev), o.ncell(lev + 1)
    R = np.stack([o.restrict(np.eye(nf)[i], lev) for i in range(nf)], axis=1)      # nc x nf
    P = np.stack([o.prolong_add(np.eye(nc)[j], np.zeros(nf), lev) for j in range(nc)], axis=1)   # nf x nc
    return R, P


def test_nested_1d_textbook_weights():
    o, _ = _oracle((16,), kinds=[W.NOFLUX, W.NOFLUX])
    R, P = _matrices(o)
    assert R.shape == (8, 16)
    for J in range(1, 7):
        assert np.array_equal(R[J, 2 * J - 1:2 * J + 3], np.array([1, 3, 3, 1]) / 8.0)
        assert np.count_nonzero(R[J]) == 4
    assert np.array_equal(R[0, :3], np.array([4, 3, 1]) / 8.0) and np.count_nonzero(R[0]) == 3
    assert np.array_equal(R[7, 13:], np.array([1, 3, 4]) / 8.0) and np.count_nonzero(R[7]) == 3
    for i in range(1, 15):
        J = i // 2
        other = J + 1 if i % 2 else J - 1
        assert P[i, J] == 0.75 and P[i, other] == 0.25 and np.count_nonzero(P[i]) == 2
    assert P[0, 0] == 1.0 and P[15, 7] == 1.0            # constant ghost on no-flux faces


def test_dirichlet_face_ghost_is_negated():
    o, _ = _oracle((16,), kinds=[W.DIRICHLET, W.NOFLUX])
    R, P = _matrices(o)
    assert P[0, 0] == 0.5 and np.count_nonzero(P[0]) == 1          # 3/4 c0 - 1/4 c0
    assert P[15, 7] == 1.0
    # the restriction does not see the boundary kind
    o2, _ = _oracle((16,), kinds=[W.NOFLUX, W.NOFLUX])
    assert np.array_equal(R, _matrices(o2)[0])


@pytest.mark.parametrize("n", [7, 9, 13, 21])
def test_odd_sizes_linear_reproduction_and_normalisation(n):
    o, _ = _oracle((n,), kinds=[W.NOFLUX, W.NOFLUX])
    R, P = _matrices(o)
    nc = (n + 1) // 2
    assert R.shape == (nc, n)
    assert np.allclose(R.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    # R is the transpose of the constant-ghost interpolation, rows normalised
    colsum = P.sum(axis=0)
    assert np.allclose(R, (P / colsum).T, rtol=0, atol=1e-15)
    # linear data in the cell-centre coordinate are reproduced away from the ends
    xf = (np.arange(n) + 0.5) / n
    xc = (np.arange(nc) + 0.5) / nc
    lin = P @ (2.0 - 3.0 * xc)
    inner = (xf > xc[0]) & (xf < xc[-1])
    assert np.max(np.abs(lin[inner] - (2.0 - 3.0 * xf[inner]))) <= 1e-14
    assert np.allclose(P @ np.ones(nc), 1.0, rtol=0, atol=1e-15)   # constants everywhere


@pytest.mark.parametrize("n", [(12, 10), (9, 16), (8, 6, 10), (7, 5, 9)])
def test_several_dimensions_are_tensor_products(n):
    dim = len(n)
    kinds = [W.NOFLUX] * (2 * dim)
    o, p = _oracle(n, kinds=kinds, dim=dim)
    rng = np.random.default_rng(4)
    axes_f = [rng.standard_normal(k) for k in n]
    fine = axes_f[0]
    for a in range(1, dim):
        fine = np.multiply.outer(axes_f[a], fine)              # [.., x] with x fastest
    got = o.restrict(fine.reshape(-1))
    want = None
    for a in range(dim):
        o1, _ = _oracle((n[a],), kinds=[W.NOFLUX, W.NOFLUX])
        r = o1.restrict(axes_f[a])
        want = r if want is None else np.multiply.outer(r, want)
    assert np.max(np.abs(got - want.reshape(-1))) <= 1e-14 * np.max(np.abs(want))
    nc = [max(1, (k + 1) // 2) for k in n]
    axes_c = [rng.standard_normal(k) for k in nc]
    coarse = axes_c[0]
    for a in range(1, dim):
        coarse = np.multiply.outer(axes_c[a], coarse)
    got = o.prolong_add(coarse.reshape(-1), np.zeros(int(np.prod(n))))
    want = None
    for a in range(dim):
        o1, _ = _oracle((n[a],), kinds=[W.NOFLUX, W.NOFLUX])
        q = o1.prolong_add(axes_c[a], np.zeros(n[a]))
        want = q if want is None else np.multiply.outer(q, want)
    assert np.max(np.abs(got - want.reshape(-1))) <= 1e-14 * np.max(np.abs(want))
