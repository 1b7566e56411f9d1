"""Pins of the hanging-node oracle (Appendix "Extension of DSS algorithms onto Non-Conforming
Interfaces"): the constrained gather reproduces polynomials of the coarse space exactly, the
constrained mass matrix integrates the volume, constants span the Laplacian's kernel, and the
assembled operator is symmetric."""
import numpy as np
import pytest

import oracle as O


CASES = [(4, (1, 1, 1), (3, 2, 3), 1), (4, (1, 1, 1), (2, 3, 2), 2), (5, (1, 2, 1), (3, 4, 3), 3)]


@pytest.mark.parametrize("mc,lo,hi,p", CASES)
def test_constrained_gather_reproduces_polynomials(mc, lo, hi, p):
    ad = O.Adaptive(mc, lo, hi, p)
    # nodal values of u = x^p y + z^p (degree <= p per direction) at every global DoF, read back
    # at every copy from the copies' own coordinates
    n, n3 = p + 1, (p + 1) ** 3
    xyz = np.zeros((ad.length, 3))
    for c in np.nonzero(ad.active)[0]:
        cr = ad.cell_corners(int(c))
        h = cr[7] - cr[0]
        for a in range(n3):
            ijk = (a % n, (a // n) % n, a // (n * n))
            xyz[c * n3 + a] = cr[0] + h * ad.t[list(ijk)]
    u = lambda X: X[:, 0] ** p * X[:, 1] + X[:, 2] ** p  # noqa: E731
    # global values: from the copies that carry a DoF with weight 1 alone
    G = ad.G.tocsr()
    one = np.asarray((G != 0).sum(axis=1)).ravel() == 1
    ug = np.zeros(ad.n_unique)
    rows = np.nonzero(one & ad.active_entries)[0]
    ug[G.indices[G.indptr[rows]]] = u(xyz[rows])
    uc = ad.gather(ug)
    act = ad.active_entries
    assert np.abs(uc[act] - u(xyz[act])).max() <= 1e-13
    assert np.all(uc[~act] == 0)


@pytest.mark.parametrize("mc,lo,hi,p", CASES[:2])
def test_constrained_operators(mc, lo, hi, p):
    ad = O.Adaptive(mc, lo, hi, p)
    one = ad.gather(np.ones(ad.n_unique))
    mass1 = ad.scatter(ad.apply_local(O.MASS, one))
    assert abs(mass1.sum() - 1.0) <= 1e-12  # the unit cube's volume
    lap1 = ad.scatter(ad.apply_local(O.LAPLACE, one))
    assert np.abs(lap1).max() <= 1e-12
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(ad.n_unique), rng.standard_normal(ad.n_unique)
    for op in (O.LAPLACE, O.MASS):
        ax = ad.scatter(ad.apply_local(op, ad.gather(x)))
        ay = ad.scatter(ad.apply_local(op, ad.gather(y)))
        assert abs(ax @ y - ay @ x) <= 1e-12 * abs(ax @ y)


def test_dss_is_a_projection_up_to_multiplicity():
    """S = G_c G_c^T: on a continuous vector u = G_c u_g, D^{-1} S u = u with D = G_c^T G_c's
    action read back (the constrained multiplicity), i.e. S maps continuous vectors to continuous
    vectors and reproduces them after the weighted average."""
    ad = O.Adaptive(4, (1, 1, 1), (3, 3, 2), 2)
    ug = np.random.default_rng(1).standard_normal(ad.n_unique)
    uc = ad.gather(ug)
    GtG = (ad.G.T @ ad.G).tocsr()
    assert np.abs(ad.dss(uc) - ad.gather(GtG @ ug)).max() <= 1e-12 * np.abs(uc).max()
