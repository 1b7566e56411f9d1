"""Pins of the 2^3-packed storage oracle (Sec. 2.2, Table "tab:memory_overhead")."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S

GOLDEN = {1: (27, 3.38), 2: (125, 1.95), 3: (343, 1.59)}


@pytest.mark.parametrize("p", [1, 2, 3])
def test_storage_ratio_of_the_table(p):
    """Stored DoFs per unit and the asymptotic storage ratio (2p+1)^3 / (2p)^3 as printed."""
    mesh = O.Mesh((8, 8, 8), p)
    pk = O.Packed(mesh)
    stored, ratio = GOLDEN[p]
    assert pk.N ** 3 == stored
    assert round(stored / (2 * p) ** 3, 2) == ratio
    # on a finite mesh the unduplicated boundary keeps the ratio below the asymptote, which
    # (m/2)^3 (2p+1)^3 / (mp+1)^3 approaches as m grows
    assert pk.length / O.or_n_unique(mesh) < stored / (2 * p) ** 3
    big = 4096
    assert abs((big // 2) ** 3 * stored / (big * p + 1) ** 3 - stored / (2 * p) ** 3) < 0.005


@pytest.mark.parametrize("p,m,dirichlet", [(1, (4, 2, 2), False), (2, (2, 4, 2), True),
                                           (3, (2, 2, 4), False)])
def test_packed_operators_agree_with_the_cellwise_ones(p, m, dirichlet):
    mesh = O.Mesh(m, p, amp=0.1, dirichlet=dirichlet)
    pk = O.Packed(mesh)
    xg = S.primal_unique(m, p, seed=4, dirichlet=dirichlet)
    xu = pk.gather(xg)
    # every copy of a node inside a unit reads the same value
    assert np.array_equal(pk.to_cellwise(xu), O.gather(mesh, xg))
    for op in (O.LAPLACE, O.MASS):
        # assembling the unit-local products gives the assembled operator
        yg = pk.scatter(pk.apply_local(op, xu))
        assert np.abs(yg - O.apply_assembled(mesh, op, xg)).max() <= 1e-13 * np.abs(yg).max()
    # multiplicity: interface nodes between units only
    mult = pk.multiplicity()
    axes = sum(1 for c in m if c // 2 >= 2)  # directions with an interface between units
    assert mult.min() == 1 and mult.max() == 2 ** axes
    assert (1.0 / mult).sum() == pytest.approx(O.or_n_unique(mesh), rel=1e-12)
