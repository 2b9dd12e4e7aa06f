"""Host logic of the rising-bubble driver (rising_bubble.py): how (Eo, Re_Gr)
lists pair up into problems, the wall choice, and the groups of each problem
(the paper's Fig. 6 pairs from tests/golden/rising_bubble_setups.txt)."""
import argparse
import math

import pytest

import rising_bubble as RB
from test_golden_setups import SETUPS


def _args(**kw):
    a = dict(size=[64, 128, 64], D=16.0, eo=[10.0], re_gr=[31.6], rho_ratio=None, t_ref=500.0, q=27, walls="all")
    a.update(kw)
    return argparse.Namespace(**a)


def test_pairs_broadcast_and_mismatch():
    assert len(RB.problems(_args(eo=[30.0], re_gr=[10.0, 20.0, 40.0]))) == 3
    assert len(RB.problems(_args(eo=[1.0, 5.0], re_gr=[40.0]))) == 2
    with pytest.raises(SystemExit):
        RB.problems(_args(eo=[1.0, 5.0], re_gr=[10.0, 20.0, 40.0]))


def test_walls_and_density_ratio():
    (p_all, _), = RB.problems(_args())
    assert p_all.wall == (1, 1, 1)
    (p_tb, _), = RB.problems(_args(walls="top-bottom", rho_ratio=100.0))
    assert p_tb.wall == (0, 1, 0) and p_tb.rho_ratio == 100.0


def test_paper_pairs_give_the_printed_groups():
    fig6 = [r for r in SETUPS if r[0].startswith("fig6")]
    args = _args(eo=[r[1] for r in fig6], re_gr=[r[2] for r in fig6], D=32.0, t_ref=18000.0, size=[96, 192, 96])
    for (prob, phi0), row in zip(RB.problems(args), fig6):
        _, Eo, Re, D, t_ref = row[:5]
        g = -prob.gravity[1]
        assert math.sqrt(D / g) == pytest.approx(t_ref, rel=1e-12)
        assert g * prob.rho_H * D * D / prob.sigma == pytest.approx(Eo, rel=1e-12)
        assert prob.rho_H * math.sqrt(g * D ** 3) / (prob.rho_H * prob.nu_H) == pytest.approx(Re, rel=1e-12)
        assert phi0.shape == prob.shape and phi0.min() < 0.01 and phi0.max() > 0.99  # a light bubble in heavy fluid
