"""The operation count of the oracle's time step (oracle/op_count.cpp), the
numerator of the FP64 step's algorithmic roofline.

The counting rules are pinned on two pieces whose operations can be counted
by hand:
- the equilibrium moments of Eq. 4: |v|^2 = vx vx + vy vy (3); e and eps
  share 3 |v|^2: rho (-2 + 3 v^2) (3 more) and rho (1 - 3 v^2) (2 more);
  rho vx, rho vy (2; -rho vx and -rho vy are the same products negated);
  rho (vx vx - vy vy) (2: the squares exist already); rho vx vy (1 more:
  rho vx exists): 13;
- the forcing moments of Eq. 6: v.F (3), 6 v.F (1; -6 v.F is its negation),
  F_x, F_y and their negations (0), 2 (vx Fx - vy Fy) (2: both products
  exist), vx Fy + vy Fx (3): 9.
"""
import json
import os

import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def test_counting_rules_on_hand_counted_pieces():
    assert O.op_count("meq")["flops"] == 13
    assert O.op_count("source_s")["flops"] == 9


def test_count_per_node_does_not_depend_on_the_lattice():
    a = O.op_count(1, 8, 8)
    b = O.op_count(1, 16, 12)
    assert a == b
    assert a["flops_per_update"] == a["add_sub_per_update"] + a["mul_per_update"] + a["div_per_update"] + \
        a["sqrt_per_update"]
    # one square root per node (psi, Eq. 10); a handful of divisions (the EOS,
    # psi's radicand, the velocity of R2)
    assert a["sqrt_per_update"] == 1 and 4 <= a["div_per_update"] <= 12


@pytest.mark.parametrize("law", ["carnahan_starling", "van_der_waals", "peng_robinson"])
def test_committed_counts_are_current(law):
    from tests.golden import make_op_count as M
    with open(os.path.join(HERE, "golden", "oracle_op_count.json")) as fh:
        doc = json.load(fh)
    assert doc["counts"][law] == O.op_count(M.LAWS[law], *doc["lattice"])
