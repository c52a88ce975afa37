"""Pins of the oracle's moment-space algebra against definitions that do not
come from the oracle itself: the textbook D2Q9 equilibrium, Guo's
velocity-space forcing, rational identities of M, and the isotropy and
conservation properties the collision (Eq. 25) must have."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

# Velocity set and lattice weights typed here from the textbook D2Q9 model
# (independent of the oracle's own tables).
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
T_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def feq_textbook(rho, ux, uy):
    eu = EX * ux + EY * uy
    u2 = ux * ux + uy * uy
    return T_W * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * u2)


def guo_force(ux, uy, Fx, Fy):
    """Guo et al. (2002) forcing in velocity space, c_s^2 = 1/3."""
    eu = EX * ux + EY * uy
    return T_W * (3 * ((EX - ux) * Fx + (EY - uy) * Fy) + 9 * eu * (EX * Fx + EY * Fy))


def test_velocity_set_and_interaction_weights():
    ex, ey, w = O.velocities()
    assert list(ex) == list(EX) and list(ey) == list(EY)
    # Eq. 7: w(1) = 1/3, w(2) = 1/12
    np.testing.assert_array_equal(w[1:5], [1 / 3] * 4)
    np.testing.assert_array_equal(w[5:], [1 / 12] * 4)
    # isotropy used by Eq. 11 and Eq. 24: sum w e_x^2 = 1, sum w e_x^4 = 1, sum w e_x^2 e_y^2 = 1/3
    assert abs((w * ex**2).sum() - 1) < 1e-15
    assert abs((w * ex**4).sum() - 1) < 1e-15
    assert abs((w * ex**2 * ey**2).sum() - 1 / 3) < 1e-15


def test_M_rows_orthogonal_and_inverse_exact():
    M, Mi = O.matrices()
    Mf = [[Fraction(int(v)) for v in row] for row in M]
    gram = [[sum(Mf[i][k] * Mf[j][k] for k in range(9)) for j in range(9)] for i in range(9)]
    for i in range(9):
        for j in range(9):
            if i != j:
                assert gram[i][j] == 0
    assert [gram[i][i] for i in range(9)] == [9, 36, 36, 6, 12, 6, 12, 4, 4]
    np.testing.assert_allclose(M @ Mi, np.eye(9), atol=1e-15)
    np.testing.assert_allclose(Mi @ M, np.eye(9), atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_meq_equals_M_times_textbook_equilibrium(seed):
    """Eq. 4 is M f_eq of the second-order equilibrium: pins M's rows, the
    velocity order and the moment order (reading R1)."""
    rng = np.random.default_rng(seed)
    M, _ = O.matrices()
    for _ in range(20):
        rho = rng.uniform(0.01, 6.0)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        np.testing.assert_allclose(M @ feq_textbook(rho, ux, uy), O.meq(rho, ux, uy),
                                   rtol=0, atol=1e-14 * max(rho, 1))


@pytest.mark.parametrize("seed", [3, 4])
def test_S_equals_M_times_guo_forcing(seed):
    """Eq. 6 is M F_bar with Guo's forcing; its ninth entry is v_x F_y + v_y F_x (R6)."""
    rng = np.random.default_rng(seed)
    M, _ = O.matrices()
    for _ in range(20):
        ux, uy, Fx, Fy = rng.uniform(-0.3, 0.3, 4)
        np.testing.assert_allclose(M @ guo_force(ux, uy, Fx, Fy), O.source_s(ux, uy, Fx, Fy),
                                   rtol=0, atol=1e-14)


def _collide_moments(p, f, Fx, Fy, Q):
    M, _ = O.matrices()
    return M @ O.collide_node(p, f, Fx, Fy, *Q)


def test_collision_conserves_mass_and_adds_force():
    rng = np.random.default_rng(5)
    p = O.Params(s=[1.0, 1.3, 0.7, 1.2, 1.5, 0.8, 1.1, 1.4, 1.6], kappa=0.4)
    for _ in range(20):
        f = feq_textbook(rng.uniform(0.1, 1), *rng.uniform(-0.1, 0.1, 2)) * rng.uniform(0.9, 1.1, 9)
        Fx, Fy = rng.uniform(-0.01, 0.01, 2)
        Q = rng.uniform(-0.01, 0.01, 3)
        fs = O.collide_node(p, f, Fx, Fy, *Q)
        assert abs(fs.sum() - f.sum()) < 1e-15
        # momentum gains exactly F per step whatever s_j is (R2: rho v = j + F/2)
        assert abs((fs * EX).sum() - (f * EX).sum() - Fx) < 1e-15
        assert abs((fs * EY).sum() - (f * EY).sum() - Fy) < 1e-15


def test_source_C_is_isotropic_and_leaves_normal_stress_of_flat_interface():
    """The change of the second-moment tensor sum f* e e caused by Q must be
    -s_nu (Q - tr(Q) I / 2) in its traceless part for any orientation of Q
    (reading R4: xx-yy and xy scaled alike), and its trace part follows
    C[1] = 1.5 s_e tr(Q)."""
    s_nu, s_e = 1.3, 0.9
    p = O.Params(s=[1, s_e, 1.1, 1, 1.1, 1, 1.1, s_nu, s_nu], kappa=1.0)
    f = feq_textbook(1.0, 0.0, 0.0)

    def dPi(Q):
        d = O.collide_node(p, f, 0.0, 0.0, *Q) - O.collide_node(p, f, 0.0, 0.0, 0.0, 0.0, 0.0)
        return np.array([[(d * EX * EX).sum(), (d * EX * EY).sum()],
                         [(d * EX * EY).sum(), (d * EY * EY).sum()]])

    rng = np.random.default_rng(6)
    for _ in range(10):
        qxx, qyy, qxy = rng.uniform(-1, 1, 3)
        Qm = np.array([[qxx, qxy], [qxy, qyy]])
        D = dPi((qxx, qyy, qxy))
        trQ = qxx + qyy
        np.testing.assert_allclose(D - np.trace(D) / 2 * np.eye(2), -s_nu * (Qm - trQ / 2 * np.eye(2)),
                                   atol=1e-14)
        # trace: e moment changes by 1.5 s_e trQ and sum f|e|^2 = (e + 4 rho)/3
        assert abs(np.trace(D) - 0.5 * s_e * trQ) < 1e-14


def test_source_C_entries():
    p = O.Params(s=[1, 1.2, 1.3, 1, 1.4, 1, 1.5, 1.6, 1.7])
    C = O.source_c(p, 0.3, 0.1, -0.2)
    np.testing.assert_allclose(C, [0, 1.5 * 1.2 * 0.4, 0, 0, 0, 0, 0, -1.6 * 0.2, 1.7 * 0.2], atol=1e-15)
    p.li_eps = True
    assert abs(O.source_c(p, 0.3, 0.1, -0.2)[2] + 1.5 * 1.3 * 0.4) < 1e-15
