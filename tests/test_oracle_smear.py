"""Pins for the oracle's stout and over-improved stout smearing (Sec. II.B and
Sec. III: rho = 0.1 stout, rho = 0.06 / eps = -0.25 over-improved).

The strongest pin ties the staple sum to the action it differentiates: the
stout generator satisfies Q_a(x,mu) = 2 tr(T_a Q) = 6 rho dS/d eta_a, with
S = sum over loops of c_loop (1/3) Re tr U_loop (plaquettes weight
(5-2eps)/3, 2x1 rectangles of both orientations weight -(1-eps)/12) and
eta_a the direction U_mu(x) -> exp(i eta T_a) U_mu(x).  S is evaluated by
an independent loop enumerator (tests/helpers.py) and differentiated by
central differences, so a missing, misplaced or mis-oriented staple, or a
wrong weight, fails."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H

DIMS = (4, 4, 4, 4)


@pytest.mark.parametrize("eps", [1.0, 0.0, -0.25])
def test_stout_generator_is_action_gradient(eps):
    rho = 0.01
    U = synth.make_field(DIMS, 0.6, 12)
    Us = oracle.smear(DIMS, U, rho, eps, 1)
    cp, cr = (5 - 2 * eps) / 3, -(1 - eps) / 12
    T = oracle.generators()
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(6):
        x, mu = int(rng.integers(256)), int(rng.integers(4))
        Q = H.log_unitary(Us[x, mu] @ U[x, mu].conj().T)
        for a in range(8):
            Qa = 2 * np.real(np.trace(T[a] @ Q))
            diffs = []
            for s in (+1, -1):
                Up = U.copy()
                Up[x, mu] = scipy.linalg.expm(1j * s * h * T[a]) @ U[x, mu]
                diffs.append(H.loop_traces(DIMS, Up, cp, cr))
            dS = np.sum(diffs[0] - diffs[1]) / (2 * h)
            assert abs(Qa - 6 * rho * dS) < 1e-8, (x, mu, a, Qa, 6 * rho * dS)


@pytest.mark.parametrize("eps,rho", [(1.0, 0.1), (-0.25, 0.06)])
def test_smeared_links_stay_in_su3(eps, rho):
    U = synth.make_field(DIMS, 0.5, 3)
    S = oracle.smear(DIMS, U, rho, eps, 6)
    assert H.unitarity_error(S) < 1e-13


def test_rho_zero_is_identity():
    U = synth.make_field(DIMS, 0.5, 3)
    assert np.abs(oracle.smear(DIMS, U, 0.0, 1.0, 3) - U).max() < 1e-15
    assert np.abs(oracle.smear(DIMS, U, 0.0, -0.25, 3) - U).max() < 1e-15
    np.testing.assert_array_equal(oracle.smear(DIMS, U, 0.1, 1.0, 0), U)


@pytest.mark.parametrize("eps", [1.0, -0.25])
def test_gauge_covariance(eps):
    U = synth.make_field(DIMS, 0.5, 3)
    G = synth.random_gauge(DIMS, 9)
    a = oracle.smear(DIMS, oracle.apply_gauge(DIMS, U, G), 0.1, eps, 3)
    b = oracle.apply_gauge(DIMS, oracle.smear(DIMS, U, 0.1, eps, 3), G)
    assert np.abs(a - b).max() < 1e-12


def test_constant_abelian_field_is_fixed_point():
    """Constant diagonal links: every staple equals the link, Omega = C U^dag
    is a real multiple of 1, Q = 0, nothing moves."""
    V = 256
    U = np.zeros((V, 4, 3, 3), np.complex128)
    for mu in range(4):
        a, b = 0.3 * (mu + 1), -0.2 * mu
        U[:, mu] = np.diag(np.exp(1j * np.array([a, b, -a - b])))
    for eps in (1.0, -0.25):
        assert np.abs(oracle.smear(DIMS, U, 0.1, eps, 2) - U).max() < 1e-14


def test_smearing_raises_plaquette():
    U = synth.make_field(DIMS, synth.W_PLAQ_06, 1)
    p0 = oracle.plaquette(DIMS, U)
    p_stout = oracle.plaquette(DIMS, oracle.smear(DIMS, U, 0.1, 1.0, 4))
    p_oi = oracle.plaquette(DIMS, oracle.smear(DIMS, U, 0.06, -0.25, 4))
    assert p_stout > p0 and p_oi > p0
