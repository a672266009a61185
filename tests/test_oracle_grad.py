"""Pins for the oracle's differentiation pieces (the training pattern that
differentiates the method; not in the paper): the Frechet derivative of exp
against scipy's expm_frechet, the staple paths against the forward staple sum,
and the reverse-mode smearing derivative against central finite differences
of the MCG functional of the smeared field."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H

DIMS = (4, 4, 4, 4)


def test_expm_frechet_matches_scipy():
    rng = np.random.default_rng(0)
    for scale in (1e-3, 0.3, 1.0, 3.0):
        for _ in range(10):
            M = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
            X = 1j * scale * (M + M.conj().T) / 2
            A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
            _, L = scipy.linalg.expm_frechet(X, A)
            assert np.abs(oracle.expm_frechet(X, A) - L).max() < 1e-13 * max(1, scale)


@pytest.mark.parametrize("eps", [1.0, -0.25])
def test_staple_paths_reproduce_staple_sum(eps):
    U = synth.make_field(DIMS, 0.6, 3)
    cp, cr = (5 - 2 * eps) / 3, -(1 - eps) / 12
    for x, mu in ((0, 0), (37, 1), (200, 3), (255, 2)):
        a = oracle.staple_sum(DIMS, U, x, mu, cp, cr)
        b = oracle.staple_sum(DIMS, U, x, mu, cp, cr, from_paths=True)
        assert np.abs(a - b).max() < 1e-13


def _loss(dims, U, rho, eps, n):
    return oracle.functional_R(dims, oracle.smear(dims, U, rho, eps, n))


@pytest.mark.parametrize("eps,rho,n", [(1.0, 0.1, 1), (1.0, 0.1, 2), (-0.25, 0.06, 1), (-0.25, 0.06, 2)])
def test_smear_backward_matches_finite_differences(eps, rho, n):
    """L(U) = R(smear_n(U)); for U_mu(x) -> exp(i h T_a) U_mu(x) the derivative
    is Re tr(G^dag i T_a U_mu(x)) with G the backward's matrix gradient."""
    U = synth.make_field(DIMS, 0.5, 7)
    S = oracle.smear(DIMS, U, rho, eps, n)
    G = oracle.smear_backward(DIMS, U, oracle.functional_matrix_grad(DIMS, S), rho, eps, n)
    T = oracle.generators()
    rng = np.random.default_rng(1)
    h = 1e-5
    for _ in range(8):
        x, mu, a = int(rng.integers(256)), int(rng.integers(4)), int(rng.integers(8))
        vals = []
        for s in (+1, -1):
            Up = U.copy()
            Up[x, mu] = scipy.linalg.expm(1j * s * h * T[a]) @ U[x, mu]
            vals.append(_loss(DIMS, Up, rho, eps, n))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = np.real(np.trace(G[x, mu].conj().T @ (1j * T[a] @ U[x, mu])))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (x, mu, a, fd, an)


def test_functional_matrix_grad_finite_differences():
    U = synth.make_field(DIMS, 0.5, 2)
    G = oracle.functional_matrix_grad(DIMS, U)
    rng = np.random.default_rng(3)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    h = 1e-6
    fd = (oracle.functional_R(DIMS, U + h * dU) - oracle.functional_R(DIMS, U - h * dU)) / (2 * h)
    an = np.sum(np.real(np.conj(G) * dU))
    assert abs(fd - an) < 1e-6 * abs(an)
