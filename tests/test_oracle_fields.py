"""Pins for the oracle's field-level definitions: the synthetic generator,
plaquette, gauge transforms, the functional R, SU(3) exponential and
re-unitarisation.  Each is pinned by a closed form, an invariant or a library
routine, never by re-running the oracle's own formula."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H

DIMS = (4, 4, 4, 4)


def test_pure_gauge_field_plaquette_is_one():
    U = synth.make_field(DIMS, 0.0, 0)
    assert abs(oracle.plaquette(DIMS, U) - 1.0) < 1e-14
    assert H.unitarity_error(U) < 1e-13


def test_plaquette_mean_matches_width_calibration():
    """Independent adjoint-invariant links: <plaq> = m(w)^4 = 0.600 at the
    calibrated width (8^4 lattice, 24576 plaquettes, statistical tolerance)."""
    dims = (8, 8, 8, 8)
    U = synth.make_field(dims, synth.W_PLAQ_06, 0)
    assert abs(oracle.plaquette(dims, U) - 0.6) < 0.006


def test_haar_second_moment():
    """E|tr g|^2 = 1 for Haar-distributed SU(3) (a textbook moment)."""
    g = synth.random_gauge((16, 16, 16, 16), 3)
    t = np.trace(g, axis1=1, axis2=2)
    assert abs(np.mean(np.abs(t) ** 2) - 1.0) < 0.03
    assert abs(np.mean(t)) < 0.02
    assert H.unitarity_error(g) < 1e-13


def test_plaquette_abelian_closed_form():
    """Diagonal links diag(e^{i a}, e^{i b}, e^{-i(a+b)}): each plaquette is
    the diagonal matrix of summed phases, so <plaq> is a mean of cosines of
    phase sums (computed from angles, not matrices)."""
    rng = np.random.default_rng(2)
    dims = (4, 2, 6, 4)
    V = int(np.prod(dims))
    ph = rng.uniform(-np.pi, np.pi, size=(V, 4, 2))
    phases = np.concatenate([ph, -ph.sum(-1, keepdims=True)], -1)  # (V,4,3)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    for k in range(3):
        U[:, :, k, k] = np.exp(1j * phases[..., k])
    P = phases.reshape(dims[3], dims[2], dims[1], dims[0], 4, 3)
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            th = P[..., mu, :] + H.fwd(P[..., nu, :], mu) - H.fwd(P[..., mu, :], nu) - P[..., nu, :]
            tot += np.cos(th).sum() / 3
    assert abs(oracle.plaquette(dims, U) - tot / (6 * V)) < 1e-14


def test_plaquette_gauge_invariant():
    U = synth.make_field(DIMS, 0.5, 1)
    G = synth.random_gauge(DIMS, 2)
    assert abs(oracle.plaquette(DIMS, oracle.apply_gauge(DIMS, U, G)) - oracle.plaquette(DIMS, U)) < 1e-13


def test_apply_gauge_identity_and_composition():
    U = synth.make_field(DIMS, 0.5, 1)
    G1 = synth.random_gauge(DIMS, 2)
    G2 = synth.random_gauge(DIMS, 4)
    np.testing.assert_array_equal(oracle.apply_gauge(DIMS, U, synth.identity_gauge(DIMS)), U)
    two = oracle.apply_gauge(DIMS, oracle.apply_gauge(DIMS, U, G1), G2)
    one = oracle.apply_gauge(DIMS, U, oracle.compose_gauge(G2, G1))
    assert np.abs(two - one).max() < 1e-13
    # explicit single-link check of U_mu(x) -> G(x) U G(x+mu)^dag
    x, mu = 37, 2
    xp = H.fwd(np.arange(256).reshape(4, 4, 4, 4), mu).ravel()[x]
    np.testing.assert_allclose(oracle.apply_gauge(DIMS, U, G1)[x, mu], G1[x] @ U[x, mu] @ G1[xp].conj().T,
                               atol=1e-14)


def test_R_closed_forms():
    """R = 9 * 4V for identity links and for any center-valued links;
    R is invariant under center gauge transforms (|tr| unchanged)."""
    V = 256
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    assert oracle.functional_R(DIMS, U) == 9.0 * 4 * V
    Z = oracle.apply_gauge(DIMS, U, synth.random_center_gauge(DIMS, 5))
    assert abs(oracle.functional_R(DIMS, Z) - 9.0 * 4 * V) < 1e-10
    W = synth.make_field(DIMS, 0.5, 1)
    Wz = oracle.apply_gauge(DIMS, W, synth.random_center_gauge(DIMS, 6))
    assert abs(oracle.functional_R(DIMS, Wz) - oracle.functional_R(DIMS, W)) < 1e-10
    assert oracle.functional_V(DIMS, U) == 1.0


def test_expm_against_scipy():
    rng = np.random.default_rng(0)
    for scale in (1e-6, 0.1, 1.0, 5.0):
        for _ in range(20):
            M = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
            Hm = (M + M.conj().T) / 2
            X = 1j * scale * Hm
            assert np.abs(oracle.expm(X) - scipy.linalg.expm(X)).max() < 1e-13 * max(1, scale)
            Y = scale * M  # general (non-normal) matrix
            E = scipy.linalg.expm(Y)
            assert np.abs(oracle.expm(Y) - E).max() < 1e-12 * max(1.0, np.abs(E).max())


def test_reunitarise_projects_to_su3():
    rng = np.random.default_rng(1)
    g = H.haar(rng, 100)
    np.testing.assert_allclose(oracle.reunitarise(g), g, atol=1e-14)  # fixed point on SU(3)
    noisy = g + 1e-6 * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    r = oracle.reunitarise(noisy)
    assert H.unitarity_error(r) < 1e-14
    assert np.abs(r - g).max() < 1e-5
