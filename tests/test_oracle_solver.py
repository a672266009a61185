"""Pins for the oracle's local SU(2)-subgroup maximisation (the trust-region
subproblem max a^T A a + 2 b.a on |a| = 1 that each subgroup step of the MCG
site update solves).  Pinned by brute force on the sphere, by the textbook
global-optimality conditions of the trust-region subproblem, and by the b = 0
special case, which is LAPACK's top eigenvector."""
import numpy as np
import pytest
import scipy.optimize

import oracle


def F(A, b, a):
    return a @ A @ a + 2 * b @ a


def random_problem(rng, kind):
    if kind == "small_b":  # b small against the eigenvalue gaps: root far from alpha_max + max|beta|
        A, b = random_problem(rng, "psd")
        return A, 0.05 * b
    if kind == "psd":  # the shape the MCG update produces: sum of Re(w^* w^T)
        w = rng.standard_normal((8, 4)) + 1j * rng.standard_normal((8, 4))
        c = rng.standard_normal(8) + 1j * rng.standard_normal(8)
        A = np.real(np.einsum("lk,lj->kj", w.conj(), w))
        b = np.real(np.einsum("l,lk->k", c.conj(), w))
    else:
        M = rng.standard_normal((4, 4))
        A = M + M.T
        b = rng.standard_normal(4)
    return A, b


def sphere_samples(rng, n):
    s = rng.standard_normal((n, 4))
    return s / np.linalg.norm(s, axis=1, keepdims=True)


@pytest.mark.parametrize("kind", ["psd", "sym", "small_b"])
def test_beats_random_sphere_samples(kind):
    rng = np.random.default_rng(11)
    for _ in range(20):
        A, b = random_problem(rng, kind)
        a, hard = oracle.trs_solve(A, b)
        assert not hard
        assert abs(np.linalg.norm(a) - 1) < 1e-14
        S = sphere_samples(rng, 100_000)
        vals = np.einsum("ni,ij,nj->n", S, A, S) + 2 * S @ b
        assert F(A, b, a) >= vals.max() - 1e-12 * (1 + abs(vals.max()))


def test_matches_dense_grid_and_polish():
    """Hyperspherical grid (48 x 24 x 24) then local polish from the best grid
    points: the polished optimum equals the oracle's value and point."""
    rng = np.random.default_rng(5)
    t1 = np.linspace(0, np.pi, 24)
    t2 = np.linspace(0, np.pi, 24)
    t3 = np.linspace(0, 2 * np.pi, 48, endpoint=False)
    T1, T2, T3 = np.meshgrid(t1, t2, t3, indexing="ij")
    G = np.stack([np.cos(T1), np.sin(T1) * np.cos(T2), np.sin(T1) * np.sin(T2) * np.cos(T3),
                  np.sin(T1) * np.sin(T2) * np.sin(T3)], -1).reshape(-1, 4)
    for k in range(8):
        A, b = random_problem(rng, "psd" if k % 2 else "small_b")
        a, _ = oracle.trs_solve(A, b)
        vals = np.einsum("ni,ij,nj->n", G, A, G) + 2 * G @ b
        best = None
        for i in np.argsort(vals)[-5:]:
            res = scipy.optimize.minimize(lambda y: -F(A, b, y / np.linalg.norm(y)), G[i], method="BFGS",
                                          options=dict(gtol=1e-12, maxiter=2000))
            y = res.x / np.linalg.norm(res.x)
            if best is None or F(A, b, y) > F(A, b, best):
                best = y
        assert abs(F(A, b, best) - F(A, b, a)) < 1e-9 * abs(F(A, b, a))
        assert np.linalg.norm(best - a) < 1e-5


@pytest.mark.parametrize("kind", ["psd", "sym", "small_b"])
def test_global_optimality_conditions(kind):
    """(mu I - A) a = b with mu >= lambda_max(A) and |a| = 1 is necessary and
    sufficient for the global maximum of the trust-region subproblem."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        A, b = random_problem(rng, kind)
        a, _ = oracle.trs_solve(A, b)
        mu = a @ A @ a + a @ b
        scale = max(np.abs(A).max(), np.abs(b).max())
        assert np.linalg.norm((mu * np.eye(4) - A) @ a - b) < 1e-11 * scale
        assert mu >= np.linalg.eigvalsh(A)[-1] - 1e-12 * scale


def test_b_zero_is_top_eigenvector():
    rng = np.random.default_rng(3)
    for _ in range(50):
        A, _ = random_problem(rng, "psd")
        a, hard = oracle.trs_solve(A, np.zeros(4))
        assert hard
        e, v = np.linalg.eigh(A)
        assert abs(abs(a @ v[:, -1]) - 1) < 1e-12
        # sign convention: largest-magnitude component of the eigenvector positive
        k = np.argmax(np.abs(v[:, -1]))
        assert a[k] > 0


def test_constructed_hard_case():
    """b orthogonal to the top eigenvector with small remaining solution:
    maximum value alpha_max + sum_i beta_i^2/(alpha_max - alpha_i) is reached."""
    rng = np.random.default_rng(9)
    Qm, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    al = np.array([5.0, 1.0, 0.0, -1.0])
    A = Qm @ np.diag(al) @ Qm.T
    beta = np.array([0.0, 0.5, 0.3, -0.2])
    b = Qm @ beta
    a, hard = oracle.trs_solve(A, b)
    assert hard
    expected = al[0] + np.sum(beta[1:] ** 2 / (al[0] - al[1:]))
    assert abs(F(A, b, a) - expected) < 1e-12
    S = sphere_samples(rng, 100_000)
    assert F(A, b, a) >= (np.einsum("ni,ij,nj->n", S, A, S) + 2 * S @ b).max() - 1e-12


def test_identity_links_keep_identity():
    """Eight identity links, subgroup (0,1): w = (2,0,0,0), c = 1 for each, so
    A = diag(32,0,0,0), b = (16,0,0,0) and the optimum is a = (1,0,0,0)."""
    A = np.diag([32.0, 0, 0, 0])
    b = np.array([16.0, 0, 0, 0])
    a, hard = oracle.trs_solve(A, b)
    assert not hard
    np.testing.assert_allclose(a, [1, 0, 0, 0], atol=1e-15)


def test_zero_weight_on_the_top_eigenvector():
    """b orthogonal to the top eigenvector (its weight exactly 0) with the
    remaining weights too large for the hard case: the multiplier lies strictly
    above lambda_max and the maximiser follows from the other terms alone.
    A = diag(3, 1, 0, 0), b = (0, 3, 0, 0): 9 / (mu - 1)^2 = 1 gives mu = 4 and
    a = (0, 1, 0, 0) with F = 1 + 6 = 7 (F(e0) = 3)."""
    A = np.diag([3.0, 1.0, 0.0, 0.0])
    b = np.array([0.0, 3.0, 0.0, 0.0])
    a, hard = oracle.trs_solve(A, b)
    assert np.all(np.isfinite(a)) and not hard
    assert np.abs(a - np.array([0.0, 1.0, 0.0, 0.0])).max() < 1e-12
    rng = np.random.default_rng(5)
    X = rng.standard_normal((100000, 4))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    F = np.einsum("ni,ij,nj->n", X, A, X) + 2 * X @ b
    assert a @ A @ a + 2 * b @ a >= F.max() - 1e-12


def near_hard_problem(rng, inside):
    """A = V diag(lam) V^T, b = V beta with a small weight on the top
    eigenvector (|beta_top| = 10^U(-12, -2)) and the other weights scaled so
    that p = sum_i beta_i / (lam_top - lam_i) v_i has |p| in (0.3, 0.95)
    (inside: the multiplier sits just above lam_top) or in (1.05, 2)."""
    q, r = np.linalg.qr(rng.standard_normal((4, 4)))
    V = q * np.sign(np.diag(r))
    lam = np.sort(rng.uniform(0.0, 12.0, 4))
    beta = np.zeros(4)
    beta[:3] = rng.standard_normal(3)
    target = rng.uniform(0.3, 0.95) if inside else rng.uniform(1.05, 2.0)
    beta[:3] *= target / np.linalg.norm(beta[:3] / (lam[3] - lam[:3]))
    beta[3] = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-12.0, -2.0)
    A = (V * lam) @ V.T
    return 0.5 * (A + A.T), V @ beta


@pytest.mark.parametrize("inside", [True, False])
def test_global_optimality_near_the_hard_case(inside):
    """The same conditions on problems near the hard case, where the
    multiplier lies within |beta_top| / sqrt(1 - |p|^2) of lambda_max (inside)
    or the top weight is negligible (outside): a secular iteration that stops
    on a step small against mu itself, rather than against mu - lambda_max,
    fails the residual here."""
    rng = np.random.default_rng(23)
    for _ in range(2000):
        A, b = near_hard_problem(rng, inside)
        a, _ = oracle.trs_solve(A, b)
        mu = a @ A @ a + a @ b
        scale = max(np.abs(A).max(), np.abs(b).max())
        assert abs(np.linalg.norm(a) - 1) < 1e-14
        assert np.linalg.norm((mu * np.eye(4) - A) @ a - b) < 1e-10 * scale
        assert mu >= np.linalg.eigvalsh(A)[-1] - 1e-12 * scale
