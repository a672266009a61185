"""Pins for the oracle's over-relaxed subgroup step.

Over-relaxation is not part of the paper's relaxation (Sec. II.A); the
mixed-precision schedule uses it for its early sweeps.  Its definition here:
with G* the element of the SU(2) subgroup (p, q) that maximises the site's
local functional, the step applies

    G_omega = ((1 - omega) 1 + omega G*) / sqrt(det((1 - omega) 1 + omega G*))

(the 2x2 block; a real combination of 1 and an SU(2) matrix is a positive
multiple of an SU(2) matrix).  omega = 1 is the plain relaxation.

The test side rebuilds each site update without the oracle's coefficient
formulas or its SU(2) parametrisation: the local functional
F(G) = sum_l |tr(G F_l)|^2 + |tr(B_l G^dag)|^2 is evaluated with explicit 3x3
matrices, its quadratic form in the quaternion parameters of
a0 1 + i(a1 s1 + a2 s2 + a3 s3) (Pauli matrices) is recovered by polarisation,
and the maximiser on the unit sphere follows from numpy's eigh and a bracketed
root of the secular equation (the textbook optimality conditions of the
trust-region subproblem: (mu - A) a = b, mu >= lambda_max(A)).  A slip in the
oracle's branch (a weight on the wrong components, a sign, a missing
renormalisation, G for G^dag on the backward links) moves the links by far
more than the 1e-11 bar.  Further pins: fixed points are shared with the plain
relaxation, and an over-relaxed fix ends at a local maximum of R on the same
gauge orbit."""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import oracle
from paper_0807_0264_gb300 import synth

PQ = ((0, 1), (0, 2), (1, 2))
S1 = np.array([[0, 1], [1, 0]], complex)
S2 = np.array([[0, -1j], [1j, 0]], complex)
S3 = np.array([[1, 0], [0, -1]], complex)


def su2(a):
    return a[0] * np.eye(2) + 1j * (a[1] * S1 + a[2] * S2 + a[3] * S3)


def embed(g, p, q):
    G = np.eye(3, dtype=complex)
    G[np.ix_((p, q), (p, q))] = g
    return G


def local_F(G, F, B):
    return sum(abs(np.trace(G @ f)) ** 2 for f in F) + sum(abs(np.trace(b @ G.conj().T)) ** 2 for b in B)


def quadratic_form(F, B, p, q):
    """A, b with F(a) = a.A.a + 2 b.a + c for G = embed(su2(a)), by polarisation
    (su2 is linear in a, so F is a quadratic polynomial on all of R^4)."""
    f = lambda a: local_F(embed(su2(np.asarray(a, float)), p, q), F, B)
    E = np.eye(4)
    c = f(np.zeros(4))
    A = np.zeros((4, 4))
    b = np.zeros(4)
    for i in range(4):
        fp, fm = f(E[i]), f(-E[i])
        A[i, i] = 0.5 * (fp + fm) - c
        b[i] = 0.25 * (fp - fm)
    for i in range(4):
        for j in range(i + 1, 4):
            A[i, j] = A[j, i] = 0.5 * (f(E[i] + E[j]) - c - A[i, i] - A[j, j] - 2 * b[i] - 2 * b[j])
    return A, b


def sphere_max(A, b):
    """argmax of a.A.a + 2 b.a on |a| = 1 from the optimality conditions."""
    al, V = np.linalg.eigh(A)
    beta = V.T @ b
    top = al[-1]
    phi = lambda mu: np.sum(beta ** 2 / (mu - al) ** 2) - 1.0
    lo, hi = top + abs(beta[-1]), top + np.linalg.norm(b)
    assert abs(beta[-1]) > 1e-8 * np.linalg.norm(b), "hard case: not used by these pins"
    mu = lo if phi(lo) <= 0 else scipy.optimize.brentq(phi, lo, hi, xtol=1e-300, rtol=4 * np.finfo(float).eps,
                                                        maxiter=500)
    a = V @ (beta / (mu - al))
    return a / np.linalg.norm(a)


def site_update(F, B, Om, omega):
    """The over-relaxed site update on copies of the site's 8 links and Omega."""
    F = [f.copy() for f in F]
    B = [b.copy() for b in B]
    Om = Om.copy()
    for p, q in PQ:
        A, bv = quadratic_form(F, B, p, q)
        gs = su2(sphere_max(A, bv))
        M = (1.0 - omega) * np.eye(2) + omega * gs
        g = M / np.sqrt(np.linalg.det(M).real)
        G = embed(g, p, q)
        F = [G @ f for f in F]
        B = [b @ G.conj().T for b in B]
        Om = G @ Om
    return F, B, Om


def index(dims, x, y, z, t):
    nx, ny, nz, _ = dims
    return x + nx * (y + ny * (z + nz * t))


def shifted(dims, c, mu, d):
    c = list(c)
    c[mu] = (c[mu] + d) % dims[mu]
    return index(dims, *c)


@pytest.mark.parametrize("omega", [1.0, 1.5, 1.85])
def test_site_update_matches_independent_construction(omega):
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 5)
    Om0 = synth.random_gauge(dims, 9)
    U1, Om1, hard = oracle.halfsweep(dims, U, Om0, 0, omega)
    assert hard == 0
    sites = [(0, 0, 0, 0), (1, 1, 0, 0), (2, 3, 1, 0), (3, 3, 3, 3), (1, 0, 2, 3)]
    for c in sites:
        assert sum(c) % 2 == 0
        x = index(dims, *c)
        back = [shifted(dims, c, mu, -1) for mu in range(4)]
        F = [U[x, mu] for mu in range(4)]
        B = [U[back[mu], mu] for mu in range(4)]
        Fn, Bn, On = site_update(F, B, Om0[x], omega)
        for mu in range(4):
            assert np.abs(U1[x, mu] - Fn[mu]).max() < 1e-11, (c, mu)
            assert np.abs(U1[back[mu], mu] - Bn[mu]).max() < 1e-11, (c, mu)
        assert np.abs(Om1[x] - On).max() < 1e-11


def test_over_relaxation_moves_further_along_the_same_direction():
    """For omega > 1 the applied element turns further from the identity than
    the maximiser, about the same axis: the first subgroup step has a
    quaternion vector part parallel to the maximiser's and a rotation angle
    that grows with omega (omega = 1: the maximiser itself); the oracle's
    transform at the site equals the three steps of the definition."""
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.6, 2)
    I3 = synth.identity_gauge(dims)
    x = index(dims, 0, 0, 0, 0)
    back = [shifted(dims, (0, 0, 0, 0), mu, -1) for mu in range(4)]
    F = [U[x, mu] for mu in range(4)]
    B = [U[back[mu], mu] for mu in range(4)]
    A, bv = quadratic_form(F, B, 0, 1)
    astar = sphere_max(A, bv)
    angles = []
    for omega in (1.0, 1.3, 1.6, 1.9):
        _, Om1, _ = oracle.halfsweep(dims, U, I3, 0, omega)
        _, _, On = site_update(F, B, np.eye(3, dtype=complex), omega)
        assert np.abs(On - Om1[x]).max() < 1e-11
        # the first subgroup step of the definition
        M = (1.0 - omega) * np.eye(2) + omega * su2(astar)
        g = M / np.sqrt(np.linalg.det(M).real)
        a0 = g.trace().real / 2
        vec = np.array([np.trace(g @ s).imag / 2 for s in (S1, S2, S3)])
        assert abs(a0 ** 2 + vec @ vec - 1) < 1e-13
        assert vec @ astar[1:] > 0
        assert np.linalg.norm(np.cross(vec, astar[1:])) < 1e-12 * np.linalg.norm(vec)
        angles.append(np.arctan2(np.linalg.norm(vec), a0))
    assert all(a2 > a1 for a1, a2 in zip(angles, angles[1:]))
    assert abs(angles[0] - np.arctan2(np.linalg.norm(astar[1:]), astar[0])) < 1e-12


@pytest.mark.parametrize("omega", [1.5, 1.85])
def test_fixed_points_are_shared(omega):
    """At a maximum of the plain relaxation every maximiser is the identity,
    and so is every over-relaxed element: an over-relaxed half-sweep leaves the
    converged 2^4 field in place."""
    dims = (2, 2, 2, 2)
    U = synth.make_field(dims, 0.5, 0)
    r = oracle.fix(dims, U, tol=-1.0, max_sweeps=2000)  # 2000 sweeps: converged to rounding
    U1, G1, _ = oracle.halfsweep(dims, r["U"], r["G"], 0, omega)
    U2, G2, _ = oracle.halfsweep(dims, U1, G1, 1, omega)
    assert np.abs(U2 - r["U"]).max() < 1e-13
    assert abs(oracle.functional_R(dims, U2) - oracle.functional_R(dims, r["U"])) < 1e-12 * 64 * 9


@pytest.mark.parametrize("seed", [0, 1])
def test_over_relaxed_fix_ends_at_a_plain_maximum(seed):
    """An over-relaxed fix (omega = 1.85) of a 2^4 field converges to a local
    maximum of R on the field's gauge orbit: no single-site rotation along any
    of the 8 generators raises R, plain half-sweeps leave it in place, and the
    plaquette and U = U0^Omega hold."""
    dims = (2, 2, 2, 2)
    U = synth.make_field(dims, 0.5, seed)
    r = oracle.fix(dims, U, tol=-1.0, max_sweeps=4000, omega=1.85)
    Uf = r["U"]
    assert abs(oracle.plaquette(dims, Uf) - oracle.plaquette(dims, U)) < 1e-13
    assert np.abs(oracle.apply_gauge(dims, U, r["G"]) - Uf).max() < 1e-11
    R0 = oracle.functional_R(dims, Uf)
    T = oracle.generators()
    for x in range(16):
        for a in range(8):
            for eps in (1e-3, -1e-3):
                G = synth.identity_gauge(dims)
                G[x] = scipy.linalg.expm(1j * eps * T[a])
                assert oracle.functional_R(dims, oracle.apply_gauge(dims, Uf, G)) <= R0 + 1e-12 * R0
    U1, G1, _ = oracle.halfsweep(dims, Uf, r["G"], 0)
    U2, _, _ = oracle.halfsweep(dims, U1, G1, 1)
    assert np.abs(U2 - Uf).max() < 1e-13


@pytest.mark.parametrize("seed", [0, 1])
def test_over_relaxed_fix_reaches_the_plain_maximum_on_4x4(seed):
    """On these 4^4 fields (w = 0.5, a single dominant maximum) the
    over-relaxed and the plain relaxation, both run to rounding level, end at
    the same maximum up to a Z3 gauge transform (which leaves R unchanged):
    equal V_U, equal |tr U_mu(x)| on every link, equal P-vortex counts."""
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, seed)
    ro = oracle.fix(dims, U, tol=-1.0, max_sweeps=3000, omega=1.85)
    rp = oracle.fix(dims, U, tol=-1.0, max_sweeps=3000, omega=1.0)
    assert abs(oracle.functional_V(dims, ro["U"]) - oracle.functional_V(dims, rp["U"])) < 1e-13
    tro = np.abs(np.trace(ro["U"], axis1=-2, axis2=-1))
    trp = np.abs(np.trace(rp["U"], axis1=-2, axis2=-1))
    assert np.abs(tro - trp).max() < 1e-9
    no, _ = oracle.vortex_count(dims, oracle.center_project(dims, ro["U"]))
    npl, _ = oracle.vortex_count(dims, oracle.center_project(dims, rp["U"]))
    assert no == npl
