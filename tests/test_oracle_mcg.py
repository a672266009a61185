"""Pins for the oracle's MCG relaxation (Sec. II.A) and preconditioning
pipeline (Sec. II.B): pure gauge reaches V_U = 1, R rises monotonically, the
converged field is a local maximum (2^4 brute force over all sites and all
eight generator directions), the field stays on its gauge orbit, and each
subgroup step is a maximum of the local functional (sampled SU(2))."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H


def test_pure_gauge_fixes_to_one():
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.0, 0)
    r = oracle.fix(dims, U, tol=1e-10, max_sweeps=2000)
    assert r["converged"]
    V = r["R_hist"][-1] / (36 * 256)
    assert V > 1 - 1e-10
    # every fixed link is then a center element times (1 - tiny)
    m = oracle.center_project(dims, r["U"])
    n, _ = oracle.vortex_count(dims, m)
    assert n == 0


def test_R_monotone_per_halfsweep():
    dims = (4, 4, 2, 6)
    U = synth.make_field(dims, 0.5, 3)
    G = synth.identity_gauge(dims)
    R = oracle.functional_R(dims, U)
    for k in range(30):
        U, G, _ = oracle.halfsweep(dims, U, G, k % 2)
        Rn = oracle.functional_R(dims, U)
        assert Rn >= R - 1e-13 * R
        R = Rn


def test_fixed_field_on_gauge_orbit():
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 0)
    r = oracle.fix(dims, U, tol=1e-10, max_sweeps=500)
    assert abs(oracle.plaquette(dims, r["U"]) - oracle.plaquette(dims, U)) < 1e-13
    assert np.abs(oracle.apply_gauge(dims, U, r["G"]) - r["U"]).max() < 1e-12


def _local_R(F_links, B_links):
    return sum(abs(np.trace(F)) ** 2 for F in F_links) + sum(abs(np.trace(B)) ** 2 for B in B_links)


def test_subgroup_step_is_local_maximum():
    """After a half-sweep, every updated site is at the maximum of its local
    functional over the last subgroup (1,2): no sampled SU(2) element of that
    subgroup raises it."""
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.7, 8)
    U1, _, _ = oracle.halfsweep(dims, U, synth.identity_gauge(dims), 0)
    Ug = H.as_grid(dims, U1)
    rng = np.random.default_rng(0)
    s = rng.standard_normal((20000, 4))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    for (t, z, y, x) in [(0, 0, 0, 0), (1, 2, 3, 0), (3, 3, 2, 0)]:
        F = [Ug[t, z, y, x, mu] for mu in range(4)]
        B = [H.fwd(Ug[..., mu, :, :], mu, -1)[t, z, y, x] for mu in range(4)]
        base = _local_R(F, B)
        best = 0.0
        for a in s[:2000]:
            G = np.eye(3, dtype=complex)
            G[1, 1], G[1, 2] = a[0] + 1j * a[3], a[2] + 1j * a[1]
            G[2, 1], G[2, 2] = -a[2] + 1j * a[1], a[0] - 1j * a[3]
            val = _local_R([G @ f for f in F], [b @ G.conj().T for b in B])
            best = max(best, val)
        assert best <= base + 1e-10 * base


@pytest.mark.parametrize("seed", [0, 1])
def test_2x4_converged_is_local_maximum(seed):
    """2^4 lattice (x+mu = x-mu: every site sees both of a link's ends
    through periodic wrap).  After convergence no single-site rotation
    exp(+-i eps T_a) along any of the 8 generators raises R, and the
    Lie-algebra gradient vanishes."""
    dims = (2, 2, 2, 2)
    U = synth.make_field(dims, 0.5, seed)
    r = oracle.fix(dims, U, tol=1e-15, max_sweeps=20000, reunit_every=50)
    Uf = r["U"]
    R0 = oracle.functional_R(dims, Uf)
    T = oracle.generators()
    grad = oracle.grad_R(dims, Uf)
    assert np.abs(grad).max() < 1e-5 * R0 / 64
    for x in range(16):
        for a in range(8):
            for eps in (1e-3, -1e-3, 1e-2, -1e-2):
                G = synth.identity_gauge(dims)
                G[x] = scipy.linalg.expm(1j * eps * T[a])
                assert oracle.functional_R(dims, oracle.apply_gauge(dims, Uf, G)) <= R0 + 1e-12 * R0


def test_precondition_pipeline_stays_on_orbit():
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 2)
    out = oracle.precondition_and_fix(dims, U, rho=0.1, eps=1.0, nsmear=4, tol=1e-10, max_sweeps=500)
    Uf = out["fixed"]["U"]
    assert abs(oracle.plaquette(dims, Uf) - oracle.plaquette(dims, U)) < 1e-12
    assert np.abs(oracle.apply_gauge(dims, U, out["G_total"]) - Uf).max() < 1e-11
    Vs = out["smeared"]["R_hist"][-1] / (36 * 256)
    Vf = out["fixed"]["R_hist"][-1] / (36 * 256)
    assert Vs > Vf  # the smeared field is smoother, so its maximum is higher
    assert 0 <= out["vortex_density"] < 1


def test_grad_R_matches_finite_differences():
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 4)
    T = oracle.generators()
    np.testing.assert_allclose(np.trace(T @ T, axis1=1, axis2=2), 0.5, atol=1e-15)
    grad = oracle.grad_R(dims, U)
    h = 1e-5
    for x in (0, 77, 255):
        for a in range(8):
            vals = []
            for s in (+1, -1):
                G = synth.identity_gauge(dims)
                G[x] = scipy.linalg.expm(1j * s * h * T[a])
                vals.append(oracle.functional_R(dims, oracle.apply_gauge(dims, U, G)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grad[x, a]) < 1e-6 * (1 + abs(grad[x, a]))
