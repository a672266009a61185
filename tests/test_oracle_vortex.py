"""Pins for the oracle's vortex removal, vortex-only field and Wilson loops
(Sec. III.A): Z U' = U, the removed field projects to the trivial sector, the
vortex-only field's plaquette is fixed by its P-vortex density, and the
Wilson loops reduce to the space-time plaquette at R = T = 1, are gauge
invariant, equal 1 on a pure gauge, match the closed form of a constant
abelian flux and, on center fields, the integer flux through the loop."""
import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H

DIMS = (4, 4, 4, 6)


def _fixed_field(seed):
    U = synth.make_field(DIMS, 0.6, seed)
    return oracle.fix(DIMS, U, None, tol=1e-9, max_sweeps=60)["U"]


def test_vortex_removal_inverts_and_projects_trivially():
    U = _fixed_field(1)
    m = oracle.center_project(DIMS, U)
    Ur = oracle.vortex_remove(DIMS, U, m)
    # Z U' = U with Z = exp(2 pi i m / 3) (numpy's own exponential)
    z = np.exp(2j * np.pi * m.astype(float) / 3.0)[..., None, None]
    assert np.abs(z * Ur.reshape(U.shape) - U).max() < 1e-15 * 4
    # the removed field's traces all sit in the trivial sector
    assert (oracle.center_project(DIMS, Ur) == 0).all()
    # det Z^dag = 1, so U' stays in SU(3)
    d = np.linalg.det(Ur.reshape(-1, 3, 3))
    assert np.abs(d - 1).max() < 1e-13


def test_vortex_only_field_sectors_and_plaquette():
    rng = np.random.default_rng(2)
    V = int(np.prod(DIMS))
    m = rng.integers(-1, 2, size=(V, 4)).astype(np.int8)
    Z = oracle.center_links(DIMS, m)
    # the center field projects back onto its sectors
    assert (oracle.center_project(DIMS, Z) == m).all()
    # each plaquette of Z is exp(2 pi i n / 3): 1 if n = 0 mod 3, else -1/2;
    # so <plaq> = 1 - (3/2) * (P-vortex plaquettes) / (6V)
    nv, _ = oracle.vortex_count(DIMS, m)
    assert nv > 0
    assert abs(oracle.plaquette(DIMS, Z) - (1.0 - 1.5 * nv / (6.0 * V))) < 1e-14


def _spacetime_plaquette(dims, U):
    """Independent numpy: mean (1/3) Re tr of the plaquettes in the (i, t)
    planes, i = x, y, z."""
    G = H.as_grid(dims, U)
    vals = []
    for i in range(3):
        Ui, Ut = G[..., i, :, :], G[..., 3, :, :]
        P = H.mm(Ui, H.fwd(Ut, i), H.dag(H.fwd(Ui, 3)), H.dag(Ut))
        vals.append(H.retr3(P).mean())
    return float(np.mean(vals))


def test_wilson_1x1_is_the_spacetime_plaquette():
    U = synth.make_field(DIMS, 0.5, 3)
    W = oracle.wilson_loops(DIMS, U, 1, 1)
    assert abs(W[0, 0] - _spacetime_plaquette(DIMS, U)) < 1e-14


def test_wilson_gauge_invariant_and_pure_gauge():
    U = synth.make_field(DIMS, 0.5, 4)
    Om = synth.random_gauge(DIMS, 5)
    W0 = oracle.wilson_loops(DIMS, U, 3, 4)
    W1 = oracle.wilson_loops(DIMS, oracle.apply_gauge(DIMS, U, Om), 3, 4)
    assert np.abs(W0 - W1).max() < 1e-13
    P = synth.make_field(DIMS, 0.0, 6)  # pure gauge
    assert np.abs(oracle.wilson_loops(DIMS, P, 3, 4) - 1.0).max() < 1e-13


def test_wilson_constant_abelian_flux_closed_form():
    """U_i(x) = diag(e^{i F_k t}) on the spatial links, U_t = 1, F_k = 2 pi n_k / N_t:
    every (i, t) plaquette carries the same flux, so
    W(R, T) = (1/3) sum_k cos(F_k R T)."""
    nt = DIMS[3]
    F = 2 * np.pi * np.array([1, 2, -3]) / nt
    V = int(np.prod(DIMS))
    t = (np.arange(V) // (DIMS[0] * DIMS[1] * DIMS[2])).astype(float)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    for mu in range(3):
        for k in range(3):
            U[:, mu, k, k] = np.exp(1j * F[k] * t)
    U[:, 3] = np.eye(3)
    W = oracle.wilson_loops(DIMS, U, 3, 5)
    for R in range(1, 4):
        for T in range(1, 6):
            assert abs(W[R - 1, T - 1] - np.cos(F * R * T).sum() / 3.0) < 1e-14


def test_wilson_on_center_field_counts_flux():
    """On a center field every loop is exp(2 pi i n / 3) with n the signed sum
    of the sectors around it: W = mean over loops of (1 if n = 0 mod 3 else -1/2),
    counted here with integers."""
    rng = np.random.default_rng(7)
    V = int(np.prod(DIMS))
    m = rng.integers(-1, 2, size=(V, 4)).astype(np.int8)
    Z = oracle.center_links(DIMS, m)
    W = oracle.wilson_loops(DIMS, Z, 2, 3)
    nx, ny, nz, nt = DIMS
    g = m.reshape(nt, nz, ny, nx, 4).astype(np.int64)
    ax = (3, 2, 1, 0)
    for R in (1, 2):
        for T in (1, 2, 3):
            vals = []
            for i in range(3):
                n = np.zeros(g.shape[:4], np.int64)
                for k in range(R):  # bottom: +i links from x
                    n += np.roll(g[..., i], -k, axis=ax[i])
                for k in range(T):  # right: +t links from x + R i
                    n += np.roll(np.roll(g[..., 3], -R, axis=ax[i]), -k, axis=ax[3])
                for k in range(R):  # top, reversed: -(+i links from x + T t)
                    n -= np.roll(np.roll(g[..., i], -T, axis=ax[3]), -k, axis=ax[i])
                for k in range(T):  # left, reversed
                    n -= np.roll(g[..., 3], -k, axis=ax[3])
                vals.append(np.where(n % 3 == 0, 1.0, -0.5).mean())
            assert abs(W[R - 1, T - 1] - np.mean(vals)) < 1e-14


OFFAXIS = [(1, 1, 0), (2, 1, 0), (1, 1, 1), (2, 0, 0)]


def test_offaxis_reduces_to_onaxis():
    """An on-axis vector averaged over its 6 cubic images (+-x, +-y, +-z)
    equals the on-axis loops along +x, +y, +z (a -i loop is a +i loop
    translated and traversed backwards: same real trace)."""
    U = synth.make_field(DIMS, 0.5, 21)
    W = oracle.wilson_loops(DIMS, U, 3, 4)
    Wo = oracle.wilson_loops_offaxis(DIMS, U, [(1, 0, 0), (2, 0, 0), (3, 0, 0)], 4)
    assert np.abs(W - Wo).max() < 1e-14


def test_offaxis_closed_loops_gauge_invariant_and_pure_gauge():
    U = synth.make_field(DIMS, 0.5, 22)
    Om = synth.random_gauge(DIMS, 23)
    W0 = oracle.wilson_loops_offaxis(DIMS, U, OFFAXIS, 3)
    W1 = oracle.wilson_loops_offaxis(DIMS, oracle.apply_gauge(DIMS, U, Om), OFFAXIS, 3)
    assert np.abs(W0 - W1).max() < 1e-13
    P = synth.make_field(DIMS, 0.0, 24)
    assert np.abs(oracle.wilson_loops_offaxis(DIMS, P, OFFAXIS, 3) - 1.0).max() < 1e-13


def test_offaxis_constant_abelian_flux_closed_form():
    """Spatial links diag(e^{i F_k t}), U_t = 1: the spatial path product is
    diag(e^{i F_k t s}) with s the signed sum of the vector's components, so a
    loop is diag(e^{-i F_k T s}); W is the mean of (1/3) sum_k cos(F_k T s)
    over the distinct images of the vector (enumerated here with itertools)."""
    import itertools

    nt = DIMS[3]
    F = 2 * np.pi * np.array([1, 2, -3]) / nt
    V = int(np.prod(DIMS))
    t = (np.arange(V) // (DIMS[0] * DIMS[1] * DIMS[2])).astype(float)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    for mu in range(3):
        for k in range(3):
            U[:, mu, k, k] = np.exp(1j * F[k] * t)
    U[:, 3] = np.eye(3)
    W = oracle.wilson_loops_offaxis(DIMS, U, OFFAXIS, 4)
    for v, r in enumerate(OFFAXIS):
        imgs = {tuple(sg * c for sg, c in zip(signs, perm))
                for perm in itertools.permutations(r) for signs in itertools.product((1, -1), repeat=3)}
        for T in range(1, 5):
            ref = np.mean([np.cos(F * T * sum(im)).sum() / 3.0 for im in imgs])
            assert abs(W[v, T - 1] - ref) < 1e-14
