"""Pins for the oracle's simulated annealing of the gauge transform (the
Gribov-copy search variant named in Sec. III.B): its Philox4x64-10 generator
against numpy's, the infinite-temperature limit (every proposal accepted, so
Omega is the product of the drawn SU(2) elements, built here from Pauli
matrices), the first half-sweep on the unit field (all eight links of a site
are Omega(x) or its adjoint, so each decision has a closed form), and the
zero-temperature limit (R never decreases)."""
import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H

DIMS = (4, 4, 4, 4)
PQ = ((0, 1, 2), (0, 2, 1), (1, 2, 0))
SIGMA = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)
MASK64 = (1 << 64) - 1


def np_philox(ctr, key):
    """numpy's Philox4x64-10 block for counter `ctr` (numpy advances its
    counter before each block, so start it one below)."""
    c = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    start = np.array([(c >> (64 * i)) & MASK64 for i in range(4)], dtype=np.uint64)
    g = np.random.Philox(counter=start, key=np.array(key, dtype=np.uint64))
    return g.random_raw(4)


def proposal(x, sweep, s, h, nhit, eps, seed, field):
    """The SU(2) proposal of hit h of subgroup s at lexicographic site x, as
    a 3x3 embedding, and the acceptance uniform."""
    w = [int(v) for v in np_philox((x, sweep, s * nhit + h, field), (seed, 0))]
    u = [(v >> 11) * 2.0**-53 for v in w]
    v = [eps * (2.0 * u[k] - 1.0) for k in range(3)]
    a0 = np.sqrt(1.0 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]))
    g2 = a0 * np.eye(2) + 1j * np.einsum("k,kij->ij", np.array(v), SIGMA)
    p, q, r = PQ[s]
    G = np.zeros((3, 3), np.complex128)
    G[r, r] = 1.0
    G[np.ix_([p, q], [p, q])] = g2
    return G, u[3]


def parity(dims, x):
    nx, ny, nz, _ = dims
    c = (x % nx, (x // nx) % ny, (x // (nx * ny)) % nz, x // (nx * ny * nz))
    return sum(c) & 1


@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (7, 0)),
                                     ((123456789, 42, 17, 3), (0xDEADBEEF12345678, 0)),
                                     ((MASK64, MASK64, MASK64, MASK64), (MASK64, MASK64)),
                                     ((5, 0, 1 << 40, 9), (3, 1 << 63))])
def test_philox_matches_numpy(ctr, key):
    assert (oracle.philox4x64(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
            == np_philox(ctr, key)).all()


def test_infinite_temperature_accepts_every_draw_and_composes_them():
    nsweeps, nhit, eps, seed, field = 2, 2, 0.45, 987654321, 2
    U0 = synth.make_field(DIMS, 0.6, 11)
    G0 = synth.identity_gauge(DIMS)
    U, G, acc = oracle.anneal(DIMS, U0, G0, [1e300] * nsweeps, nhit, eps, seed, first_sweep=3, field=field)
    V = int(np.prod(DIMS))
    assert acc == V * 3 * nhit * nsweeps
    Om = np.empty((V, 3, 3), np.complex128)
    for x in range(V):
        M = np.eye(3, dtype=np.complex128)
        for k in range(nsweeps):
            for s in range(3):
                for h in range(nhit):
                    M = proposal(x, 3 + k, s, h, nhit, eps, seed, field)[0] @ M
        Om[x] = M
    assert np.abs(G.reshape(V, 3, 3) - Om).max() < 1e-13
    og = Om.reshape(DIMS[3], DIMS[2], DIMS[1], DIMS[0], 3, 3)
    ug = H.as_grid(DIMS, U0)
    for mu in range(4):
        expect = H.mm(og, ug[..., mu, :, :], H.dag(H.fwd(og, mu)))
        assert np.abs(H.as_grid(DIMS, U)[..., mu, :, :] - expect).max() < 1e-13


@pytest.mark.parametrize("T", [10.0, 2.5])
def test_unit_field_first_half_sweep_decisions_in_closed_form(T):
    # On the unit field the even half-sweep sees, at each even x, forward links
    # Omega(x) and backward links Omega(x)^dag, so the site functional is
    # 8 |tr Omega(x)|^2 and each Metropolis decision is fixed by it.
    nhit, eps, seed, field, sweep = 1, 0.5, 2024, 3, 5
    V = int(np.prod(DIMS))
    U0 = np.zeros((V, 4, 3, 3), np.complex128)
    U0[..., 0, 0] = U0[..., 1, 1] = U0[..., 2, 2] = 1.0
    U, G, acc = oracle.anneal_halfsweep(DIMS, U0, synth.identity_gauge(DIMS), 0, T, sweep, nhit, eps, seed, field)
    Om = np.tile(np.eye(3, dtype=np.complex128), (V, 1, 1))
    expect_acc = 0
    for x in range(V):
        if parity(DIMS, x):
            continue
        M = np.eye(3, dtype=np.complex128)
        for s in range(3):
            Gp, u = proposal(x, sweep, s, 0, nhit, eps, seed, field)
            dF = 8.0 * (abs(np.trace(Gp @ M)) ** 2 - abs(np.trace(M)) ** 2)
            if dF >= 0 or u < np.exp(dF / T):
                M = Gp @ M
                expect_acc += 1
        Om[x] = M
    assert 0 < expect_acc < 3 * V // 2
    assert acc == expect_acc
    assert np.abs(G.reshape(V, 3, 3) - Om).max() < 1e-14
    og = Om.reshape(DIMS[3], DIMS[2], DIMS[1], DIMS[0], 3, 3)
    for mu in range(4):
        assert np.abs(H.as_grid(DIMS, U)[..., mu, :, :] - H.mm(og, H.dag(H.fwd(og, mu)))).max() < 1e-14


def test_zero_temperature_never_lowers_R():
    U = synth.make_field(DIMS, 0.6, 5)
    G = synth.identity_gauge(DIMS)
    R = oracle.functional_R(DIMS, U)
    total = 0
    for k in range(3):
        for par in (0, 1):
            U, G, acc = oracle.anneal_halfsweep(DIMS, U, G, par, 1e-300, k, 3, 0.2, 77)
            R_new = oracle.functional_R(DIMS, U)
            assert R_new >= R - 1e-10 * R
            R, total = R_new, total + acc
    assert 0 < total < int(np.prod(DIMS)) * 3 * 3 * 3


def test_first_sweep_continues_the_stream_and_the_field_stays_on_the_orbit():
    U0 = synth.make_field(DIMS, 0.6, 8)
    G0 = synth.identity_gauge(DIMS)
    T = [4.0, 1.0, 0.3]
    U, G, acc = oracle.anneal(DIMS, U0, G0, T, 2, 0.3, 99)
    U1, G1, a1 = oracle.anneal(DIMS, U0, G0, T[:1], 2, 0.3, 99)
    U2, G2, a2 = oracle.anneal(DIMS, U1, G1, T[1:], 2, 0.3, 99, first_sweep=1)
    assert acc == a1 + a2
    assert np.abs(U2 - U).max() < 1e-12 and np.abs(G2 - G).max() < 1e-12
    # gauge invariance: the annealed field is U0 transformed by the returned Omega
    assert np.abs(oracle.apply_gauge(DIMS, U0, G) - U).max() < 1e-12
    assert abs(oracle.plaquette(DIMS, U) - oracle.plaquette(DIMS, U0)) < 1e-13


def test_zero_sweeps_only_reunitarise():
    U0 = synth.make_field(DIMS, 0.6, 13)
    G0 = synth.random_gauge(DIMS, 14)
    U, G, acc = oracle.anneal(DIMS, U0, G0, [], 2, 0.3, 1)
    assert acc == 0
    assert np.abs(U - oracle.reunitarise(U0)).max() == 0 and np.abs(G - oracle.reunitarise(G0)).max() == 0
    assert np.abs(U - U0).max() < 1e-14
