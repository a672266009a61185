"""Pins for center projection and P-vortex identification (Sec. II.A).

Center sector: the oracle's exact-comparison rule is checked against the two
definitions the paper gives, the nearest phase 2 pi m / 3 to arg tr U and the
center element closest to U on the group manifold (largest Re tr(Z^dag U)).
Vortex counting: closed-form counts for hand-placed configurations (fixtures
in tests/golden/), Z3 gauge invariance, and an independent count through
complex center phases."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import synth
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OMEGA = np.exp(2j * np.pi / 3)


def _links_from_traces(traces):
    """Diagonal SU(3) links are awkward to aim at a given trace; instead store
    the trace on the diagonal of an (unphysical) matrix: the projection reads
    only (U00 + U11) + U22."""
    U = np.zeros((len(traces), 3, 3), np.complex128)
    U[:, 0, 0] = traces
    return U


def test_center_elements_project_to_themselves():
    V = 16
    dims = (2, 2, 2, 2)
    for k, m in ((0, 0), (1, 1), (2, -1)):
        U = np.zeros((V, 4, 3, 3), np.complex128)
        U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = OMEGA ** k
        assert (oracle.center_project(dims, U) == m).all()


def test_sector_golden_table():
    with open(os.path.join(GOLDEN, "center_sectors.json")) as f:
        g = json.load(f)
    tr = np.array([c[0] + 1j * c[1] for c in g["cases"]])
    want = np.array([c[2] for c in g["cases"]], np.int8)
    n = len(tr)
    pad = (-n) % 4
    U = np.zeros((n + pad, 3, 3), np.complex128)
    U[:n, 0, 0] = tr
    m = oracle.center_project((1, 1, 1, (n + pad) // 4), U.reshape(-1, 4, 3, 3)).ravel()[:n]
    np.testing.assert_array_equal(m, want)


def test_sector_is_nearest_phase_and_closest_center_element():
    rng = np.random.default_rng(0)
    g = H.haar(rng, 40000)
    U = g.reshape(-1, 4, 3, 3)
    dims = (1, 1, 1, U.shape[0])
    m = oracle.center_project(dims, U).ravel()
    t = np.trace(g, axis1=1, axis2=2)
    phi = np.angle(t)
    cand = np.array([0, 1, -1])
    dist = np.abs(np.angle(np.exp(1j * (phi[:, None] - 2 * np.pi * cand[None, :] / 3))))
    np.testing.assert_array_equal(m, cand[np.argmin(dist, axis=1)])
    # closest center element on the manifold: max_m Re tr(Z_m^dag U)
    score = np.real(np.conj(OMEGA ** cand[None, :]) * t[:, None])
    np.testing.assert_array_equal(m, cand[np.argmax(score, axis=1)])


def _vortex_count_by_phases(dims, m):
    """Independent count: multiply the center phases around each plaquette
    as complex numbers; pierced when the product is not 1."""
    nx, ny, nz, nt = dims
    z = (OMEGA ** m.astype(np.int64)).reshape(nt, nz, ny, nx, 4)
    per = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = z[..., mu] * H.fwd(z[..., nu], mu) * np.conj(H.fwd(z[..., mu], nu)) * np.conj(z[..., nu])
            per.append(int(np.sum(np.abs(P - 1) > 0.5)))
    return sum(per), per


def test_single_link_pierces_six_plaquettes():
    dims = (4, 4, 4, 4)
    m = np.zeros((256, 4), np.int8)
    m[100, 2] = 1
    tot, per = oracle.vortex_count(dims, m)
    assert tot == 6
    planes = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    for p, (a, b) in enumerate(planes):
        assert per[p] == (2 if 2 in (a, b) else 0)


def test_golden_vortex_configurations():
    with open(os.path.join(GOLDEN, "vortex_configs.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        dims = tuple(c["dims"])
        nx, ny, nz, nt = dims
        V = nx * ny * nz * nt
        m = np.zeros((nt, nz, ny, nx, 4), np.int8)
        for (x, y, z, t, mu, val) in c["links"]:
            m[t, z, y, x, mu] = val
        for rule in c.get("rules", []):
            sel = np.ones((nt, nz, ny, nx), bool)
            grid = np.indices((nt, nz, ny, nx))
            for axis_name, val in rule["where"].items():
                ax = {"x": 3, "y": 2, "z": 1, "t": 0}[axis_name]
                sel &= grid[ax] == val
            m[..., rule["mu"]][sel] = rule["value"]
        tot, per = oracle.vortex_count(dims, m.reshape(V, 4))
        assert tot == c["expected_total"], c["name"]
        assert list(per) == c["expected_per_plane"], c["name"]


def test_vortex_count_random_and_z3_gauge_invariant():
    dims = (4, 6, 4, 2)
    V = int(np.prod(dims))
    rng = np.random.default_rng(4)
    m = rng.integers(-1, 2, size=(V, 4)).astype(np.int8)
    tot, per = oracle.vortex_count(dims, m)
    tot2, per2 = _vortex_count_by_phases(dims, m)
    assert tot == tot2 and list(per) == per2
    # Z3 gauge transform m_mu(x) -> m_mu(x) + k(x) - k(x+mu)  (mod 3, to {-1,0,1})
    k = rng.integers(0, 3, size=V).reshape(dims[3], dims[2], dims[1], dims[0])
    mg = m.reshape(dims[3], dims[2], dims[1], dims[0], 4).astype(int).copy()
    for mu in range(4):
        mg[..., mu] = mg[..., mu] + k - H.fwd(k, mu)
    mg = ((mg + 1) % 3) - 1
    tg, pg = oracle.vortex_count(dims, mg.reshape(V, 4).astype(np.int8))
    assert tg == tot and list(pg) == list(per)


def test_center_gauge_keeps_vortex_count_of_field():
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.8, 7)
    n0, _ = oracle.vortex_count(dims, oracle.center_project(dims, U))
    Uz = oracle.apply_gauge(dims, U, synth.random_center_gauge(dims, 1))
    n1, _ = oracle.vortex_count(dims, oracle.center_project(dims, Uz))
    assert n0 == n1
