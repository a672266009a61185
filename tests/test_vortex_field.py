"""Pins for the planted-vortex workload (synth.center_sheets /
make_vortex_field): the documented sheet geometry, the center-only field's
plaquette 1 - 3 rho / 2 and its P-vortex count through the oracle's center
projection and vortex counter (against an independent count of the planted
fluxes), and the calibration of the noise width to a mean plaquette of 0.6
at 20^3 x 40 with 48 sheet pairs (3.1 % pierced plaquettes)."""
import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import synth

AXIS = (3, 2, 1, 0)


def flux(dims, k):
    """Center flux (mod 3) of every plaquette (mu < nu), shape (6, t, z, y, x)."""
    nx, ny, nz, nt = dims
    kg = k.reshape(nt, nz, ny, nx, 4).astype(np.int64)
    out = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            out.append((kg[..., mu] + np.roll(kg[..., nu], -1, axis=AXIS[mu]) - np.roll(kg[..., mu], -1, axis=AXIS[nu])
                        - kg[..., nu]) % 3)
    return np.stack(out)


def test_one_pair_pierces_two_sheets_where_documented():
    dims = (4, 6, 4, 8)
    k = synth.center_sheets(dims, 1, 7)
    f = flux(dims, k)
    nz_planes = [p for p in range(6) if f[p].any()]
    assert len(nz_planes) == 1
    pairs = [(mu, nu) for mu in range(4) for nu in range(mu + 1, 4)]
    mu, nu = pairs[nz_planes[0]]
    V = int(np.prod(dims))
    assert (f[nz_planes[0]] != 0).sum() == 2 * V // (dims[mu] * dims[nu])
    # the fluxes are +c and -c: one sheet of each non-zero value
    vals = f[nz_planes[0]][f[nz_planes[0]] != 0]
    assert set(vals.tolist()) == {1, 2} and (vals == 1).sum() == (vals == 2).sum()
    # each sheet fills every value of the two other coordinates
    other = [d for d in range(4) if d not in (mu, nu)]
    F = f[nz_planes[0]]
    cnt = (F != 0).sum(axis=tuple(AXIS[d] for d in other))
    assert set(np.unique(cnt).tolist()) <= {0, dims[other[0]] * dims[other[1]]}


@pytest.mark.parametrize("npairs", [1, 5, 20])
def test_center_field_plaquette_and_vortices(npairs):
    dims = (4, 4, 6, 8)
    U, k = synth.make_vortex_field(dims, 0.0, 3, npairs, gauge=False)
    f = flux(dims, k)
    V = int(np.prod(dims))
    pierced = int((f != 0).sum())
    assert pierced > 0
    rho = pierced / (6 * V)
    # each pierced plaquette is a center element with Re z = -1/2, the rest 1
    assert abs(oracle.plaquette(dims, U) - (1 - 1.5 * rho)) < 1e-14
    m = oracle.center_project(dims, U)
    expect = np.where(k == 0, 0, np.where(k == 1, 1, -1))
    assert np.array_equal(m, expect)
    n, _ = oracle.vortex_count(dims, m)
    assert n == pierced
    # a random gauge rotation leaves the plaquette and (after projection of the
    # gauge-free field) the count unchanged
    Ug, _ = synth.make_vortex_field(dims, 0.0, 3, npairs, gauge=True)
    assert abs(oracle.plaquette(dims, Ug) - oracle.plaquette(dims, U)) < 1e-13


def test_workload_calibration_20x40():
    dims = (20, 20, 20, 40)
    k = synth.center_sheets(dims, synth.VORTEX_PAIRS_20x40, 0)
    pierced = int((flux(dims, k) != 0).sum())
    V = int(np.prod(dims))
    assert 0.025 < pierced / (6 * V) < 0.035
    w = synth.width_for_plaquette(0.6, pierced / (6 * V), nsamples=100_000)
    assert abs(w - synth.W_VORTEX_06) < 2e-3
    U, _ = synth.make_vortex_field(dims, synth.W_VORTEX_06, 0, synth.VORTEX_PAIRS_20x40)
    assert abs(oracle.plaquette(dims, U) - 0.6) < 2e-3
