"""GPU parity for the center decomposition and the Wilson loops (Sec. III.A)
against the oracle, through the C ABI: vortex removal and the vortex-only
field bit-exact in FP64 (same literals, unfused products on both sides),
Wilson loops within summation-order rounding (1e-12 relative in FP64), at
small sizes with ragged blocks and at the 20^3 x 40 workload size."""
import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcg():
    from paper_0807_0264_gb300 import mcg as m

    return m


def pack(mcg, U, dims, prec=0):
    return mcg.mcg_pack_links(torch.from_numpy(np.ascontiguousarray(U)).to("cuda").unsqueeze(0), dims, prec)


def unpack(mcg, Ud, dims):
    return mcg.mcg_unpack_links(Ud, dims)[0].cpu().numpy()


def sectors(mcg, Z, dims):
    return mcg.mcg_unpack_center(Z, dims)[0].cpu().numpy()


@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (6, 4, 2, 6)])
def test_vortex_remove_bit_exact(mcg, dims):
    U = synth.make_field(dims, 0.9, 11)
    Ud = pack(mcg, U, dims)
    Z, _ = mcg.mcg_center_project(Ud, dims)
    m = sectors(mcg, Z, dims)
    assert (m == oracle.center_project(dims, U)).all()
    assert (m != 0).any()
    Ur, Zl = mcg.mcg_vortex_remove(Ud, Z, dims)
    assert np.array_equal(unpack(mcg, Ur, dims), oracle.vortex_remove(dims, U, m))
    assert np.array_equal(unpack(mcg, Zl, dims), oracle.center_links(dims, m))
    # in place: U_removed = U
    r = mcg.library().mcg_vortex_remove(mcg._ptr(Ud), mcg._ptr(Z), mcg._ptr(Ud), None,
                                        mcg.lattice(dims, 1, mcg.F64), None)
    assert r == 0
    assert np.array_equal(unpack(mcg, Ud, dims), oracle.vortex_remove(dims, U, m))
    # the removed field projects to the trivial sector
    Z2, counts = mcg.mcg_center_project(Ud, dims)
    assert (sectors(mcg, Z2, dims) == 0).all() and counts[0][0] == 0


def test_vortex_remove_fp32_close(mcg):
    dims = (4, 4, 4, 6)
    U = synth.make_field(dims, 0.9, 12)
    U32 = pack(mcg, U, dims, 1)
    Z, _ = mcg.mcg_center_project(U32, dims)
    m = sectors(mcg, Z, dims)
    Ur, _ = mcg.mcg_vortex_remove(U32, Z, dims, center=False)
    assert np.abs(unpack(mcg, Ur, dims) - oracle.vortex_remove(dims, U, m)).max() < 3e-7


def test_vortex_remove_full_size(mcg):
    dims = (20, 20, 20, 40)
    U = synth.make_field(dims, synth.W_PLAQ_06, 0)
    Ud = pack(mcg, U, dims)
    Z, _ = mcg.mcg_center_project(Ud, dims)
    m = sectors(mcg, Z, dims)
    Ur, Zl = mcg.mcg_vortex_remove(Ud, Z, dims)
    assert np.array_equal(unpack(mcg, Ur, dims), oracle.vortex_remove(dims, U, m))
    assert np.array_equal(unpack(mcg, Zl, dims), oracle.center_links(dims, m))


@pytest.mark.parametrize("dims,R,T", [((4, 4, 4, 6), 3, 5), ((6, 4, 2, 6), 2, 6), ((2, 2, 2, 2), 2, 2)])
def test_wilson_loops_match_oracle(mcg, dims, R, T):
    U = synth.make_field(dims, 0.5, 13)
    W = mcg.mcg_wilson_loops(pack(mcg, U, dims), dims, R, T)[0]
    ref = oracle.wilson_loops(dims, U, R, T)
    assert np.abs(W - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_wilson_loops_fp32_and_center_field(mcg):
    dims = (4, 4, 4, 6)
    U = synth.make_field(dims, 0.5, 14)
    ref = oracle.wilson_loops(dims, U, 3, 4)
    W32 = mcg.mcg_wilson_loops(pack(mcg, U, dims, 1), dims, 3, 4)[0]
    assert np.abs(W32 - ref).max() < 2e-6
    # vortex-only field of a rough field: exact rational loop averages
    Ud = pack(mcg, synth.make_field(dims, 1.2, 15), dims)
    Z, _ = mcg.mcg_center_project(Ud, dims)
    _, Zl = mcg.mcg_vortex_remove(Ud, Z, dims, removed=False)
    Wz = mcg.mcg_wilson_loops(Zl, dims, 3, 4)[0]
    refz = oracle.wilson_loops(dims, oracle.center_links(dims, sectors(mcg, Z, dims)), 3, 4)
    assert np.abs(Wz - refz).max() < 1e-14


def test_wilson_loops_full_size(mcg):
    dims = (20, 20, 20, 40)
    U = synth.make_field(dims, synth.W_PLAQ_06, 0)
    W = mcg.mcg_wilson_loops(pack(mcg, U, dims), dims, 2, 2)[0]
    ref = oracle.wilson_loops(dims, U, 2, 2)
    assert np.abs(W - ref).max() < 1e-12


def test_wilson_loops_bad_args(mcg):
    dims = (4, 4, 4, 6)
    Ud = pack(mcg, synth.make_field(dims, 0.5, 16), dims)
    for R, T in ((0, 1), (5, 1), (1, 7)):
        with pytest.raises(mcg.MCGError):
            mcg.mcg_wilson_loops(Ud, dims, R, T)


OFFAXIS = [(1, 1, 0), (2, 1, 0), (1, 1, 1), (2, 0, 0), (-1, 2, 1)]


@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (6, 4, 4, 4)])
def test_wilson_offaxis_match_oracle(mcg, dims):
    U = synth.make_field(dims, 0.5, 17)
    Ud = pack(mcg, U, dims)
    W = mcg.mcg_wilson_loops_offaxis(Ud, dims, OFFAXIS, 3)[0]
    ref = oracle.wilson_loops_offaxis(dims, U, OFFAXIS, 3)
    assert np.abs(W - ref).max() < 1e-12
    # on-axis vectors reproduce the on-axis routine
    Won = mcg.mcg_wilson_loops(Ud, dims, 2, 3)[0]
    Wv = mcg.mcg_wilson_loops_offaxis(Ud, dims, [(1, 0, 0), (0, 2, 0)], 3)[0]
    assert np.abs(Won - Wv).max() < 1e-13
    W32 = mcg.mcg_wilson_loops_offaxis(pack(mcg, U, dims, 1), dims, OFFAXIS, 3)[0]
    assert np.abs(W32 - ref).max() < 2e-6


def test_wilson_offaxis_full_size(mcg):
    dims = (20, 20, 20, 40)
    U = synth.make_field(dims, synth.W_PLAQ_06, 0)
    W = mcg.mcg_wilson_loops_offaxis(pack(mcg, U, dims), dims, [(1, 1, 0)], 2)[0]
    ref = oracle.wilson_loops_offaxis(dims, U, [(1, 1, 0)], 2)
    assert np.abs(W - ref).max() < 1e-12


def test_wilson_offaxis_bad_args(mcg):
    dims = (4, 4, 4, 6)
    Ud = pack(mcg, synth.make_field(dims, 0.5, 18), dims)
    for vecs, T in (([(0, 0, 0)], 1), ([(4, 0, 0)], 1), ([(1, 1, 0)], 7), ([(1, 1, 0)], 0)):
        with pytest.raises(mcg.MCGError):
            mcg.mcg_wilson_loops_offaxis(Ud, dims, vecs, T)
