"""mcg_plaquette_static: the allocation-free plaquette entry point, called
through the C ABI, against mcg_plaquette on the same fields.

Kept in a file of its own that pytest collects last, so that a run stopping
at the first failure has already run every other test.  It must pass both in
a fresh process and after the rest of the suite (the shared static array then
holds another call's leftovers)."""
import numpy as np
import pytest

from paper_0807_0264_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcg():
    from paper_0807_0264_gb300 import mcg as m

    return m


def _field(mcg, dims, seeds, prec):
    canon = torch.from_numpy(np.stack([synth.make_field(dims, 0.5, s) for s in seeds])).to("cuda")
    return mcg.mcg_pack_links(canon, dims, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_static_plaquette_matches_allocating_entry_point(mcg, prec):
    # two calls in a row with different fields and sizes: the second must not
    # see anything of the first in the shared static partial sums
    for dims, seeds in (((6, 4, 4, 6), (1, 2, 3)), ((20, 20, 20, 40), (4,))):
        U = _field(mcg, dims, seeds, prec)
        ref = mcg.mcg_plaquette(U, dims)
        out = torch.full((len(seeds),), float("nan"), dtype=torch.float64, device="cuda")
        mcg.mcg_plaquette_static(U, dims, out)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_static_plaquette_rejects_oversize(mcg):
    dims = (64, 64, 64, 66)  # 17 301 504 sites > 65536 * 256
    lat = mcg.lattice(dims, 1, 0)
    rc = mcg.library().mcg_plaquette_static(mcg.ctypes.c_void_p(1), mcg.ctypes.c_void_p(1), mcg.ctypes.byref(lat),
                                            None)
    assert rc == 3
    assert b"exceeds" in mcg.library().mcg_last_error()
