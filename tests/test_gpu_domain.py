"""Domain decomposition of one lattice along t on the GPU: the ranks' slabs
(each with its ghost layers) swept by mcg_halfsweep_slab and exchanging
boundary t-links through the decomposition's driver, all ranks in one
process phase by phase on cuda:0 (no kernel waits on another), reproduce the
single-domain GPU relaxation bit for bit in every link and in Omega (the same
kernel does the same per-site arithmetic), R to rounding, and the oracle to
the FP64 parity bar."""
import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import domain, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NEVER = -1e300


@pytest.mark.parametrize("dims,world", [((4, 4, 4, 8), 2), ((4, 4, 2, 8), 4), ((6, 4, 4, 4), 1)])
def test_device_slabs_match_single_domain(dims, world):
    from paper_0807_0264_gb300 import mcg

    U = synth.make_field(dims, 0.5, 3)
    G = synth.random_gauge(dims, 4)
    doms = [domain.SlabDomain(dims, r, world) for r in range(world)]
    bks = [domain.DeviceSlab(d, *d.scatter(U, G)) for d in doms]
    res = domain.run_ranks_lockstep([domain.Sweeper(d, b) for d, b in zip(doms, bks)], NEVER, 7, reunit_every=3)
    Uo = np.concatenate([d.owned(*b.local_arrays())[0] for d, b in zip(doms, bks)])
    Go = np.concatenate([d.owned(*b.local_arrays())[1] for d, b in zip(doms, bks)])
    Ud = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), dims)
    Gd = mcg.mcg_pack_gauge(torch.from_numpy(G).unsqueeze(0).cuda(), dims)
    single = mcg.mcg_fix(Ud, Gd, dims, mcg.Params(tol=NEVER, max_sweeps=7, check_every=7, reunit_every=3),
                         history=True)
    assert np.array_equal(Uo, mcg.mcg_unpack_links(Ud, dims)[0].cpu().numpy())
    assert np.array_equal(Go, mcg.mcg_unpack_gauge(Gd, dims)[0].cpu().numpy())
    np.testing.assert_allclose(res["R_hist"], single["R_hist"][0], rtol=1e-13, atol=0)
    ref = oracle.fix(dims, U, G, tol=NEVER, max_sweeps=7, reunit_every=3)
    assert np.abs(Uo - ref["U"]).max() < 1e-11 and np.abs(Go - ref["G"]).max() < 1e-11


def test_device_slabs_stop_at_the_single_domain_sweep():
    from paper_0807_0264_gb300 import mcg

    dims = (4, 4, 4, 8)
    U = synth.make_field(dims, 0.5, 0)
    G = synth.identity_gauge(dims)
    doms = [domain.SlabDomain(dims, r, 2) for r in range(2)]
    bks = [domain.DeviceSlab(d, *d.scatter(U, G)) for d in doms]
    res = domain.run_ranks_lockstep([domain.Sweeper(d, b) for d, b in zip(doms, bks)], 1e-10, 2000)
    ref = oracle.fix(dims, U, tol=1e-10, max_sweeps=2000)
    assert res["converged"] and res["sweeps"] == ref["sweeps"]
