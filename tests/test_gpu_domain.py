"""Domain decomposition of one lattice along t on the GPU: the ranks' slabs
(each with its ghost layers) swept by mcg_halfsweep_slab and exchanging
boundary faces on the device (mcg_slab_face) through the decomposition's driver, all ranks in one
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


@pytest.mark.parametrize("prec", ["F64", "F32"])
def test_slab_face_is_the_layer_of_t_links(prec):
    """mcg_slab_face reads exactly the t-links of one parity on one layer, in
    (x, y, z) order, and writes back only those."""
    from paper_0807_0264_gb300 import mcg

    P = getattr(mcg, prec)
    dims = (4, 6, 2, 6)
    U = synth.make_field(dims, 0.7, 11)
    Ud = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), dims, P)
    n = 4 * 6 * 2 // 2
    dom = domain.SlabDomain(dims, 0, 1)  # t0 = 0: global parity = local parity ^ 1
    for t in (0, 3, 5):
        for p in (0, 1):
            buf = mcg.mcg_slab_face(Ud, mcg.empty_face(dims, P), dims, t, p, False)
            torch.cuda.synchronize()
            got = buf.cpu().numpy()
            want = Ud[0, 3, p, :, t * n:(t + 1) * n, :].cpu().numpy()  # [entry, site, re/im]
            assert np.array_equal(got, want)
            # the same sites as the domain's face of global parity p ^ 1
            sites = dom.face_sites(t, p ^ dom.t_offset)
            ref = U[sites, 3].reshape(-1, 9).T
            tol = 0 if prec == "F64" else 1e-6
            assert np.abs(got[..., 0] + 1j * got[..., 1] - ref).max() <= tol
    # write: a face of zeros lands on exactly those entries
    V0 = Ud.clone()
    mcg.mcg_slab_face(Ud, torch.zeros_like(mcg.empty_face(dims, P)), dims, 2, 1, True)
    torch.cuda.synchronize()
    changed = (Ud != V0).any(dim=-1)[0]  # (mu, parity, entry, site)
    expect = torch.zeros_like(changed)
    expect[3, 1, :, 2 * n:3 * n] = V0[0, 3, 1, :, 2 * n:3 * n].ne(0).any(dim=-1)
    assert torch.equal(changed, expect)


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
