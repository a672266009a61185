"""Domain decomposition of one lattice along t (paper_0807_0264_gb300.domain),
on CPU: the oracle's slab half-sweep as each rank's compute, driven by the
decomposition's exchange protocol, reproduces the single-domain oracle
relaxation (Sec. II.A) bit for bit in every link and in Omega, with R equal to
rounding (the ranks' partial sums add in another order) and the same stop
sweep.  Covered in one process (all ranks phase by phase) and with two gloo
ranks in two processes."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import domain, synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NEVER = -1e300


class OracleSlab:
    """Slab backend on the oracle: the local arrays of one rank."""

    def __init__(self, dom, U, G, omega=1.0):
        self.dom = dom
        self.U, self.G = dom.scatter(U, G)
        self.omega = omega

    def halfsweep(self, parity):
        d = self.dom
        oracle.halfsweep_slab(d.local_dims, self.U, self.G, parity, 1, d.L + 1, d.t_offset, self.omega)

    def get_face(self, t_local, parity):
        return self.U[self.dom.face_sites(t_local, parity), 3].copy()

    def set_face(self, t_local, parity, a):
        self.U[self.dom.face_sites(t_local, parity), 3] = a

    def owned_R(self):
        Uo, _ = self.dom.owned(self.U, self.G)
        return float(np.sum(np.abs(np.trace(Uo, axis1=-2, axis2=-1)) ** 2))

    def reunitarise(self):
        s = slice(self.dom.layer, (self.dom.L + 1) * self.dom.layer)
        self.U[s] = oracle.reunitarise(self.U[s])
        self.G[s] = oracle.reunitarise(self.G[s])


def gather(doms, backends):
    Us, Gs = zip(*[d.owned(b.U, b.G) for d, b in zip(doms, backends)])
    return np.concatenate(Us), np.concatenate(Gs)


def test_partition_geometry():
    dom = domain.SlabDomain((4, 6, 2, 8), 1, 2)
    assert dom.L == 4 and dom.local_dims == (4, 6, 2, 6) and dom.t0 == 4
    for P in (0, 1):
        g, t = dom.ghost_sites(P), dom.last_layer_sites(P)
        assert len(g) == len(t) == 4 * 6 * 2 // 2
        assert np.array_equal(dom.face_sites(0, P), g) and np.array_equal(dom.face_sites(dom.L, P), t)
        # a face's sites are one contiguous in-parity range of the local array,
        # of local parity P ^ t_offset, in (x, y, z) order on both layers
        for layer in (0, dom.L):
            f = dom.face_sites(layer, P)
            x, y, z, tl = f % 4, (f // 4) % 6, (f // 24) % 2, f // 48
            assert np.all((x + y + z + tl) % 2 == dom.local_parity(P))
            assert np.array_equal(f // 2, layer * 24 + np.arange(24))
    # the ghost layer is global t0 - 1 = 3 (odd): parity of (x, y, z) flipped
    assert dom.global_parity_of_layer(0)[0] == 1 and dom.global_parity_of_layer(1)[0] == 0
    with pytest.raises(ValueError):
        domain.SlabDomain((4, 4, 4, 6), 0, 2)  # slabs of 3 layers
    with pytest.raises(ValueError):
        domain.SlabDomain((4, 4, 4, 8), 0, 3)


def test_slab_halfsweeps_cover_the_halfsweep():
    """Two complementary slab half-sweeps on the whole lattice (no ghosts)
    give the oracle's half-sweep exactly."""
    dims = (4, 4, 4, 6)
    U = synth.make_field(dims, 0.6, 1)
    G = synth.random_gauge(dims, 2)
    Ur, Gr, _ = oracle.halfsweep(dims, U, G, 1)
    Us, Gs = U.copy(), G.copy()
    oracle.halfsweep_slab(dims, Us, Gs, 1, 0, 4, 0)
    oracle.halfsweep_slab(dims, Us, Gs, 1, 4, 6, 0)
    assert np.array_equal(Us, Ur) and np.array_equal(Gs, Gr)


@pytest.mark.parametrize("dims,world", [((4, 4, 4, 8), 1), ((4, 4, 4, 8), 2), ((4, 2, 4, 8), 4),
                                        ((6, 4, 4, 4), 2)])
def test_lockstep_matches_single_domain(dims, world):
    U = synth.make_field(dims, 0.5, 3)
    G = synth.random_gauge(dims, 4)
    ref = oracle.fix(dims, U, G, tol=NEVER, max_sweeps=7, reunit_every=3)
    doms = [domain.SlabDomain(dims, r, world) for r in range(world)]
    bks = [OracleSlab(d, U, G) for d in doms]
    res = domain.run_ranks_lockstep([domain.Sweeper(d, b) for d, b in zip(doms, bks)], NEVER, 7, reunit_every=3)
    Uo, Go = gather(doms, bks)
    assert np.array_equal(Uo, ref["U"]) and np.array_equal(Go, ref["G"])
    np.testing.assert_allclose(res["R_hist"], ref["R_hist"], rtol=1e-13, atol=0)


def test_lockstep_stops_at_the_oracle_sweep():
    dims = (4, 4, 4, 8)
    U = synth.make_field(dims, 0.5, 0)
    ref = oracle.fix(dims, U, tol=1e-10, max_sweeps=2000)
    assert ref["converged"]
    G = synth.identity_gauge(dims)
    doms = [domain.SlabDomain(dims, r, 2) for r in range(2)]
    bks = [OracleSlab(d, U, G) for d in doms]
    res = domain.run_ranks_lockstep([domain.Sweeper(d, b) for d, b in zip(doms, bks)], 1e-10, 2000)
    assert res["converged"] and res["sweeps"] == ref["sweeps"]
    Uo, _ = gather(doms, bks)
    assert np.array_equal(Uo, ref["U"])


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, dims, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U = synth.make_field(dims, 0.5, 5)
    G = synth.identity_gauge(dims)
    dom = domain.SlabDomain(dims, rank, world)
    b = OracleSlab(dom, U, G)
    res = domain.run_rank(domain.Sweeper(dom, b), NEVER, 6, reunit_every=4)
    Uo, Go = dom.owned(b.U, b.G)
    out[rank] = (Uo.tobytes(), Go.tobytes(), res["R_hist"])
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_domain():
    dims = (4, 4, 4, 8)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, _free_port(), dims, out), nprocs=2, join=True)
        res = dict(out)
    U = synth.make_field(dims, 0.5, 5)
    ref = oracle.fix(dims, U, tol=NEVER, max_sweeps=6, reunit_every=4)
    Uo = np.concatenate([np.frombuffer(res[r][0], np.complex128).reshape(-1, 4, 3, 3) for r in (0, 1)])
    Go = np.concatenate([np.frombuffer(res[r][1], np.complex128).reshape(-1, 3, 3) for r in (0, 1)])
    assert np.array_equal(Uo, ref["U"]) and np.array_equal(Go, ref["G"])
    assert res[0][2] == res[1][2]  # both ranks saw the same all-reduced R
    np.testing.assert_allclose(res[0][2], ref["R_hist"], rtol=1e-13, atol=0)
