"""One lattice split into slabs along t, one slab per process: domain
decomposition of the checkerboard MCG relaxation (Sec. II.A).

Partition.  Rank r of W owns the sites with global t in [r L, (r + 1) L),
L = Nt / W, and their four forward links U_mu(x) and Omega(x).  L must be
even, so every slab starts on an even t.  The rank's local array is a
lattice of Nx x Ny x Nz x (L + 2) sites: local t = 0 is a ghost layer (global
t0 - 1), local t = 1 .. L the owned layers, local t = L + 1 a second ghost
layer that is never read (it keeps every local extent even, which the
device layout needs).  A local site at local t has global parity
(x + y + z + t + 1) mod 2, since t0 - 1 is odd.

Exchange.  The site update at x touches U_mu(x) and U_mu(x - mu).  The only
such link outside the slab is U_t(x - t) for x on the first owned layer: the
forward t-link of a site on the last layer of rank r - 1.  A half-sweep of
parity P updates the first-layer sites of parity P, whose backward t-links
start on sites of parity 1 - P.  So, per half-sweep:
  1. every rank sends the t-links of its last-layer sites of parity 1 - P to
     rank r + 1, which stores them in its ghost layer;
  2. every rank updates its sites of parity P (in parallel: same-parity sites
     share no link);
  3. every rank returns the updated ghost t-links to rank r - 1, which writes
     them back into its last layer.
Nx Ny Nz / 2 links move each way per half-sweep (FP64: 144 bytes each).  The
functional R = sum |tr U|^2 is the sum over ranks of R over the owned links:
one all-reduce per sweep; every rank then takes the same stop decision
(V_U(k) - V_U(k-1) < tol, Sec. II.A).  Re-unitarisation acts on owned links
and Omega.

The driver is independent of where the slab lives: a backend supplies the
slab half-sweep, reads and writes of one face (the t-links of one parity on
one layer), the owned R and the re-unitarisation; `run_ranks_lockstep` drives all ranks from one process
(phase by phase, no rank ever waits on another), `run_rank` drives one rank
of a torch.distributed group.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SlabDomain:
    dims: tuple
    rank: int
    world: int

    def __post_init__(self):
        nx, ny, nz, nt = self.dims
        if self.world < 1 or nt % self.world:
            raise ValueError(f"Nt = {nt} is not a multiple of the {self.world} slabs")
        L = nt // self.world
        if L % 2 or L < 2:
            raise ValueError(f"slab thickness {L} must be even and >= 2")
        if min(nx, ny, nz) < 2 or nx % 2 or ny % 2 or nz % 2:
            raise ValueError("spatial extents must be even and >= 2")
        self.L = L
        self.t0 = self.rank * L
        self.local_dims = (nx, ny, nz, L + 2)
        self.layer = nx * ny * nz
        xyz = np.arange(self.layer)
        x = xyz % nx
        y = (xyz // nx) % ny
        z = xyz // (nx * ny)
        self._xyz_parity = (x + y + z) & 1

    # local site indices (canonical order i = x + Nx (y + Ny (z + Nz t)))
    def layer_sites(self, t_local: int) -> np.ndarray:
        return t_local * self.layer + np.arange(self.layer)

    def global_parity_of_layer(self, t_local: int) -> np.ndarray:
        return (self._xyz_parity + self.t0 - 1 + t_local) & 1

    def last_layer_sites(self, parity: int) -> np.ndarray:
        """Sites of the last owned layer with global parity `parity`, in
        (x, y, z) order."""
        t = self.L
        return self.layer_sites(t)[self.global_parity_of_layer(t) == parity]

    def ghost_sites(self, parity: int) -> np.ndarray:
        """Ghost-layer sites (global t0 - 1) of global parity `parity`, in the
        same (x, y, z) order as rank r - 1's last_layer_sites(parity)."""
        return self.layer_sites(0)[self.global_parity_of_layer(0) == parity]

    def face_sites(self, t_local: int, parity: int) -> np.ndarray:
        """Sites of local layer t_local with global parity `parity`, in
        (x, y, z) order: one face of the exchange."""
        return self.layer_sites(t_local)[self.global_parity_of_layer(t_local) == parity]

    def local_parity(self, parity: int) -> int:
        """Parity, in the local array's own checkerboard, of the sites of
        global parity `parity` (the same on every layer)."""
        return parity ^ self.t_offset

    def owned_sites(self) -> np.ndarray:
        return np.arange(self.layer, (self.L + 1) * self.layer)

    @property
    def t_offset(self) -> int:
        """Local -> global parity offset: global parity = (x+y+z+t_local+1) mod 2."""
        return (self.t0 - 1) & 1

    # ---- canonical host arrays (V, 4, 3, 3) / (V, 3, 3) ---------------------
    def scatter(self, U, G):
        """The rank's local arrays from the whole lattice's canonical U, G:
        owned layers and both ghost layers filled from the periodic lattice."""
        nx, ny, nz, nt = self.dims
        Ug = U.reshape(nt, self.layer, 4, 3, 3)
        Gg = G.reshape(nt, self.layer, 3, 3)
        ts = [(self.t0 - 1 + t) % nt for t in range(self.L + 2)]
        Ul = np.ascontiguousarray(Ug[ts].reshape(-1, 4, 3, 3))
        Gl = np.ascontiguousarray(Gg[ts].reshape(-1, 3, 3))
        return Ul, Gl

    def owned(self, Ul, Gl):
        """The owned layers of local arrays, as the slab of the whole lattice."""
        s = slice(self.layer, (self.L + 1) * self.layer)
        return Ul[s], Gl[s]


class Sweeper:
    """The decomposed relaxation for one rank, phase by phase.  `backend`:
      halfsweep(parity)              update the owned sites of global parity
      get_face(t_local, parity)      t-links (mu = 3) of the sites of global
                                     parity `parity` on a local layer, in
                                     (x, y, z) order (any array type)
      set_face(t_local, parity, d)   write such a face back
      owned_R() -> float             sum |tr U|^2 over the owned links
      reunitarise()                  owned links and Omega
    """

    def __init__(self, dom: SlabDomain, backend):
        self.dom = dom
        self.b = backend

    def send_up(self, P):
        return self.b.get_face(self.dom.L, 1 - P)

    def recv_from_below(self, P, data):
        self.b.set_face(0, 1 - P, data)

    def compute(self, P):
        self.b.halfsweep(P)

    def send_down(self, P):
        return self.b.get_face(0, 1 - P)

    def recv_from_above(self, P, data):
        self.b.set_face(self.dom.L, 1 - P, data)


def _stop(R, R_prev, norm, tol):
    return (R - R_prev) * norm < tol


def run_ranks_lockstep(sweepers, tol: float, max_sweeps: int, reunit_every: int = 50):
    """All ranks of one lattice driven from one process, phase by phase (the
    exchanges are plain copies between the ranks' backends).  Returns
    dict(sweeps, converged, R_hist)."""
    W = len(sweepers)
    dims = sweepers[0].dom.dims
    norm = 1.0 / (36.0 * float(np.prod(dims)))
    R_prev = sum(s.b.owned_R() for s in sweepers)
    hist = [R_prev]
    for k in range(1, max_sweeps + 1):
        for P in (0, 1):
            up = [s.send_up(P) for s in sweepers]
            for r, s in enumerate(sweepers):
                s.recv_from_below(P, up[(r - 1) % W])
            for s in sweepers:
                s.compute(P)
            down = [s.send_down(P) for s in sweepers]
            for r, s in enumerate(sweepers):
                s.recv_from_above(P, down[(r + 1) % W])
        if reunit_every > 0 and k % reunit_every == 0:
            for s in sweepers:
                s.b.reunitarise()
        R = sum(s.b.owned_R() for s in sweepers)
        hist.append(R)
        if _stop(R, R_prev, norm, tol):
            return dict(sweeps=k, converged=True, R_hist=hist)
        R_prev = R
    return dict(sweeps=max_sweeps, converged=False, R_hist=hist)


def run_rank(sweeper: Sweeper, tol: float, max_sweeps: int, reunit_every: int = 50, group=None):
    """One rank of a torch.distributed group (rank = sweeper.dom.rank): the
    exchanges are point-to-point messages with the neighbouring slabs, the
    functional one all-reduce per sweep.  Every rank returns the same
    dict(sweeps, converged, R_hist)."""
    import torch
    import torch.distributed as dist

    dom = sweeper.dom
    W, r = dom.world, dom.rank
    up_rank, down_rank = (r + 1) % W, (r - 1) % W
    norm = 1.0 / (36.0 * float(np.prod(dom.dims)))

    # faces travel as they are when the group's backend can send them (host
    # tensors; device tensors under NCCL), else through host memory
    device_ok = W > 1 and dist.get_backend(group) == "nccl"

    def sendrecv(x, to, frm):
        host = isinstance(x, np.ndarray)
        t_send = torch.from_numpy(np.ascontiguousarray(x).view(np.float64)) if host else x.contiguous()
        if not host and t_send.is_cuda and not device_ok:
            t_send = t_send.cpu()
        t_recv = torch.empty_like(t_send)
        if W == 1:
            t_recv.copy_(t_send)
        else:
            req = dist.isend(t_send, to, group=group)
            dist.recv(t_recv, frm, group=group)
            req.wait()
        return t_recv.numpy().view(np.complex128).reshape(x.shape) if host else t_recv

    def allreduce(x):
        t = torch.tensor([x], dtype=torch.float64)
        if W > 1:
            dist.all_reduce(t, group=group)
        return float(t[0])

    R_prev = allreduce(sweeper.b.owned_R())
    hist = [R_prev]
    for k in range(1, max_sweeps + 1):
        for P in (0, 1):
            sweeper.recv_from_below(P, sendrecv(sweeper.send_up(P), up_rank, down_rank))
            sweeper.compute(P)
            sweeper.recv_from_above(P, sendrecv(sweeper.send_down(P), down_rank, up_rank))
        if reunit_every > 0 and k % reunit_every == 0:
            sweeper.b.reunitarise()
        R = allreduce(sweeper.b.owned_R())
        hist.append(R)
        if _stop(R, R_prev, norm, tol):
            return dict(sweeps=k, converged=True, R_hist=hist)
        R_prev = R
    return dict(sweeps=max_sweeps, converged=False, R_hist=hist)


class DeviceSlab:
    """Slab backend on libmcg: the rank's local arrays (FP64, even/odd layout)
    on its GPU; half-sweeps by mcg_halfsweep_slab (exact FP64 local solve),
    faces read and written on the device by mcg_slab_face (a face is a
    (9, Nx Ny Nz / 2, 2) float64 tensor on the slab's device, ready for a
    device-to-device copy or an NCCL send), R from the odd half-sweep's fused
    partial (each link has exactly one odd end, so the slabs' partials add up
    to the lattice's R)."""

    def __init__(self, dom: SlabDomain, U, G, device="cuda"):
        import torch

        from . import mcg

        self.dom, self.mcg, self.torch = dom, mcg, torch
        d = dom.local_dims
        self.U = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).to(device), d)
        self.G = mcg.mcg_pack_gauge(torch.from_numpy(G).unsqueeze(0).to(device), d)
        self.R_owned = float(np.sum(np.abs(np.trace(dom.owned(U, G)[0], axis1=-2, axis2=-1)) ** 2))
        self._dev = self.U.device

    def halfsweep(self, parity):
        d = self.dom
        r = self.mcg.mcg_halfsweep_slab(self.U, self.G, d.local_dims, d.local_parity(parity), 1, d.L + 1,
                                        want_R=(parity == 1))
        if parity == 1:
            self.R_owned = r

    def get_face(self, t_local, parity):
        d = self.dom
        buf = self.mcg.empty_face(d.local_dims, self.mcg.F64, self._dev)
        return self.mcg.mcg_slab_face(self.U, buf, d.local_dims, t_local, d.local_parity(parity), False)

    def set_face(self, t_local, parity, data):
        d = self.dom
        buf = data.to(self._dev).contiguous()
        self.mcg.mcg_slab_face(self.U, buf, d.local_dims, t_local, d.local_parity(parity), True)

    def owned_R(self):
        return self.R_owned

    def reunitarise(self):
        self.mcg.mcg_reunitarise(self.U, 0, self.dom.local_dims)
        self.mcg.mcg_reunitarise(self.G, 1, self.dom.local_dims)

    def local_arrays(self):
        d = self.dom.local_dims
        return (self.mcg.mcg_unpack_links(self.U, d)[0].cpu().numpy(),
                self.mcg.mcg_unpack_gauge(self.G, d)[0].cpu().numpy())
