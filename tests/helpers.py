"""Test-side helpers: independent numpy restatements of definitions that pin
the oracle (loop sums, sector choice by brute force), plus small utilities.
Nothing here is imported by the product path or by the oracle."""
from __future__ import annotations

import numpy as np
import scipy.linalg

AXIS_OF_MU = (3, 2, 1, 0)  # canonical array (t, z, y, x, ...) -> axis of direction mu


def as_grid(dims, U):
    nx, ny, nz, nt = dims
    return U.reshape(nt, nz, ny, nx, 4, 3, 3)


def fwd(F, mu, n=1):
    """F(x + n*mu) for a per-site array on the (t, z, y, x) grid."""
    return np.roll(F, -n, axis=AXIS_OF_MU[mu])


def dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def mm(*Ms):
    out = Ms[0]
    for M in Ms[1:]:
        out = np.einsum("...ij,...jk->...ik", out, M)
    return out


def retr3(M):
    return np.real(np.trace(M, axis1=-2, axis2=-1)) / 3.0


def loop_traces(dims, U, cp, cr):
    """Per-loop weighted (1/3) Re tr of every plaquette (weight cp, each
    unoriented plaquette once) and every 2x1 rectangle (weight cr, both
    orientations), as one flat array (so differences can be taken loop by
    loop before summing)."""
    G = as_grid(dims, U)
    out = []
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            Um, Un = G[..., mu, :, :], G[..., nu, :, :]
            if mu < nu:
                P = mm(Um, fwd(Un, mu), dag(fwd(Um, nu)), dag(Un))
                out.append(cp * retr3(P).ravel())
            if cr != 0:
                # long side along mu: x -> x+mu -> x+2mu -> up nu -> back 2 mu -> down
                R = mm(Um, fwd(Um, mu), fwd(Un, mu, 2), dag(fwd(fwd(Um, nu), mu)), dag(fwd(Um, nu)), dag(Un))
                out.append(cr * retr3(R).ravel())
    return np.concatenate(out)


def expm_herm_i(H):
    """exp(i H) for Hermitian H via eigen-decomposition (numpy)."""
    e, v = np.linalg.eigh(H)
    return (v * np.exp(1j * e)[..., None, :]) @ dag(v)


def log_unitary(W):
    """Q Hermitian with exp(iQ) = W for unitary W with eigenphases in (-pi, pi)."""
    return -1j * scipy.linalg.logm(W)


def haar(rng, n):
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    q = q * np.exp(-1j * np.angle(np.linalg.det(q)) / 3)[:, None, None]
    return q


def unitarity_error(M):
    M = M.reshape(-1, 3, 3)
    e1 = np.abs(mm(M, dag(M)) - np.eye(3)).max()
    e2 = np.abs(np.linalg.det(M) - 1).max()
    return max(e1, e2)
