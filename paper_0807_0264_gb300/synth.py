"""Seeded synthetic inputs: SU(3) gauge fields, Haar gauge transforms.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from.  It holds no step of the gauge-fixing method itself: it only
draws random numbers and assembles the synthetic field that stands in for the
paper's ensemble of quenched Luescher-Weisz configurations (Sec. III: 20^3 x 40,
beta = 4.52), which is not available.

Field model.  U_mu(x) = g(x) . exp(i w sum_a theta_a lambda_a / 2) . g(x+mu)^dagger
with g(x) Haar-random in SU(3), theta_a ~ N(0, 1) i.i.d. and lambda_a the
Gell-Mann matrices (tr lambda_a lambda_b = 2 delta_ab).  Because the algebra
noise is invariant under the adjoint action, E[exp(iH)] = m(w) * 1 and the mean
plaquette of such a field is m(w)^4 exactly in expectation.  The width
W_PLAQ_06 = 0.4326 gives m^4 = 0.600 (Monte Carlo estimate of m(w) with 4e5
algebra samples and bisection on w), the roughness the 20^3 x 40 workload asks
for.  w = 0 gives a pure-gauge field (plaquette exactly 1, maximal center gauge
functional reachable at 1).

Canonical host layout (the one every public converter accepts):
    U[t, z, y, x, mu, row, col]  complex128, x fastest; mu = 0..3 is x, y, z, t
    g[t, z, y, x, row, col]      complex128
i.e. site index i = x + Nx*(y + Ny*(z + Nz*t)), dims = (Nx, Ny, Nz, Nt).

Random streams: numpy's Philox4x32-10 counter-based generator keyed by the
seed, so the same seed gives the same field on x86 and Arm hosts.
"""
from __future__ import annotations

import numpy as np

W_PLAQ_06 = 0.4326

# Planted-vortex workload (make_vortex_field): 48 sheet pairs on 20^3 x 40
# pierce 60 000 of the 1 920 000 plaquettes (3.1 %, the order of the paper's
# P-vortex densities, Sec. III Table 1); with them the width 0.4123 gives a
# mean plaquette of 0.600 (width_for_plaquette(0.6, 0.03125)).
VORTEX_PAIRS_20x40 = 48
W_VORTEX_06 = 0.4123

_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1] = -1j
_GELL_MANN[1][1, 0] = 1j
_GELL_MANN[2][0, 0] = 1
_GELL_MANN[2][1, 1] = -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2] = -1j
_GELL_MANN[4][2, 0] = 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2] = -1j
_GELL_MANN[6][2, 1] = 1j
_GELL_MANN[7] = np.diag([1.0, 1.0, -2.0]) / np.sqrt(3.0)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3), tr(l_a l_b) = 2 delta_ab."""
    return _GELL_MANN.copy()


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-random SU(3) matrices (Mezzadri 2007: QR of a complex Ginibre
    matrix with the phases of diag(R) divided out, then the determinant's
    principal cube root divided out)."""
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q * np.exp(-1j * np.angle(det) / 3.0)[:, None, None]
    return q


def _exp_i_hermitian(h: np.ndarray) -> np.ndarray:
    e, v = np.linalg.eigh(h)
    return np.einsum("nij,nj,nkj->nik", v, np.exp(1j * e), v.conj())


def lattice_volume(dims) -> int:
    nx, ny, nz, nt = (int(d) for d in dims)
    return nx * ny * nz * nt


def make_field(dims, width: float, seed: int, gauge: bool = True) -> np.ndarray:
    """Synthetic SU(3) link field in the canonical layout, shape (V, 4, 3, 3).

    dims = (Nx, Ny, Nz, Nt).  width is the algebra noise w; width = 0 gives a
    pure-gauge field.  gauge=False skips the random gauge rotation g(x) (links
    then sit near the identity).
    """
    nx, ny, nz, nt = (int(d) for d in dims)
    vol = nx * ny * nz * nt
    rng = _rng(seed)
    g = haar_su3(rng, vol).reshape(nt, nz, ny, nx, 3, 3)
    theta = rng.standard_normal((vol * 4, 8))
    h = (width / 2.0) * np.einsum("na,aij->nij", theta, _GELL_MANN)
    e = _exp_i_hermitian(h).reshape(nt, nz, ny, nx, 4, 3, 3)
    if not gauge:
        return np.ascontiguousarray(e.reshape(vol, 4, 3, 3))
    u = np.empty_like(e)
    axis_of_mu = (3, 2, 1, 0)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=axis_of_mu[mu])
        u[..., mu, :, :] = np.einsum("...ij,...jk,...lk->...il", g, e[..., mu, :, :], g_fwd.conj())
    return np.ascontiguousarray(u.reshape(vol, 4, 3, 3))


def center_sheets(dims, npairs: int, seed: int) -> np.ndarray:
    """Center phases k_mu(x) in {0, 1, 2} of npairs planted thin vortex-sheet
    pairs (link U_mu(x) is to be multiplied by exp(2 pi i k_mu(x) / 3)).

    Each pair draws a plane (mu, nu), mu != nu, a layer n0 of x_nu, a segment
    a <= x_mu < b with 1 <= a < b <= N_mu, and a charge c in {1, 2}; the links
    U_nu(x) with x_nu = n0 and x_mu in the segment get k += c (mod 3).  A
    (mu, nu) plaquette holds U_nu(x + mu) U_nu(x)^dag, so the center flux
    pierces the (mu, nu) plaquettes at x_nu = n0, x_mu = a - 1 (+c) and
    x_mu = b - 1 (-c), for every value of the two other coordinates: two
    sheets of V / (N_mu N_nu) plaquettes.  Sheets of different pairs that
    pierce the same plaquette add their fluxes mod 3.  Shape (V, 4), int8."""
    nx, ny, nz, nt = (int(d) for d in dims)
    n = (nx, ny, nz, nt)
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 0x5EED]))
    k = np.zeros((nt, nz, ny, nx, 4), dtype=np.int64)
    axis_of = (3, 2, 1, 0)  # array axis of direction mu in (t, z, y, x, mu)
    for _ in range(npairs):
        mu, nu = rng.choice(4, size=2, replace=False)
        n0 = int(rng.integers(0, n[nu]))
        a = int(rng.integers(1, n[mu]))
        b = int(rng.integers(a + 1, n[mu] + 1))
        c = int(rng.integers(1, 3))
        sl = [slice(None)] * 4
        sl[axis_of[nu]] = n0
        sl[axis_of[mu]] = slice(a, b)
        k[tuple(sl) + (nu,)] += c
    return np.ascontiguousarray((k % 3).astype(np.int8).reshape(nx * ny * nz * nt, 4))


def make_vortex_field(dims, width: float, seed: int, npairs: int, gauge: bool = True):
    """make_field(dims, width, seed, gauge) with the center phases of
    center_sheets(dims, npairs, seed) multiplied into the links: a field with
    planted thin center vortices, whose P-vortices a maximal-center-gauge
    fix and center projection should recover.  A center element commutes with
    every matrix, so the links are z^k g(x) exp(i w theta.lambda/2) g(x+mu)^dag.
    The mean plaquette is m(w)^4 (1 - 3 rho / 2) in expectation, rho the
    fraction of pierced plaquettes (each pierced one has Re z = -1/2).
    Returns (U, k)."""
    U = make_field(dims, width, seed, gauge)
    k = center_sheets(dims, npairs, seed)
    U = U * np.exp(2j * np.pi * k.astype(np.float64) / 3.0)[:, :, None, None]
    return np.ascontiguousarray(U), k


def mean_trace(width: float, nsamples: int = 400_000, seed: int = 12345) -> float:
    """Monte Carlo estimate of m(w) = E[(1/3) Re tr exp(i w theta.lambda / 2)]
    over the generator's algebra noise (theta_a ~ N(0, 1))."""
    rng = _rng(seed)
    theta = rng.standard_normal((nsamples, 8))
    h = (width / 2.0) * np.einsum("na,aij->nij", theta, _GELL_MANN)
    e = np.linalg.eigvalsh(h)
    return float(np.mean(np.cos(e).sum(axis=1)) / 3.0)


def width_for_plaquette(target: float, pierced_fraction: float = 0.0, nsamples: int = 400_000) -> float:
    """Noise width w with m(w)^4 (1 - 3 rho / 2) = target (bisection on the
    Monte Carlo m(w), common random numbers across w)."""
    goal = target / (1.0 - 1.5 * pierced_fraction)
    lo, hi = 0.0, 2.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if mean_trace(mid, nsamples) ** 4 > goal:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def random_gauge(dims, seed: int) -> np.ndarray:
    """Haar-random gauge transform, one SU(3) matrix per site, shape (V, 3, 3)."""
    vol = lattice_volume(dims)
    return np.ascontiguousarray(haar_su3(_rng(seed), vol))


def identity_gauge(dims) -> np.ndarray:
    vol = lattice_volume(dims)
    g = np.zeros((vol, 3, 3), dtype=np.complex128)
    g[:, 0, 0] = g[:, 1, 1] = g[:, 2, 2] = 1.0
    return g


def random_center_gauge(dims, seed: int) -> np.ndarray:
    """Gauge transform with a random Z3 center element exp(2 pi i k / 3) per site."""
    vol = lattice_volume(dims)
    k = _rng(seed).integers(0, 3, size=vol)
    g = np.zeros((vol, 3, 3), dtype=np.complex128)
    z = np.exp(2j * np.pi * k / 3.0)
    g[:, 0, 0] = g[:, 1, 1] = g[:, 2, 2] = z
    return g
