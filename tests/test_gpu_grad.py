"""Differentiation on the GPU (the training pattern that differentiates the
method; not in the paper): dR/dOmega, the matrix gradient of R, the
hand-written smearing backward (stout and over-improved stout) against the
oracle's independent reverse mode, autograd through StoutSmear + MCGFunctional
against the oracle and against central finite differences (h = 1e-6), and the
gradient-ascent refinement stage."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_0807_0264_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcg():
    from paper_0807_0264_gb300 import mcg as m

    return m


def pack(mcg, U, dims):
    return mcg.mcg_pack_links(torch.from_numpy(np.ascontiguousarray(U)).to("cuda").unsqueeze(0), dims)


def unpack(mcg, Ud, dims):
    return mcg.mcg_unpack_links(Ud, dims)[0].cpu().numpy()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 6)])
def test_grad_R_matches_oracle(mcg, dims):
    U = synth.make_field(dims, 0.5, 3)
    g = mcg.mcg_grad_R(pack(mcg, U, dims), dims)[0].cpu().numpy()
    ref = oracle.grad_R(dims, U)
    assert np.abs(g - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_functional_matrix_grad_matches_oracle(mcg):
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 4)
    G = mcg.mcg_functional_matrix_grad(pack(mcg, U, dims), dims)
    np.testing.assert_allclose(unpack(mcg, G, dims), oracle.functional_matrix_grad(dims, U), atol=1e-14)


@pytest.mark.parametrize("eps,rho", [(1.0, 0.1), (-0.25, 0.06)])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 6)])
def test_smear_backward_step_matches_oracle(mcg, dims, eps, rho):
    U = synth.make_field(dims, 0.5, 5)
    rng = np.random.default_rng(0)
    Gout = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    ref = oracle.smear_step_backward(dims, U, Gout, rho, eps)
    Gin = mcg.mcg_smear_backward_step(pack(mcg, U, dims), pack(mcg, Gout, dims), dims, rho, eps)
    got = unpack(mcg, Gin, dims)
    assert np.abs(got - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("eps,rho,n", [(1.0, 0.1, 3), (-0.25, 0.06, 2)])
def test_autograd_through_smearing_and_functional(mcg, eps, rho, n):
    """L(U) = R(smear_n(U)): autograd gradient equals the oracle's reverse mode
    and central finite differences of the GPU forward."""
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 6)
    Ud = pack(mcg, U, dims).requires_grad_(True)
    L = mcg.MCGFunctional.apply(mcg.StoutSmear.apply(Ud, dims, rho, eps, n), dims).sum()
    L.backward()
    G = unpack(mcg, Ud.grad.detach().contiguous(), dims)
    S = oracle.smear(dims, U, rho, eps, n)
    ref = oracle.smear_backward(dims, U, oracle.functional_matrix_grad(dims, S), rho, eps, n)
    assert np.abs(G - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())
    T = oracle.generators()
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(6):
        x, mu, a = int(rng.integers(256)), int(rng.integers(4)), int(rng.integers(8))
        vals = []
        for s in (+1, -1):
            Up = U.copy()
            Up[x, mu] = scipy.linalg.expm(1j * s * h * T[a]) @ U[x, mu]
            vals.append(mcg.mcg_functional(mcg.mcg_smear(pack(mcg, Up, dims), dims, rho, eps, n), dims)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        an = np.real(np.trace(G[x, mu].conj().T @ (1j * T[a] @ U[x, mu])))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_ascent_step_first_order(mcg):
    """d/d alpha R(ascent step alpha) at alpha = 0 equals |dR/d eps|^2."""
    dims = (4, 4, 4, 4)
    U = synth.make_field(dims, 0.5, 7)
    Ud = pack(mcg, U, dims)
    grad = mcg.mcg_grad_R(Ud, dims)
    g2 = float((grad ** 2).sum())
    alpha = 1e-6
    vals = []
    for s in (+1, -1):
        Ut, Gt = Ud.clone(), mcg.identity_gauge(dims)
        mcg.mcg_ascent_step(Ut, Gt, grad, dims, s * alpha)
        vals.append(mcg.mcg_functional(Ut, dims)[0])
        # the transform is tracked: U_t = U^G_t
        np.testing.assert_allclose(unpack(mcg, Ut, dims),
                                   oracle.apply_gauge(dims, U, mcg.mcg_unpack_gauge(Gt, dims)[0].cpu().numpy()),
                                   atol=1e-13)
    assert abs((vals[0] - vals[1]) / (2 * alpha) - g2) < 1e-6 * g2


def test_ascent_refinement_stage(mcg):
    """Gradient ascent raises R from a partly relaxed field and leaves a
    converged field (a local maximum) where it is."""
    dims = (6, 4, 4, 6)
    U = synth.make_field(dims, 0.5, 8)
    Ud, Gd = pack(mcg, U, dims), mcg.identity_gauge(dims)
    mcg.mcg_fix(Ud, Gd, dims, mcg.Params(tol=-1e300, max_sweeps=3))
    R0 = mcg.mcg_functional(Ud, dims)[0]
    res = mcg.ascent_refine(Ud, Gd, dims, steps=15, alpha=0.02)
    assert res["R"] > R0
    assert all(b >= a for a, b in zip(res["R_hist"], res["R_hist"][1:]))
    np.testing.assert_allclose(unpack(mcg, Ud, dims),
                               oracle.apply_gauge(dims, U, mcg.mcg_unpack_gauge(Gd, dims)[0].cpu().numpy()),
                               atol=1e-12)
    Uc, Gc = pack(mcg, U, dims), mcg.identity_gauge(dims)
    mcg.mcg_fix(Uc, Gc, dims, mcg.Params(tol=1e-12, max_sweeps=3000))
    Rc = mcg.mcg_functional(Uc, dims)[0]
    rc = mcg.ascent_refine(Uc, Gc, dims, steps=5, alpha=0.02)
    assert rc["R"] - Rc < 1e-8 * Rc


def test_differentiation_16x4_stout10(mcg):
    """The 16^4, n = 10, rho = 0.1 FP64 case: forward + hand-written backward
    run at full size; the gradient agrees with central differences of the GPU
    forward along sampled link directions."""
    dims = (16, 16, 16, 16)
    U = synth.make_field(dims, 0.5, 9)
    Ud = pack(mcg, U, dims).requires_grad_(True)
    L = mcg.MCGFunctional.apply(mcg.StoutSmear.apply(Ud, dims, 0.1, 1.0, 10), dims).sum()
    L.backward()
    G = unpack(mcg, Ud.grad.detach().contiguous(), dims)
    assert np.isfinite(G).all()
    T = oracle.generators()
    # R ~ 2e6 here: rounding of R (~ulp 2e-10) over 2h limits central
    # differences, so h = 1e-4 (truncation ~h^2, rounding ~1e-6)
    h = 1e-4
    rng = np.random.default_rng(3)
    for _ in range(3):
        x, mu, a = int(rng.integers(65536)), int(rng.integers(4)), int(rng.integers(8))
        vals = []
        for s in (+1, -1):
            Up = U.copy()
            Up[x, mu] = scipy.linalg.expm(1j * s * h * T[a]) @ U[x, mu]
            vals.append(mcg.mcg_functional(mcg.mcg_smear(pack(mcg, Up, dims), dims, 0.1, 1.0, 10), dims)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        an = np.real(np.trace(G[x, mu].conj().T @ (1j * T[a] @ U[x, mu])))
        assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (fd, an)
