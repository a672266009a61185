"""Restarts of the FP32 phase (mcg_params.fp32_restart): a field that has not
reached fp32_tol after `fp32_restart` sweeps since its (re)start begins the
phase again from the call's input with the next over-relaxation of the
sequence omega - d, omega + d, omega - 2d, ...  The restarted phase is a fresh
run with that over-relaxation: the same links and transform bit for bit, its
sweeps added to those before the restart.  Per-field arithmetic does not
depend on the batch, so a field restarted inside a batch (per-field chains
up to 16 fields, one launch per half-sweep above) ends as it does alone."""
import numpy as np
import pytest

from paper_0807_0264_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcg():
    from paper_0807_0264_gb300 import mcg as m

    return m


def params(mcg, omega, restart=0, domega=0.0):
    # d = 0.15 from omega = 1.9: one restart (omega 1.75), then 2.05 is out of
    # (0, 2) and the field carries on
    return mcg.Params(tol=1e-10, max_sweeps=6000, check_every=10, reunit_every=50, fp32_sweeps=6000, fp32_tol=5e-11,
                      fp32_window=25, fp32_overrelax=omega, fp64_df=1, fp32_restart=restart,
                      fp32_restart_domega=domega)


def packed(mcg, U, dims):
    return mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), dims)


def test_restarted_phase_is_a_fresh_run_with_the_next_omega(mcg):
    dims = (6, 4, 4, 6)
    U = synth.make_field(dims, 0.5, 12)
    Ur, Gr = packed(mcg, U, dims), mcg.identity_gauge(dims)
    rr = mcg.mcg_precondition_fix(Ur, Gr, dims, params(mcg, 1.9, restart=30, domega=0.15))[0]
    Uf, Gf = packed(mcg, U, dims), mcg.identity_gauge(dims)
    rf = mcg.mcg_precondition_fix(Uf, Gf, dims, params(mcg, 1.75))[0]
    assert rr["fp32_restarts"] == 1 and rf["fp32_restarts"] == 0
    assert rr["status"] == 0 and rf["status"] == 0
    assert torch.equal(Ur, Uf) and torch.equal(Gr, Gf)
    assert rr["V_fixed"] == rf["V_fixed"]
    # the sweeps before the restart: the first chunk boundary at or past 30,
    # plus the chunk already in flight when it was read
    pre = rr["sweeps_fixed"] - rf["sweeps_fixed"]
    assert pre == rr["sweeps_fp32"] - rf["sweeps_fp32"]
    assert 30 <= pre <= 50, pre


@pytest.mark.parametrize("nfields", [3, 18])
def test_restart_inside_a_batch_equals_the_field_alone(mcg, nfields):
    """3 fields: per-field chains (restart descriptors of the chain); 18
    fields: one launch per half-sweep for the batch (the batch's
    descriptors).  Each field is compared with its own restarted run."""
    dims_list = [(4, 4, 4, 6) if k % 2 else (4, 4, 4, 4) for k in range(nfields)]
    Us = [synth.make_field(d, 0.5, 70 + k) for k, d in enumerate(dims_list)]
    p = params(mcg, 1.9, restart=30, domega=0.15)
    Ub = [packed(mcg, U, d) for U, d in zip(Us, dims_list)]
    Gb = [mcg.identity_gauge(d) for d in dims_list]
    rb = mcg.mcg_fix_batch(Ub, Gb, dims_list, p)
    for k in sorted({0, 1, nfields // 2, nfields - 1}):
        d = dims_list[k]
        U1, G1 = packed(mcg, Us[k], d), mcg.identity_gauge(d)
        r1 = mcg.mcg_fix(U1, G1, d, p)
        assert rb["sweeps"][k] == r1["sweeps"][0]
        assert torch.equal(Ub[k], U1) and torch.equal(Gb[k], G1)
    # the restart took place: field 0 ends elsewhere without it
    U0, G0 = packed(mcg, Us[0], dims_list[0]), mcg.identity_gauge(dims_list[0])
    mcg.mcg_fix(U0, G0, dims_list[0], params(mcg, 1.9))
    assert not torch.equal(Ub[0], U0)


def test_restart_off_changes_nothing(mcg):
    """fp32_restart = 0 (the default) is the schedule without restarts, bit
    for bit, whatever fp32_restart_domega says."""
    dims = (4, 4, 4, 6)
    U = synth.make_field(dims, 0.5, 5)
    a, ga = packed(mcg, U, dims), mcg.identity_gauge(dims)
    ra = mcg.mcg_fix(a, ga, dims, params(mcg, 1.9))
    b, gb = packed(mcg, U, dims), mcg.identity_gauge(dims)
    rb = mcg.mcg_fix(b, gb, dims, params(mcg, 1.9, restart=0, domega=0.3))
    assert ra["sweeps"] == rb["sweeps"] and torch.equal(a, b) and torch.equal(ga, gb)


def test_random_restart_is_a_fresh_run_from_the_random_copy(mcg):
    """fp32_restart_random = 1: the k-th restart applies the transform W0 of
    mcg_random_gauge(seed MCG_RESTART_SEED, seq k) to the links and
    left-multiplies the transform by it; from there the phase is a fresh run
    with the next over-relaxation, bit for bit."""
    dims = (6, 4, 4, 6)
    U = synth.make_field(dims, 0.5, 12)
    p = params(mcg, 1.9, restart=30, domega=0.15)
    p.fp32_restart_random = 1
    Ur, Gr = packed(mcg, U, dims), mcg.identity_gauge(dims)
    rr = mcg.mcg_fix(Ur, Gr, dims, p)
    W0 = mcg.mcg_random_gauge(dims, seed=mcg.RESTART_SEED, seq=1)
    Uf = packed(mcg, U, dims)
    mcg.mcg_apply_gauge(Uf, W0, dims)
    Gf = W0.clone()
    rf = mcg.mcg_fix(Uf, Gf, dims, params(mcg, 1.75))
    assert rr["converged"] and rf["converged"]
    assert torch.equal(Ur, Uf) and torch.equal(Gr, Gf)
    assert 30 <= rr["sweeps"][0] - rf["sweeps"][0] <= 50


def test_random_gauge_is_haar_su3(mcg):
    """mcg_random_gauge: every matrix in SU(3) to rounding, the same in each
    field, reproducible, another sequence another draw; the first two moments
    of the trace are those of the Haar measure on SU(3): E tr G = 0 and
    E |tr G|^2 = 1 (one irreducible representation), within 5 standard
    errors over the 2 * 8^3 * 16 sites."""
    dims = (8, 8, 8, 16)
    G = mcg.mcg_random_gauge(dims, nfields=2, seed=5, seq=3)
    M = mcg.mcg_unpack_gauge(G, dims).cpu().numpy()
    assert np.array_equal(M[0], M[1])
    assert torch.equal(G, mcg.mcg_random_gauge(dims, nfields=2, seed=5, seq=3))
    assert not torch.equal(G, mcg.mcg_random_gauge(dims, nfields=2, seed=5, seq=4))
    m = M[0]
    eye = np.eye(3)
    assert np.abs(np.einsum("nji,njk->nik", m.conj(), m) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(m) - 1.0).max() < 1e-14
    tr = np.einsum("nii->n", m)
    n = len(tr)
    assert abs(tr.mean()) < 5.0 / np.sqrt(n)
    a2 = np.abs(tr) ** 2
    assert abs(a2.mean() - 1.0) < 5.0 * a2.std() / np.sqrt(n)


def test_creep_detector_restarts_only_the_creeping_fix(mcg):
    """The benchmark workload (20^3 x 40, stout rho = 0.1, n = 0, 4, 10, 20,
    omega 1.9): the preconditioned fix of level 20 creeps toward the lower
    maximum (per-chunk dV_U ~2e-10, flat for 20 000 sweeps) while every other
    fix's dV_U decays to the FP32 drift floor (~3e-11).  With the creep test
    alone (3 000 sweeps, no sweep-count restart) only that fix restarts, early,
    and every level converges."""
    dims = (20, 20, 20, 40)
    U = mcg.mcg_pack_links(torch.from_numpy(synth.make_field(dims, synth.W_PLAQ_06, 0)).unsqueeze(0).cuda(), dims)
    p = mcg.Params(tol=1e-10, max_sweeps=30000, check_every=25, reunit_every=50, fp32_sweeps=30000, fp32_tol=5e-11,
                   fp32_window=25, fp32_overrelax=1.9, fp64_solve32=1, fp64_df=1, fp32_restart=0,
                   fp32_restart_domega=0.03, fp32_restart_random=1, fp32_restart_creep=3000)
    res = mcg.mcg_precondition_levels(U, dims, [0, 4, 10, 20], p, rho=0.1, eps=1.0, smear_precision=mcg.F32)[3]
    print([(r["sweeps_smeared"], r["sweeps_fixed"], r["fp32_restarts"], r["status"]) for r in res])
    assert [r["status"] for r in res] == [0, 0, 0, 0]
    assert [r["fp32_restarts"] for r in res[:3]] == [0, 0, 0]
    assert res[3]["fp32_restarts"] >= 1
    # the creeping fix gave up after ~3 400 sweeps, not after the 30 000 cap
    assert res[3]["sweeps_fixed"] < 15000


def test_plain_fp32_finish_converges_by_the_oracle_criterion(mcg):
    """fp32_plain_finish = 1: plain FP32 sweeps follow the over-relaxed ones
    before the hand-off; the fix still ends on the paper's criterion (one more
    exact FP64 sweep of the oracle raises V_U by less than 1e-10) and on the
    input's gauge orbit.  With omega = 1 the flag changes nothing."""
    import oracle

    dims = (8, 8, 8, 8)
    U = synth.make_field(dims, synth.W_PLAQ_06, 1)
    p = params(mcg, 1.9)
    p.fp32_plain_finish = 1
    Ud, Gd = packed(mcg, U, dims), mcg.identity_gauge(dims)
    res = mcg.mcg_fix(Ud, Gd, dims, p)
    assert res["converged"]
    Uf = mcg.mcg_unpack_links(Ud, dims)[0].cpu().numpy()
    Gf = mcg.mcg_unpack_gauge(Gd, dims)[0].cpu().numpy()
    assert np.abs(oracle.apply_gauge(dims, U, Gf) - Uf).max() < 1e-12
    r = oracle.fix(dims, Uf, Gf, tol=-1e300, max_sweeps=1, reunit_every=0)
    assert (r["R_hist"][1] - r["R_hist"][0]) / (36 * 4096) < 1e-10
    a, ga = packed(mcg, U, dims), mcg.identity_gauge(dims)
    b, gb = packed(mcg, U, dims), mcg.identity_gauge(dims)
    q = params(mcg, 1.0)
    ra = mcg.mcg_fix(a, ga, dims, q)
    q.fp32_plain_finish = 1
    rb = mcg.mcg_fix(b, gb, dims, q)
    assert ra["sweeps"] == rb["sweeps"] and torch.equal(a, b) and torch.equal(ga, gb)
