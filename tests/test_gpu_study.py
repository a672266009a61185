"""The comparison of preconditioning levels across configurations (Tables 2
and 3 of Sec. III) on the GPU: the per-configuration, per-level maxima and
P-vortex counts of precondition_study equal the oracle's pipeline run level
by level, and its tables equal the host statistics of the oracle's values."""
import numpy as np
import pytest

import oracle
from paper_0807_0264_gb300 import synth
from paper_0807_0264_gb300.analysis import precondition_study, transition_tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_precondition_study_matches_oracle():
    from paper_0807_0264_gb300 import mcg

    dims = (4, 4, 4, 4)
    levels = (0, 2, 4)
    fields = [synth.make_field(dims, 0.9, seed) for seed in (31, 32, 33)]
    dev = [mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), dims) for U in fields]
    p = mcg.Params(tol=1e-10, max_sweeps=1500)
    st = precondition_study(dev, dims, levels, p, rho=0.1, eps=1.0, smear_precision=mcg.F64)
    Vo, no = [], []
    for U in fields:
        row_v, row_n = [], []
        for ns in levels:
            o = oracle.precondition_and_fix(dims, U, rho=0.1, eps=1.0, nsmear=ns, tol=1e-10, max_sweeps=1500)
            row_v.append(o["fixed"]["R_hist"][-1] / (36 * 256))
            row_n.append(o["vortices"])
        Vo.append(row_v)
        no.append(row_n)
    assert np.abs(np.array(st["V"]) - np.array(Vo)).max() < 1e-10
    assert st["vortices"] == no
    ref = transition_tables(Vo, no)
    for k in ("fewer_vortices_pct", "higher_max_pct", "fewer_given_higher_pct", "vortex_reduction_pct"):
        np.testing.assert_allclose(st["tables"][k], ref[k], equal_nan=True)


def test_anneal_study_matches_oracle():
    """Simulated annealing as a Gribov-copy search variant: the plain and the
    annealed-then-relaxed maxima and P-vortex counts of anneal_study equal
    the oracle's anneal and relaxation run per configuration."""
    from paper_0807_0264_gb300 import mcg
    from paper_0807_0264_gb300.analysis import anneal_study

    dims = (4, 4, 4, 4)
    fields = [synth.make_field(dims, 0.9, seed) for seed in (41, 42, 43)]
    U = mcg.mcg_pack_links(torch.from_numpy(np.stack(fields)).cuda(), dims)
    T = mcg.anneal_schedule(2.0, 0.05, 10)
    p = mcg.Params(tol=1e-10, max_sweeps=1500)
    st = anneal_study(U, dims, p, T, nhit=2, eps=0.3, seed=3)
    V4 = 36.0 * 256
    for f, Uc in enumerate(fields):
        plain = oracle.fix(dims, Uc, None, tol=1e-10, max_sweeps=1500, reunit_every=50)
        Ua, Ga, acc = oracle.anneal(dims, Uc, synth.identity_gauge(dims), T, 2, 0.3, 3, field=f)
        ann = oracle.fix(dims, Ua, Ga, tol=1e-10, max_sweeps=1500, reunit_every=50)
        for name, o in (("plain", plain), ("annealed", ann)):
            assert st[name]["sweeps"][f] == o["sweeps"]
            assert abs(st[name]["V"][f] - o["R_hist"][-1] / V4) < 1e-11
            assert st[name]["vortices"][f] == oracle.vortex_count(dims, oracle.center_project(dims, o["U"]))[0]
        assert st["annealed"]["acceptance"][f] == acc / (len(T) * 256 * 3 * 2)
    V = [[a, b] for a, b in zip(st["plain"]["V"], st["annealed"]["V"])]
    n = [[a, b] for a, b in zip(st["plain"]["vortices"], st["annealed"]["vortices"])]
    ref = transition_tables(V, n)
    assert np.array_equal(np.nan_to_num(st["tables"]["higher_max_pct"], nan=-1),
                          np.nan_to_num(ref["higher_max_pct"], nan=-1))


def test_precondition_levels_mixed_fp32_smearing_matches_oracle_pipeline():
    """The entry point the benchmark times, with the benchmark's schedule
    (FP32 smearing, over-relaxed FP32 phase, double-float FP64-class finish),
    against the oracle's FP64 pipeline (plain relaxation, FP64 smearing) level
    by level on 8^4: the same maxima (V_U of the smeared and of the fixed
    field, the latter to 1e-9), the same P-vortex counts, the plaquette
    unchanged, and every output field equal to the input transformed by its
    output transform.  On this field each level has one dominant maximum, so
    the over-relaxed schedule and the plain relaxation end on it."""
    from paper_0807_0264_gb300 import mcg

    dims = (8, 8, 8, 8)
    U = synth.make_field(dims, 0.5, 7)
    levels = [0, 2, 4]
    Ud = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), dims)
    p = mcg.Params(tol=1e-10, max_sweeps=20000, check_every=25, reunit_every=50, fp32_sweeps=20000, fp32_tol=5e-11,
                   fp32_window=25, fp32_overrelax=1.85, fp64_solve32=1, fp64_df=1)
    Uo, Go, Zo, res = mcg.mcg_precondition_levels(Ud, dims, levels, p, rho=0.1, eps=1.0, smear_precision=mcg.F32)
    V4 = 36.0 * 4096
    for l, n in enumerate(levels):
        o = oracle.precondition_and_fix(dims, U, rho=0.1, eps=1.0, nsmear=n, tol=1e-10, max_sweeps=20000)
        r = res[l]
        assert r["status"] == 0
        assert abs(r["V_fixed"] - o["fixed"]["R_hist"][-1] / V4) < 1e-9
        if n:
            assert abs(r["V_smeared"] - o["smeared"]["R_hist"][-1] / V4) < 1e-6  # FP32 smearing
        assert r["vortices"] == o["vortices"]
        assert abs(r["plaquette_out"] - r["plaquette_in"]) < 1e-13
        Uf = mcg.mcg_unpack_links(Uo[l:l + 1], dims)[0].cpu().numpy()
        Gf = mcg.mcg_unpack_gauge(Go[l:l + 1], dims)[0].cpu().numpy()
        assert np.abs(oracle.apply_gauge(dims, U, Gf) - Uf).max() < 1e-12


def test_levels_report_convergence_per_level():
    """A level's status is its own: MCG_OK exactly when its fixes stopped
    below the sweep cap; the call's status is MCG_NOT_CONVERGED when any
    level is not converged."""
    from paper_0807_0264_gb300 import mcg

    dims = (6, 6, 6, 6)
    U = mcg.mcg_pack_links(torch.from_numpy(synth.make_field(dims, 0.9, 41)).unsqueeze(0).cuda(), dims)
    # the oracle's plain FP64 relaxation needs 2209 sweeps at n = 0, 91 + 1073
    # at n = 6 and 56 + 1456 at n = 12 on this field: a cap of 1200 stops
    # levels 0 and 12 and lets level 6 converge
    cap = 1200
    res = mcg.mcg_precondition_levels(U, dims, [0, 6, 12], mcg.Params(tol=1e-10, max_sweeps=cap), rho=0.1,
                                      eps=1.0, smear_precision=mcg.F64)[3]
    hit = []
    for n, r in zip((0, 6, 12), res):
        capped = r["sweeps_fixed"] >= cap or (n > 0 and r["sweeps_smeared"] >= cap)
        assert (r["status"] == mcg.OK) == (not capped), (n, r)
        hit.append(capped)
    assert hit == [True, False, True]
