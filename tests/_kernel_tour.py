"""Run one small case through every kernel family of libmcg and print one
JSON line: the observables each call returns and, for an index-checking
build (MCG_LIBRARY naming libmcg_check.so), the number of out-of-range
indices the kernels met.  Used by tests/test_gpu_check_build.py, which runs
it once on the regular and once on the checking library."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_0807_0264_gb300 import mcg, synth  # noqa: E402


def main():
    dev = torch.device("cuda", 0)
    out = {}
    mcg.mcg_bounds_violations(reset=True)
    for dims in ((4, 4, 4, 6), (6, 4, 2, 8)):
        key = "x".join(map(str, dims))
        U0 = mcg.mcg_pack_links(torch.from_numpy(synth.make_field(dims, 0.6, 1)).unsqueeze(0).to(dev), dims)
        G0 = mcg.mcg_pack_gauge(torch.from_numpy(synth.random_gauge(dims, 2)).unsqueeze(0).to(dev), dims)
        r = {}
        r["plaq"] = mcg.mcg_plaquette(U0, dims)[0]
        S = mcg.mcg_smear(U0, dims, 0.1, 1.0, 2)
        r["plaq_stout"] = mcg.mcg_plaquette(S, dims)[0]
        r["plaq_oi"] = mcg.mcg_plaquette(mcg.mcg_smear(U0, dims, 0.06, -0.25, 2), dims)[0]
        r["plaq_stout32"] = mcg.mcg_plaquette(mcg.mcg_smear(mcg.mcg_convert(U0, mcg.F32), dims, 0.1, 1.0, 2), dims)[0]
        Ua = U0.clone()
        mcg.mcg_apply_gauge(Ua, G0, dims)
        r["R_applied"] = mcg.mcg_functional(Ua, dims)[0]
        for name, p in (("exact", mcg.Params(tol=-1e300, max_sweeps=20, check_every=5, reunit_every=7)),
                        ("solve32", mcg.Params(tol=-1e300, max_sweeps=20, check_every=5, reunit_every=7,
                                               fp64_solve32=1)),
                        ("mixed_df", mcg.Params(tol=1e-10, max_sweeps=3000, check_every=25, fp32_sweeps=3000,
                                                fp32_tol=5e-11, fp32_window=25, fp32_overrelax=1.85, fp64_solve32=1,
                                                fp64_df=1))):
            U, G = U0.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
            res = mcg.mcg_fix(U, G, dims, p)
            r["R_" + name] = res["R"][0]
            r["sweeps_" + name] = res["sweeps"][0]
        Z, counts = mcg.mcg_center_project(U, dims)
        r["vortices"] = counts[0][0]
        Ur, Zl = mcg.mcg_vortex_remove(U, Z, dims)
        r["plaq_removed"] = mcg.mcg_plaquette(Ur, dims)[0]
        r["W"] = mcg.mcg_wilson_loops(U, dims, 2, 2)[0].ravel().tolist()
        r["W_off"] = mcg.mcg_wilson_loops_offaxis(U, dims, [[1, 1, 0], [1, 1, 1]], 2)[0].ravel().tolist()
        U, G = U0.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
        r["acc"] = mcg.mcg_anneal(U, G, dims, [1.0, 0.5], 2, 0.3, 7)["accepted"][0]
        r["grad"] = float(mcg.mcg_grad_R(U0, dims).abs().sum())
        gin = mcg.mcg_smear_backward_step(U0, torch.ones_like(U0), dims, 0.1, 1.0)
        r["smear_bwd"] = float(gin.abs().sum())
        # slab half-sweep and face copies on the lattice itself
        U, G = U0.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
        r["R_slab"] = mcg.mcg_halfsweep_slab(U, G, dims, 1, 1, dims[3] - 1, want_R=True)
        face = mcg.mcg_slab_face(U, mcg.empty_face(dims), dims, dims[3] - 1, 0, False)
        mcg.mcg_slab_face(U, face, dims, 0, 0, True)
        r["R_after_face"] = mcg.mcg_functional(U, dims)[0]
        # batches of several fields, and the levels pipeline
        Us = [U0.clone(), mcg.mcg_pack_links(torch.from_numpy(synth.make_field(dims, 0.6, 3)).unsqueeze(0).to(dev),
                                             dims)]
        Gs = [mcg.identity_gauge(dims, 1, mcg.F64, dev) for _ in Us]
        b = mcg.mcg_fix_batch(Us, Gs, [dims, dims], mcg.Params(tol=-1e300, max_sweeps=30, check_every=10,
                                                               fp32_sweeps=30, fp32_tol=-1e300, fp32_window=25,
                                                               fp32_overrelax=1.85))
        r["R_batch"] = b["R"]
        lv = mcg.mcg_precondition_levels(U0, dims, [0, 2], mcg.Params(tol=1e-10, max_sweeps=3000, check_every=25,
                                                                      fp32_sweeps=3000, fp32_tol=5e-11,
                                                                      fp32_window=25, fp32_overrelax=1.85,
                                                                      fp64_solve32=1, fp64_df=1),
                                         rho=0.1, eps=1.0, smear_precision=mcg.F32)[3]
        r["levels"] = [[x["V_smeared"], x["V_fixed"], x["sweeps_fixed"], x["vortices"]] for x in lv]
        # restarts of the FP32 phase from random gauge copies, and the random transforms themselves
        U, G = U0.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
        rr = mcg.mcg_fix(U, G, dims, mcg.Params(tol=1e-10, max_sweeps=3000, check_every=10, fp32_sweeps=3000,
                                                fp32_tol=5e-11, fp32_window=25, fp32_overrelax=1.9, fp64_df=1,
                                                fp32_restart=30, fp32_restart_domega=0.15, fp32_restart_random=1,
                                                fp32_restart_creep=200))
        r["R_restarted"] = rr["R"][0]
        r["random_gauge"] = float(mcg.mcg_random_gauge(dims, seed=3, seq=1).abs().sum())
        out[key] = r
    # the local solve entry point, both precisions, on a few seeded problems
    rng = np.random.default_rng(5)
    A = rng.standard_normal((70, 4, 4))
    A = torch.from_numpy(A + A.transpose(0, 2, 1)).to(dev)
    b = torch.from_numpy(rng.standard_normal((70, 4))).to(dev)
    for name, prec in (("local_f64", mcg.F64), ("local_f32", mcg.F32)):
        a, fb = mcg.mcg_local_solve(A, b, prec)
        out[name] = [float(a.abs().sum()), int(fb.sum())]
    torch.cuda.synchronize()
    print(json.dumps({"violations": mcg.mcg_bounds_violations(), "results": out}), flush=True)


if __name__ == "__main__":
    main()
