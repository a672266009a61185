"""Comparison of preconditioning levels across configurations (Sec. III,
Tables 2 and 3): host-side statistics over per-configuration results of the
preconditioning pipeline, plus a driver that produces those results on the
GPU for a batch of configurations.

For levels ordered l_0 < l_1 < ... (by smearing), configuration c has a
gauge-fixing maximum V[c][l] and a P-vortex count n[c][l].  For a pair of
levels i < j (row i, column j in the paper's upper triangles):
  - fewer_vortices_pct[i][j]: % of configurations with n[c][j] < n[c][i]
    (Table 2, upper triangle);
  - vortex_reduction_pct[j][i] (mean) and its standard deviation: the %
    reduction 100 (n[c][i] - n[c][j]) / n[c][i] over those configurations
    (Table 2, lower triangle);
  - higher_max_pct[i][j]: % of configurations with V[c][j] > V[c][i]
    (Table 3, upper triangle);
  - fewer_given_higher_pct[j][i]: of those, the % with n[c][j] < n[c][i]
    (Table 3, lower triangle).
Entries without configurations to average over are NaN.
"""
from __future__ import annotations

import numpy as np


def transition_tables(V, vortices) -> dict:
    """Tables 2 and 3 of Sec. III from V[c][l] and vortex counts n[c][l]."""
    V = np.asarray(V, dtype=np.float64)
    n = np.asarray(vortices, dtype=np.float64)
    if V.shape != n.shape or V.ndim != 2:
        raise ValueError("V and vortices must both be (configurations, levels)")
    nc, nl = V.shape
    nan = np.full((nl, nl), np.nan)
    fewer, red_mean, red_std, higher, fewer_given = nan.copy(), nan.copy(), nan.copy(), nan.copy(), nan.copy()
    for i in range(nl):
        for j in range(i + 1, nl):
            dec = n[:, j] < n[:, i]
            fewer[i, j] = 100.0 * dec.mean()
            if dec.any():
                r = 100.0 * (n[dec, i] - n[dec, j]) / n[dec, i]
                red_mean[j, i] = r.mean()
                red_std[j, i] = r.std()
            hi = V[:, j] > V[:, i]
            higher[i, j] = 100.0 * hi.mean()
            if hi.any():
                fewer_given[j, i] = 100.0 * (n[hi, j] < n[hi, i]).mean()
    return {"configurations": nc, "fewer_vortices_pct": fewer, "vortex_reduction_pct": red_mean,
            "vortex_reduction_std": red_std, "higher_max_pct": higher, "fewer_given_higher_pct": fewer_given}


def precondition_study(fields, dims, levels, params, rho: float = 0.1, eps: float = 1.0, smear_precision=None):
    """Runs the preconditioning pipeline at every level for each configuration
    of `fields` (FP64 device tensors, one field each) and returns the
    per-configuration results with the Tables 2/3 statistics:
    dict(V=[c][l], vortices=[c][l], sweeps=[c][l], converged=[c][l], tables=...)."""
    from . import mcg

    V, nv, sw, conv = [], [], [], []
    for U in fields:
        res = mcg.mcg_precondition_levels(U, dims, list(levels), params, rho=rho, eps=eps,
                                          smear_precision=smear_precision)[3]
        V.append([r["V_fixed"] for r in res])
        nv.append([r["vortices"] for r in res])
        sw.append([r["sweeps_smeared"] + r["sweeps_fixed"] for r in res])
        conv.append([r["status"] == 0 for r in res])
    return {"V": V, "vortices": nv, "sweeps": sw, "converged": conv, "tables": transition_tables(V, nv)}


def anneal_study(U, dims, params, T, nhit: int = 4, eps: float = 0.3, seed: int = 0) -> dict:
    """Simulated annealing as a Gribov-copy search variant (Sec. III.B): for each
    configuration of U (an FP64 device tensor of nf fields of one lattice),
    the relaxation `params` from Omega = 1 against annealing with the
    temperatures T from Omega = 1 followed by the same relaxation.  Returns,
    per variant ("plain", "annealed"), V_U, P-vortex counts, sweeps and
    convergence (and the acceptance of the annealing), plus the Tables 2/3
    statistics with level 0 = plain and level 1 = annealed."""
    from . import mcg

    nf = U.shape[0]
    vol = 1
    for d in dims:
        vol *= d
    out = {}
    for name in ("plain", "annealed"):
        Uw = U.clone()
        G = mcg.identity_gauge(dims, nf)
        acc = mcg.mcg_anneal(Uw, G, dims, T, nhit, eps, seed)["acceptance"] if name == "annealed" else None
        r = mcg.mcg_fix(Uw, G, dims, params)
        counts = mcg.mcg_center_project(Uw, dims)[1]
        out[name] = {"V": [R / (36.0 * vol) for R in r["R"]], "vortices": [c[0] for c in counts],
                     "sweeps": list(r["sweeps"]), "converged": bool(r["converged"]), "acceptance": acc}
    V = [[p, a] for p, a in zip(out["plain"]["V"], out["annealed"]["V"])]
    n = [[p, a] for p, a in zip(out["plain"]["vortices"], out["annealed"]["vortices"])]
    out["tables"] = transition_tables(V, n)
    return out
