"""Benchmark: MCG site-updates/s and time to dV_U < 1e-10 on the 20^3 x 40
preconditioning workload (Sec. II.B / Sec. III: stout smearing rho = 0.1 with
n in {0, 4, 10, 20} sweeps, each level conducted independently from the same
field), batched/mixed-precision form against the plain FP64 GPU sweep.

One step = the whole hot path over one synthetic field: smear (one chain,
snapshots at every level), MCG-fix the smeared fields as a batch, apply each
transform to a copy of the original, MCG-fix the preconditioned fields as a
batch, center-project and count P-vortices, plaquettes (mcg_precondition_levels).
A site-update is one site of one parity with all three SU(2) subgroups, so a
full sweep of one field is V = 320 000 site-updates.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM traffic of the dominant kernel per launch, from one ncu capture of a
# full 20^3 x 40 launch (the profile named below); reported only while the
# kernel source is the one that was profiled
TRAFFIC_FP32 = {"bytes_per_launch": 79.17e6, "source_sha256_prefix": "4c98a7ce6c5570b0",
                "profile": "profiles/k_halfsweep_c12_f32_20x20x20x40.md"}

def fp32_kernel_fingerprint() -> str:
    """sha256 over the sources of the FP32 half-sweep kernel (its unit, the
    shared sweep header, the device building blocks)."""
    import hashlib

    h = hashlib.sha256()
    for name in ("mcg_sweep_f32.cu", "mcg_sweep.cuh", "mcg_common.cuh"):
        with open(os.path.join(ROOT, "paper_0807_0264_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


METRIC = "MCG site-updates/s & time-to-ΔR<1e-10 at 20^3x40: batched/mixed vs plain FP64"
UNIT = "site-updates/s"
DIMS = (20, 20, 20, 40)
LEVELS = (0, 4, 10, 20)
RHO = 0.1
# over-relaxation of the FP32 phase; a scan over 1.7..1.95 (steps of 0.01
# from 1.85 to 1.93) on this workload converged every level only at 1.9 and
# 1.92 (the others leave one to four levels creeping)
OMEGA = float(os.environ.get("MCG_OMEGA", "1.9"))
# restart of a field's FP32 phase once it has run this many sweeps without
# reaching fp32_tol, from a random gauge copy of its input with the next
# over-relaxation of omega -+ k * 0.03: converging phases on these workloads
# take 2 000 to ~10 000 sweeps, the creeping (trap) ones run on to the cap
RESTART = int(os.environ.get("MCG_FP32_RESTART", "10000"))
RESTART_DOMEGA = float(os.environ.get("MCG_RESTART_DOMEGA", "0.03"))
RESTART_RANDOM = int(os.environ.get("MCG_RESTART_RANDOM", "1"))
# ... and once its per-chunk dV_U has stayed within [2, 20] x fp32_tol without
# decaying for this many sweeps (the creeping approach to a lower maximum;
# on the three 20^3 x 40 workloads only the creeping fixes meet it)
RESTART_CREEP = int(os.environ.get("MCG_RESTART_CREEP", "3000"))
# plain FP32 sweeps after the over-relaxed ones, before the hand-off (they
# remove the over-relaxation's oscillating residue at FP32 cost)
PLAIN_FINISH = int(os.environ.get("MCG_FP32_PLAIN_FINISH", "1"))


def hbm_peak():
    """The HBM roofline denominator: the measured copy bandwidth of this GPU
    pool (MEASURED_PEAKS.json, written by the driver), else the profiling
    recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--dims", type=int, nargs=4, default=list(DIMS))
    ap.add_argument("--levels", type=int, nargs="+", default=list(LEVELS))
    ap.add_argument("--rho", type=float, default=RHO)
    ap.add_argument("--eps", type=float, default=1.0, help="1: stout; -0.25: over-improved stout (Sec. II.B)")
    ap.add_argument("--config3", action="store_true",
                    help="the over-improved stout workload: eps = -0.25, rho = 0.06, n in {10, 20, 40}")
    ap.add_argument("--vortex-sheets", action="store_true",
                    help="the planted-vortex workload instead of the plain synthetic field: 48 thin center-vortex "
                         "sheet pairs (3.1 %% of the plaquettes pierced at 20^3 x 40), noise width recalibrated to a "
                         "mean plaquette of 0.6")
    ap.add_argument("--no-mixed-error", action="store_true",
                    help="skip the mixed schedule's error against the oracle's FP64 relaxation from the same "
                         "hand-off field")
    ap.add_argument("--mixed-error-levels", type=int, nargs="+", default=None,
                    help="levels for the mixed-error block (default: every level)")
    ap.add_argument("--mixed-error-cap", type=int, default=1500, help="oracle sweeps cap per level")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-observables", action="store_true",
                    help="skip the Sec. III.A measurement (vortex removal, Wilson loops) on the level-0 result")
    ap.add_argument("--profile-slice", action="store_true",
                    help="one bench step with sweeps capped (FP32 100 + FP64 1 per fix, levels 0 and 4, block sizes "
                         "128): the same kernels and launch shapes in ~1000 launches, for an ncu launch list")
    ap.add_argument("--gribov", action="store_true",
                    help="the batched Gribov-copy search at full size instead of the main step: 16 x 12^4, "
                         "16 x 16^3 x 32 and 16 x 20^3 x 40 configurations with 8 random initial transforms "
                         "each (384 fields, 60.4 M sites), fields generated on the GPU; one JSON line")
    ap.add_argument("--anneal", action="store_true",
                    help="simulated annealing as a Gribov-copy search variant instead of the main step: plain "
                         "relaxation against annealing (200 sweeps, T 2 -> 0.02, 4 hits) + relaxation on 16 x 12^4 "
                         "configurations (MCG_ANNEAL_DIMS, MCG_ANNEAL_CONFIGS), and the annealing sweep timed at "
                         "20^3 x 40; one JSON line")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="every kernel of the library once or twice on the 20^3 x 40 workload (smearing FP32/FP64/"
                         "over-improved, fix phases FP32/FP64 exact/FP64 with FP32 solve, hand-off, gauge "
                         "transforms, observables, center projection, vortex removal, Wilson loops, annealing, "
                         "gradients, input check): the launches for a per-kernel ncu metrics capture")
    ap.add_argument("--slabs", action="store_true",
                    help="time the t-slab decomposition of the FP64 relaxation (slabs in lockstep on this GPU, "
                         "faces exchanged on the device) against the single-domain FP64 sweep")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="measured FMA throughput of the GPU (FP64, FP32, packed FP32), one JSON line")
    ap.add_argument("--profile-kernel", choices=["f32", "f64"],
                    help="time the FP32 (or FP64) half-sweep on the field after 300 FP32 sweeps (the regime the FP32 "
                         "phase runs in), odd then even sites, 3 launches each, L2 flushed: the launches for an ncu "
                         "capture of the dominant kernel (the warm-up runs 600 FP32 half-sweeps first)")
    a = ap.parse_args()
    if a.config3:
        a.eps, a.rho, a.levels = -0.25, 0.06, [10, 20, 40]
    return a


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(U, dims, seconds: float, threads: int | None = None):
    """Oracle MCG sweeps on the workload field (identity start), bounded to
    about `seconds` of CPU work, on `threads` host threads (default: all the
    process may use); returns (site-updates/s, sweeps, threads)."""
    import oracle

    cores = threads or len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    V = 1
    for d in dims:
        V *= d
    t0 = time.perf_counter()
    r = oracle.fix(dims, U, None, tol=-1e300, max_sweeps=1, reunit_every=0)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.fix(dims, r["U"], r["G"], tol=-1e300, max_sweeps=n, reunit_every=0)
    dt = time.perf_counter() - t0
    return n * V / dt, n, cores


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_0807_0264_gb300 import synth

    dims = tuple(args.dims)
    U = synth.make_field(dims, synth.W_PLAQ_06, 0)
    import oracle

    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    V = 1
    for d in dims:
        V *= d
    per_step = max(1, int(os.environ.get("MCG_REF_SWEEPS_PER_STEP", "2")))
    state = oracle.fix(dims, U, None, tol=-1e300, max_sweeps=1, reunit_every=0)
    for _ in range(args.warmup):
        state = oracle.fix(dims, state["U"], state["G"], tol=-1e300, max_sweeps=1, reunit_every=0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        state = oracle.fix(dims, state["U"], state["G"], tol=-1e300, max_sweeps=per_step, reunit_every=0)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per_step * V / (ms / 1e3)
    sample = f"{per_step} oracle MCG sweeps per step on the {dims[0]}x{dims[1]}x{dims[2]}x{dims[3]} field"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(args, "oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_over_ranks(dist, x: float, op: str, device) -> float:
    """MAX or SUM of a scalar over the ranks of the default process group
    (identity without one)."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def smearing_name(args):
    return "stout" if args.eps == 1.0 else f"over-improved stout eps={args.eps:g}"


def config_of(args, form):
    d = tuple(args.dims)
    return {"workload": f"Sec. II.B preconditioned MCG, {d[0]}x{d[1]}x{d[2]}x{d[3]} SU(3), {smearing_name(args)} "
                        f"rho={args.rho:g} n in {list(args.levels)}, levels batched, dV_U<1e-10",
            "lattice": list(d), "levels": list(args.levels), "rho": args.rho, "eps": args.eps, "tol": 1e-10,
            "form": form,
            "field": ("synthetic z^k(x) g(x) exp(i w theta.lambda/2) g(x+mu)^dag with 48 planted center-vortex "
                      "sheet pairs (3.1 % of plaquettes pierced), w=0.4123 (plaquette 0.60), seed 0"
                      if args.vortex_sheets else
                      "synthetic g(x) exp(i w theta.lambda/2) g(x+mu)^dag, w=0.4326 (plaquette 0.60), seed 0"),
            "l2": "inputs larger than L2 (184 MB FP64 field, 4 x 184 MB outputs)"}


# ---------------------------------------------------------------------------
# batched Gribov-copy search at full size (--gribov)
# ---------------------------------------------------------------------------
def _haar_su3(n, gen, dev):
    """n Haar-random SU(3) matrices on the GPU, elementwise: Gram-Schmidt on two
    complex Gaussian rows (a Haar U(3) pair of rows), row 2 = conj(row0 x row1)
    (determinant 1)."""
    import torch

    r = torch.complex(torch.randn((n, 2, 3), generator=gen, dtype=torch.float64, device=dev),
                      torch.randn((n, 2, 3), generator=gen, dtype=torch.float64, device=dev))
    r0 = r[:, 0] / torch.linalg.vector_norm(r[:, 0], dim=-1, keepdim=True)
    r1 = r[:, 1] - (r0.conj() * r[:, 1]).sum(-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.linalg.cross(r0, r1, dim=-1).conj()
    return torch.stack((r0, r1, r2), dim=1).contiguous()


def _gpu_field(dims, w, seed, dev):
    """The synthetic field g(x) exp(i w theta.lambda/2) g(x+mu)^dag of the
    workload, generated with torch on the GPU (canonical layout, (1, V, 4, 3, 3))."""
    import torch

    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    g = _haar_su3(V, gen, dev).reshape(nt, nz, ny, nx, 3, 3)
    lam = torch.zeros((8, 3, 3), dtype=torch.complex128, device=dev)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / 3 ** 0.5
    lam[7, 2, 2] = -2 / 3 ** 0.5
    links = []
    for mu, ax in zip(range(4), (3, 2, 1, 0)):
        th = torch.randn((nt, nz, ny, nx, 8), generator=gen, dtype=torch.float64, device=dev).to(torch.complex128)
        H = torch.einsum("...a,aij->...ij", th, lam) * (0.5 * w)
        E = torch.linalg.matrix_exp(1j * H)
        gs = torch.roll(g, shifts=-1, dims=ax)
        links.append(g @ E @ gs.conj().transpose(-1, -2))
    return torch.stack(links, dim=4).reshape(1, V, 4, 3, 3).contiguous()


def run_gribov(args, mcg, dev, rank):
    import torch

    per = int(os.environ.get("MCG_GRIBOV_CONFIGS_PER_SIZE", "16"))
    sizes = [((12, 12, 12, 12), per), ((16, 16, 16, 32), per), ((20, 20, 20, 40), per)]
    ncopy = 8
    t_gen = time.perf_counter()
    Us, Gs, dims_list, cfg = [], [], [], []
    c = 0
    for dims, nconf in sizes:
        V = dims[0] * dims[1] * dims[2] * dims[3]
        for _ in range(nconf):
            canon = _gpu_field(dims, synth_w(), c, dev)
            if not bool(torch.isfinite(torch.view_as_real(canon)).all()):
                print(f"gribov: config {c} {dims} generated non-finite links", file=sys.stderr, flush=True)
            U = mcg.mcg_pack_links(canon, dims)
            del canon
            for k in range(ncopy):
                gen = torch.Generator(device=dev)
                gen.manual_seed(1000 + ncopy * c + k)
                Gc = mcg.mcg_pack_gauge(_haar_su3(V, gen, dev).unsqueeze(0), dims)
                Us.append(U.clone())
                Gs.append(Gc)
                dims_list.append(dims)
                cfg.append(c)
            del U
            c += 1
    torch.cuda.synchronize(dev)
    t_gen = time.perf_counter() - t_gen
    print(f"gribov: generated {len(Us)} fields in {t_gen:.1f} s", file=sys.stderr, flush=True)
    nconf_tot = c
    p = mcg.Params(tol=1e-10, max_sweeps=20000, check_every=25, reunit_every=50, fp32_sweeps=20000, fp32_tol=5e-11,
                   fp32_window=25, fp32_overrelax=OMEGA, fp64_solve32=1, fp32_restart=RESTART,
                   fp32_restart_domega=RESTART_DOMEGA, fp32_restart_random=RESTART_RANDOM,
                   fp32_restart_creep=RESTART_CREEP,
                   fp32_plain_finish=PLAIN_FINISH)
    tune = mcg.autotune_schedule(Us, dims_list, p, trial_sweeps=20, chunks=(25, 50))
    print(f"gribov: autotuned {tune['block']} x {tune['check_every']}", file=sys.stderr, flush=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = mcg.mcg_kernel_launches()
    e0.record()
    res = mcg.mcg_gribov_search(Us, Gs, dims_list, cfg, nconf_tot, p)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    vols = [d[0] * d[1] * d[2] * d[3] for d in dims_list]
    updates = sum(sw * v for sw, v in zip(res["sweeps"], vols))
    Vs = [r / (36.0 * v) for r, v in zip(res["R"], vols)]
    import math

    gain = []
    for cc in range(nconf_tot):
        ks = [k for k in range(len(cfg)) if cfg[k] == cc and math.isfinite(Vs[k])]
        if ks:
            gain.append(res["best_V"][cc] - sum(Vs[k] for k in ks) / len(ks))
    per_size = {}
    for dims, _ in sizes:
        ks = [k for k in range(len(dims_list)) if dims_list[k] == dims]
        fin = [Vs[k] for k in ks if math.isfinite(Vs[k])]
        per_size["x".join(map(str, dims))] = {
            "copies": len(ks), "non_finite_R": len(ks) - len(fin),
            "at_sweep_cap": sum(1 for k in ks if res["sweeps"][k] >= p.max_sweeps),
            "sweeps_mean": sum(res["sweeps"][k] for k in ks) / len(ks),
            "V_mean": (sum(fin) / len(fin)) if fin else None}
        if len(fin) < len(ks):
            print(f"gribov: non-finite R for copies {[k for k in ks if not math.isfinite(Vs[k])]}",
                  file=sys.stderr, flush=True)
    if rank == 0:
        print(json.dumps({
            "mode": "gribov_search", "metric": "batched Gribov-copy search site-updates/s", "unit": UNIT,
            "value": updates / (ms / 1e3), "ms": ms, "configs": nconf_tot, "copies": len(Us),
            "sites": sum(vols), "fp64_link_bytes": sum(vols) * 4 * 144, "site_updates": updates,
            "converged": res["converged"], "sweeps_min": min(res["sweeps"]), "sweeps_max": max(res["sweeps"]),
            "sweeps_mean": sum(res["sweeps"]) / len(res["sweeps"]),
            "best_minus_mean_copy_V": {"mean": sum(gain) / max(1, len(gain)), "max": max(gain) if gain else None},
            "per_size": per_size,
            "autotune": {"block": tune["block"], "check_every": tune["check_every"]},
            "generation_s": t_gen, "data": "synthetic fields and random transforms generated with torch on the GPU",
            "gpu_launches": mcg.mcg_kernel_launches() - launches0}), flush=True)


ANNEAL_T = (2.0, 0.02, 200)  # first and last temperature, sweeps (geometric schedule)


def anneal_flop_per_site(nhit: int) -> int:
    """FP64 flops of one annealing site update: per subgroup the local problem
    (8 links x 64), the move applied to 9 matrices (756), the start value of
    the quadratic form and the normalisation (56), and per hit the proposal,
    SU(2) product, quadratic form and acceptance (~110)."""
    return 3 * (512 + 756 + 56 + 110 * nhit)


def run_slabs(mcg, dims, U_host, dev, sweeps=20):
    """The domain decomposition along t (paper_0807_0264_gb300.domain) on one
    GPU: W slabs of the workload field driven in lockstep from the host, each
    half-sweep one mcg_halfsweep_slab launch per slab and one face copy each
    way per boundary (mcg_slab_face, device to device).  Times `sweeps` exact
    FP64 sweeps after 2 warm-up sweeps, against the single-domain FP64 sweep
    (mcg_fix, same arithmetic), and checks the links are the same bits."""
    import time

    import numpy as np
    import torch

    from paper_0807_0264_gb300 import domain, synth

    NEVER = -1e300
    G_host = synth.identity_gauge(dims)
    Ud = mcg.mcg_pack_links(torch.from_numpy(U_host).unsqueeze(0).to(dev), dims)
    Gd = mcg.identity_gauge(dims, 1, mcg.F64, dev)
    mcg.mcg_fix(Ud, Gd, dims, mcg.Params(tol=NEVER, max_sweeps=2, check_every=2, reunit_every=0))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    mcg.mcg_fix(Ud, Gd, dims, mcg.Params(tol=NEVER, max_sweeps=sweeps, check_every=sweeps, reunit_every=0))
    torch.cuda.synchronize(dev)
    single_ms = (time.perf_counter() - t0) * 1e3 / sweeps
    U_single = mcg.mcg_unpack_links(Ud, dims)[0].cpu().numpy()
    del Ud, Gd
    face_bytes = 9 * dims[0] * dims[1] * dims[2] // 2 * 16
    out = {"slabs": {"dims": list(dims), "sweeps": sweeps, "single_domain_ms_per_sweep": single_ms,
                     "face_bytes": face_bytes, "runs": []}}
    for W in (1, 2, 4):
        doms = [domain.SlabDomain(dims, r, W) for r in range(W)]
        bks = [domain.DeviceSlab(d, *d.scatter(U_host, G_host), device=dev) for d in doms]
        sw = [domain.Sweeper(d, b) for d, b in zip(doms, bks)]
        domain.run_ranks_lockstep(sw, NEVER, 2, reunit_every=0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        domain.run_ranks_lockstep(sw, NEVER, sweeps, reunit_every=0)
        torch.cuda.synchronize(dev)
        ms = (time.perf_counter() - t0) * 1e3 / sweeps
        Uo = np.concatenate([d.owned(*b.local_arrays())[0] for d, b in zip(doms, bks)])
        out["slabs"]["runs"].append({"W": W, "slab_layers": dims[3] // W, "ms_per_sweep": ms,
                                     "overhead": ms / single_ms - 1.0,
                                     "face_copies_per_sweep": 4 * W, "same_bits_as_single_domain":
                                     bool(np.array_equal(Uo, U_single))})
        del bks, sw
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_anneal(args, mcg, dev, rank):
    import torch

    from paper_0807_0264_gb300 import analysis

    T0, T1, ns = ANNEAL_T
    sched = mcg.anneal_schedule(T0, T1, ns)
    # (1) the annealing sweep at the 20^3 x 40 workload size, per sweep, from
    # the difference of a 12-sweep and a 2-sweep call (the fixed cost of a
    # call -- re-unitarisation and the counter read -- cancels)
    dims = (20, 20, 20, 40)
    U0 = mcg.mcg_pack_links(_gpu_field(dims, synth_w(), 0, dev), dims)
    sites = dims[0] * dims[1] * dims[2] * dims[3]
    timing = {}
    for nhit in (1, 4):
        ms = {}
        for nsw in (2, 12, 2, 12):
            U = U0.clone()
            G = mcg.identity_gauge(dims)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = mcg.mcg_anneal(U, G, dims, [1.0] * nsw, nhit, 0.3, 1)
            e1.record()
            torch.cuda.synchronize(dev)
            ms[nsw] = e0.elapsed_time(e1)  # the second (warm) call of each length is kept
        per_sweep = (ms[12] - ms[2]) / 10.0
        flop = anneal_flop_per_site(nhit) * sites
        timing[f"nhit{nhit}"] = {"ms_per_sweep": per_sweep, "site_updates_per_s": sites / (per_sweep / 1e3),
                                 "fp64_tflops_est": flop / (per_sweep / 1e3) / 1e12,
                                 "acceptance_at_T_1": r["acceptance"][0]}
    del U0
    # (2) the study: 16 configurations of 12^4 unless MCG_ANNEAL_DIMS ("nx,ny,nz,nt")
    # and MCG_ANNEAL_CONFIGS say otherwise
    dims = tuple(int(v) for v in os.environ.get("MCG_ANNEAL_DIMS", "12,12,12,12").split(","))
    nconf = int(os.environ.get("MCG_ANNEAL_CONFIGS", "16"))
    Us = torch.cat([_gpu_field(dims, synth_w(), 100 + c, dev) for c in range(nconf)])
    U = mcg.mcg_pack_links(Us, dims)
    del Us
    p = mcg.Params(tol=1e-10, max_sweeps=20000, check_every=25, reunit_every=50, fp32_sweeps=20000, fp32_tol=5e-11,
                   fp32_window=25, fp32_overrelax=OMEGA, fp64_solve32=1)
    t = time.perf_counter()
    st = analysis.anneal_study(U, dims, p, sched, nhit=4, eps=0.3, seed=7)
    t = time.perf_counter() - t
    pl, an = st["plain"], st["annealed"]
    tb = st["tables"]

    def mean(x):
        return sum(x) / len(x)

    if rank == 0:
        print(json.dumps({
            "mode": "anneal_study", "schedule": {"T0": T0, "T1": T1, "sweeps": ns, "nhit": 4, "eps": 0.3},
            "sweep_timing_20x20x20x40": timing,
            "configs": nconf, "dims": list(dims), "seconds": t,
            "V_mean": {"plain": mean(pl["V"]), "annealed": mean(an["V"])},
            "V_gain_mean": mean([b - a for a, b in zip(pl["V"], an["V"])]),
            "vortices_mean": {"plain": mean(pl["vortices"]), "annealed": mean(an["vortices"])},
            "higher_max_pct": tb["higher_max_pct"][0][1], "fewer_vortices_pct": tb["fewer_vortices_pct"][0][1],
            "fewer_given_higher_pct": tb["fewer_given_higher_pct"][1][0],
            "sweeps_mean": {"plain": mean(pl["sweeps"]), "annealed": mean(an["sweeps"])},
            "converged": {"plain": pl["converged"], "annealed": an["converged"]},
            "acceptance_mean": mean(an["acceptance"]),
            "data": "synthetic fields generated with torch on the GPU"}), flush=True)


def synth_w():
    from paper_0807_0264_gb300 import synth

    return synth.W_PLAQ_06


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def profile_kernels(mcg, U, dims, dev):
    """Each library kernel on the 20^3 x 40 workload field, for a per-kernel
    ncu capture (no timing here)."""
    Gi = mcg.identity_gauge(dims, 1, mcg.F64, dev)
    for eps, prec in ((1.0, mcg.F32), (1.0, mcg.F64), (-0.25, mcg.F64)):
        Us = mcg.mcg_convert(U, prec) if prec == mcg.F32 else U
        mcg.mcg_smear(Us, dims, 0.1, eps, 2)
    # the mixed fix: FP32 phase (compact conversion, half-sweeps, reductions),
    # hand-off, FP64 phase with the FP32 local solve; then the exact FP64 phase
    Uf, Gf = U.clone(), Gi.clone()
    mcg.mcg_fix(Uf, Gf, dims, mcg.Params(tol=-1e300, max_sweeps=4, check_every=2, reunit_every=2, fp32_sweeps=2,
                                         fp32_tol=-1e300, fp32_window=1, fp32_overrelax=OMEGA, fp64_solve32=1))
    mcg.mcg_fix(Uf, Gf, dims, mcg.Params(tol=-1e300, max_sweeps=2, check_every=2, reunit_every=2))
    mcg.mcg_fix(Uf, Gf, dims, mcg.Params(tol=-1e300, max_sweeps=2, check_every=2, fp64_df=1))
    mcg.mcg_apply_gauge(Uf, Gf, dims)
    mcg.mcg_reunitarise(Gf, 1, dims)
    mcg.mcg_plaquette(Uf, dims)
    mcg.mcg_functional(Uf, dims)
    Z, _ = mcg.mcg_center_project(Uf, dims)
    mcg.mcg_vortex_remove(Uf, Z, dims)
    mcg.mcg_wilson_loops(Uf, dims, 2, 2)
    mcg.mcg_anneal(Uf, Gf, dims, [1.0, 0.5], nhit=2, eps=0.3)
    mcg.mcg_grad_R(Uf, dims)
    Gout = torch_randn_like_links(U)
    mcg.mcg_smear_backward_step(U, Gout, dims, 0.1, 1.0)
    # a restart of the FP32 phase from a random gauge copy (random transform,
    # applied to the links, left-multiplied into the transform), and the local
    # solve on its own for one half-sweep's worth of problems, both precisions
    Ur, Gr = U.clone(), Gi.clone()
    mcg.mcg_fix(Ur, Gr, dims, mcg.Params(tol=-1e300, max_sweeps=6, check_every=2, fp32_sweeps=6, fp32_tol=-1e300,
                                         fp32_window=1, fp32_overrelax=OMEGA, fp32_restart=2,
                                         fp32_restart_domega=0.03, fp32_restart_random=1))
    import numpy as np
    import torch

    rng = np.random.default_rng(0)
    n = int(np.prod(dims)) // 2
    A = rng.standard_normal((n, 4, 4))
    A = torch.from_numpy(A + A.transpose(0, 2, 1)).to(dev)
    b = torch.from_numpy(rng.standard_normal((n, 4))).to(dev)
    for prec in (mcg.F64, mcg.F32):
        mcg.mcg_local_solve(A, b, prec)

    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_kernels": True, "dims": dims, "launches": mcg.mcg_kernel_launches()}), flush=True)


def torch_randn_like_links(U):
    import torch

    g = torch.Generator(device=U.device)
    g.manual_seed(0)
    return torch.randn(U.shape, dtype=U.dtype, device=U.device, generator=g)


def mixed_error_block(args, mcg, U, dims, levels, mixed, dev):
    """Error of the mixed schedule against the oracle, per level, on the
    preconditioned fix (the one that yields the level's fixed field): the
    level's preconditioned field (the smeared field, FP32 smearing as in the step, fixed with
    the mixed schedule; its transform applied to the input) runs the mixed
    schedule up to its hand-off and first FP64 sweep; from that same field
    H the GPU's FP64 finish (the bench's, local solve in FP32) and the GPU's
    exact FP64 finish run to dV_U < 1e-10, and so does the oracle's plain FP64
    relaxation on the host cores.  Reported: sweeps, V_U, |V_gpu - V_oracle|,
    max per-link |U_gpu - U_oracle|, P-vortex counts."""
    import numpy as np

    import oracle

    V = int(np.prod(dims))
    oracle.set_threads(len(os.sched_getaffinity(0)))
    handoff = mcg.Params(tol=1e300, max_sweeps=mixed.max_sweeps, check_every=mixed.check_every,
                         reunit_every=mixed.reunit_every, fp32_sweeps=mixed.fp32_sweeps, fp32_tol=mixed.fp32_tol,
                         fp32_window=mixed.fp32_window, fp32_overrelax=mixed.fp32_overrelax,
                         fp64_solve32=mixed.fp64_solve32, fp64_df=mixed.fp64_df, fp32_restart=mixed.fp32_restart,
                         fp32_restart_domega=mixed.fp32_restart_domega,
                         fp32_restart_random=mixed.fp32_restart_random,
                         fp32_restart_creep=mixed.fp32_restart_creep,
                         fp32_plain_finish=mixed.fp32_plain_finish)

    def compare(F):
        """F (device, FP64) -> hand-off H in place; finishes from H compared."""
        Gh = mcg.identity_gauge(dims, 1, mcg.F64, dev)
        h = mcg.mcg_fix(F, Gh, dims, handoff)
        H = mcg.mcg_unpack_links(F, dims)[0].cpu().numpy()
        row = {"handoff_sweeps": h["sweeps"][0]}
        finishes = (("gpu_bench_finish", dict(fp64_solve32=mixed.fp64_solve32, fp64_df=mixed.fp64_df)),
                    ("gpu_exact_finish", dict(fp64_solve32=0, fp64_df=0)))
        for name, kw in finishes:
            Ug, Gg = F.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
            rg = mcg.mcg_fix(Ug, Gg, dims, mcg.Params(tol=1e-10, max_sweeps=20000, check_every=25, reunit_every=50,
                                                      **kw))
            _, cnt = mcg.mcg_center_project(Ug, dims)
            row[name] = {"sweeps": rg["sweeps"][0], "converged": rg["converged"], "V": rg["R"][0] / (36.0 * V),
                         "vortices": int(cnt[0][0]), "U": mcg.mcg_unpack_links(Ug, dims)[0].cpu().numpy()}
            del Ug, Gg
        ro = oracle.fix(dims, H, None, tol=1e-10, max_sweeps=args.mixed_error_cap, reunit_every=50)
        Vo = ro["R_hist"][-1] / (36.0 * V)
        no = int(oracle.vortex_count(dims, oracle.center_project(dims, ro["U"]))[0])
        row["oracle_finish"] = {"sweeps": ro["sweeps"], "converged": ro["converged"], "V": Vo, "vortices": no}
        for name in ("gpu_bench_finish", "gpu_exact_finish"):
            r = row[name]
            Ug = r.pop("U")
            r["V_rel_err"] = abs(r["V"] - Vo) / Vo
            r["max_link_err"] = float(np.abs(Ug - ro["U"]).max())
            r["vortices_equal"] = r["vortices"] == no
        return row, Gh

    def smeared(n):
        """The step's smeared field of level n: FP32 smearing, back to FP64,
        re-unitarised (as mcg_precondition_levels does it)."""
        S = mcg.mcg_convert(mcg.mcg_smear(mcg.mcg_convert(U, mcg.F32), dims, args.rho, args.eps, n), mcg.F64)
        mcg.mcg_reunitarise(S, 0, dims)
        return S

    out = []
    for n in levels:
        t0 = time.perf_counter()
        row = {"level": n}
        Up = U.clone()
        if n > 0:
            row["smeared_fix"], _ = compare(smeared(n))
            # the preconditioning transform: the mixed fix of the smeared field
            S = smeared(n)
            G1 = mcg.identity_gauge(dims, 1, mcg.F64, dev)
            mcg.mcg_fix(S, G1, dims, mixed)
            mcg.mcg_reunitarise(G1, 1, dims)
            mcg.mcg_apply_gauge(Up, G1, dims)
            del S, G1
        row["preconditioned_fix"], _ = compare(Up)
        row["seconds"] = time.perf_counter() - t0
        out.append(row)
        del Up
    return {"method": "per level and per fix (the smeared field's, then the preconditioned field's): the mixed "
                      "schedule runs to its hand-off and first FP64 sweep (field H); from H the GPU's FP64 finish "
                      "(the bench's: double-float moves, local solve in FP32) and the GPU's exact FP64 finish run to dV_U<1e-10, and "
                      "so does the oracle's plain FP64 relaxation on the host cores; the step's FP32 smearing",
            "levels": out}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return

    from paper_0807_0264_gb300 import mcg, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.anneal:
        run_anneal(args, mcg, dev, rank)
        if dist:
            dist.destroy_process_group()
        return
    if args.gribov:
        run_gribov(args, mcg, dev, rank)
        if dist:
            dist.destroy_process_group()
        return
    dims = tuple(args.dims)
    V = 1
    for d in dims:
        V *= d
    levels = list(args.levels)
    # each rank is an independent replica on its own synthetic field
    if args.vortex_sheets:
        U_host, _ = synth.make_vortex_field(dims, synth.W_VORTEX_06, rank, synth.VORTEX_PAIRS_20x40)
    else:
        U_host = synth.make_field(dims, synth.W_PLAQ_06, rank)
    canon_pinned = torch.from_numpy(U_host).unsqueeze(0).pin_memory()
    canon_dev = canon_pinned.to(dev)
    U = mcg.mcg_pack_links(canon_dev, dims, mcg.F64)
    nl = len(levels)
    U_out = mcg.empty_links(dims, nl, mcg.F64, dev)
    G_out = mcg.empty_gauge(dims, nl, mcg.F64, dev)
    Z_out = torch.empty((nl, 4, 2, V // 2), dtype=torch.int8, device=dev)
    def warm_field(sweeps=300):
        """The input field after `sweeps` over-relaxed FP32 sweeps (handed off
        to FP64): the regime the FP32 phase spends its sweeps in."""
        Uw, Gw = U.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
        mcg.mcg_fix(Uw, Gw, dims, mcg.Params(tol=-1e300, max_sweeps=sweeps, check_every=25, fp32_sweeps=sweeps,
                                             fp32_tol=-1e300, fp32_window=25, fp32_overrelax=OMEGA))
        return Uw

    if args.profile_kernel:
        prec = mcg.F32 if args.profile_kernel == "f32" else mcg.F64
        Uw = warm_field()
        Ut = mcg.mcg_convert(Uw, mcg.F32) if prec == mcg.F32 else Uw
        Gt = mcg.identity_gauge(dims, 1, prec, dev)
        mcg.mcg_set_sweep_block(prec, 128)
        ms = {p: mcg.mcg_time_halfsweep(Ut, Gt, dims, parity=p, nreps=3, flush_l2=True) for p in (1, 0)}
        print(json.dumps({"profile_kernel": args.profile_kernel, "dims": dims, "ms_per_launch": ms}), flush=True)
        return

    if args.probe_peaks:
        print(json.dumps({"probe_peaks": mcg.mcg_probe_peaks(), "hbm_gbs": hbm_peak()[0]}), flush=True)
        return

    if args.profile_kernels:
        profile_kernels(mcg, U, dims, dev)
        return

    if args.slabs:
        run_slabs(mcg, dims, U_host, dev)
        return

    if args.profile_slice:
        # FP32 : FP64 sweeps 100 : 1 per fix, close to the full step's ratio
        sl = mcg.Params(tol=-1e300, max_sweeps=101, check_every=25, reunit_every=50, fp32_sweeps=100,
                        fp32_tol=-1e300, fp32_window=25, fp32_overrelax=OMEGA, fp64_solve32=1, fp64_df=1)
        mcg.mcg_set_sweep_block(mcg.F32, 128)
        mcg.mcg_set_sweep_block(mcg.F64, 128)
        torch.cuda.synchronize(dev)
        n0 = mcg.mcg_kernel_launches()
        res = mcg.mcg_precondition_levels(U, dims, [0, 4], sl, rho=RHO, eps=1.0, smear_precision=mcg.F32)[3]
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_slice": True, "launches": mcg.mcg_kernel_launches() - n0,
                          "sweeps": [r["sweeps_smeared"] + r["sweeps_fixed"] for r in res]}), flush=True)
        return

    U_warm = warm_field()
    tuned = {"f32": mcg.autotune_sweep_block(mcg.mcg_convert(U_warm, mcg.F32), dims),
             "f64": mcg.autotune_sweep_block(U_warm.clone(), dims, reps=3)}
    mixed = mcg.Params(tol=1e-10, max_sweeps=30000, check_every=25, reunit_every=50, fp32_sweeps=30000,
                       fp32_tol=float(os.environ.get("MCG_FP32_TOL", "5e-11")), fp32_window=25,
                       fp32_overrelax=OMEGA, fp64_solve32=1, fp64_df=int(os.environ.get("MCG_FP64_DF", "1")),
                       fp32_restart=RESTART, fp32_restart_domega=RESTART_DOMEGA,
                       fp32_restart_random=RESTART_RANDOM, fp32_restart_creep=RESTART_CREEP,
                       fp32_plain_finish=PLAIN_FINISH)
    stream = torch.cuda.current_stream(dev)

    def step(params, smear_prec):
        return mcg.mcg_precondition_levels(U, dims, levels, params, rho=args.rho, eps=args.eps,
                                           smear_precision=smear_prec, U_out=U_out, G_out=G_out, Z_out=Z_out)[3]

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x: float) -> float:
        return reduce_over_ranks(dist, x, "max", dev)

    def sum_over_ranks(x: float) -> float:
        return reduce_over_ranks(dist, x, "sum", dev)

    for _ in range(args.warmup):
        res = step(mixed, mcg.F32)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = mcg.mcg_kernel_launches()
    mcg.mcg_phase_stats(reset=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        site_updates = 0
        for _ in range(args.steps):
            res = step(mixed, mcg.F32)
            site_updates += sum(r["sweeps_smeared"] + r["sweeps_fixed"] for r in res) * V
        e1.record(stream)
        barrier()
    launches = mcg.mcg_kernel_launches() - launches0
    phases = mcg.mcg_phase_stats(reset=True)
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    ms = ms_total / args.steps
    total_updates = sum_over_ranks(site_updates)
    value = total_updates / (ms_total / 1e3)
    mixed_res = res
    sw32 = sum(r["sweeps_fp32"] for r in res)
    sw_all = sum(r["sweeps_smeared"] + r["sweeps_fixed"] for r in res)

    # plain FP64 comparison (the paper's relaxation, FP64 throughout) on the
    # unpreconditioned level: it is capped, because on this field it creeps
    # (dV_U ~ 5e-10 per sweep for 1e4+ sweeps); the mixed form is timed on the
    # same single fix for a like-for-like ratio
    plain_info = None
    if not args.no_plain:
        cap = int(os.environ.get("MCG_PLAIN_CAP", "4000"))
        one = mcg.Params(tol=1e-10, max_sweeps=cap, check_every=50, reunit_every=50)
        Up = U.clone()
        Gp = mcg.identity_gauge(dims, 1, mcg.F64, dev)
        barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pr = mcg.mcg_fix(Up, Gp, dims, one, history=True)
        p1.record(stream)
        barrier()
        pms = max_over_ranks(p0.elapsed_time(p1))
        import numpy as np

        h = pr["R_hist"][0] / (36.0 * V)
        d = np.diff(h)
        info = {"level": 0, "cap_sweeps": cap, "sweeps": pr["sweeps"][0], "converged": pr["converged"],
                "ms": pms, "ms_per_sweep": pms / max(1, pr["sweeps"][0]), "V": float(h[-1]),
                "dV_last": float(d[-1]) if len(d) else None}
        if not pr["converged"] and len(d) > 1000 and d[-1] > 0:
            # dV_U(k) ~ C exp(-k / tau) fitted over the last 1000 sweeps
            k = np.arange(len(d) - 1000, len(d))
            sl = np.polyfit(k, np.log(np.maximum(d[-1000:], 1e-300)), 1)[0]
            if sl < 0:
                tau = -1.0 / sl
                extra = tau * np.log(d[-1] / 1e-10)
                info["fit_tau_sweeps"] = float(tau)
                info["extrapolated_sweeps_to_tol"] = float(len(d) + max(0.0, extra))
                info["extrapolated_ms_to_converged"] = float(info["extrapolated_sweeps_to_tol"] * info["ms_per_sweep"])
        Um = U.clone()
        Gm = mcg.identity_gauge(dims, 1, mcg.F64, dev)
        barrier()
        p0.record(stream)
        mr = mcg.mcg_fix(Um, Gm, dims, mixed)
        p1.record(stream)
        barrier()
        mms = max_over_ranks(p0.elapsed_time(p1))
        info["mixed_same_fix"] = {"ms": mms, "sweeps": mr["sweeps"][0], "converged": mr["converged"],
                                  "V": mr["R"][0] / (36.0 * V)}
        info["speedup_lower_bound"] = pms / mms if mr["converged"] else None
        if "extrapolated_ms_to_converged" in info and mr["converged"]:
            info["speedup_extrapolated"] = info["extrapolated_ms_to_converged"] / mms
        if pr["converged"] and mr["converged"]:
            info["speedup"] = pms / mms
        plain_info = info
        del Up, Gp, Um, Gm

    # dominant kernel: per-launch durations of the FP32 and FP64 half-sweep,
    # L2 flushed between launches, on a scratch copy of the field after 300
    # FP32 sweeps (the regime the FP32 phase spends its sweeps in)
    Uc = U_warm
    Gc = mcg.identity_gauge(dims, 1, mcg.F64, dev)
    U32 = mcg.mcg_convert(Uc, mcg.F32)
    G32 = mcg.identity_gauge(dims, 1, mcg.F32, dev)
    t32 = mcg.mcg_time_halfsweep(U32, G32, dims, parity=1, nreps=20, flush_l2=True)
    t32_even = mcg.mcg_time_halfsweep(U32, G32, dims, parity=0, nreps=20, flush_l2=True)
    t64 = mcg.mcg_time_halfsweep(Uc, Gc, dims, parity=1, nreps=5, flush_l2=True)
    del Uc, Gc, U32, G32
    vh = V // 2
    bytes32 = vh * (8 * 48 * 2 + 48 * 2)  # 8 links + W read and written, FP32 rows 0 and 1
    same_src = fp32_kernel_fingerprint().startswith(TRAFFIC_FP32["source_sha256_prefix"])
    peak, peak_src = hbm_peak()
    # the dominant kernel inside the timed region: the FP32 sweep graphs
    # (half-sweeps + end-of-sweep reduction), CUDA events around each graph
    # launch in the library, site-updates from the fields' sweep counts
    p32, p64 = phases["f32"], phases["f64"]
    achieved = p32["site_updates"] * 864 / (p32["ms"] / 1e3) / 1e9 if p32["ms"] > 0 else 0.0
    roof = {"bound": "hbm", "kernel": "k_halfsweep_c12", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": TRAFFIC_FP32["bytes_per_launch"] if same_src else None,
            "traffic_source": TRAFFIC_FP32["profile"] if same_src else "kernel changed since the capture",
            "traffic_launch": "one 20^3 x 40 half-sweep (160 000 site-updates, 138.24 MB algorithmic)",
            "algorithmic_bytes_per_site_update": 864, "peak_source": peak_src,
            "method": "live in the timed region: FP32 sweep-graph GPU time (CUDA events in the library around "
                      "each graph launch; the end-of-sweep reduction kernel included) over the FP32 site-updates "
                      "x 864 B",
            "timed_region": {"fp32_ms": p32["ms"], "fp32_site_updates": p32["site_updates"],
                             "fp64_ms": p64["ms"], "fp64_site_updates": p64["site_updates"],
                             "fp64_ms_per_field_sweep": p64["ms"] / max(1e-9, p64["site_updates"] / V),
                             "fp32_ms_per_field_sweep": p32["ms"] / max(1e-9, p32["site_updates"] / V),
                             "share_of_step": {"fp32": p32["ms"] / ms_total, "fp64": p64["ms"] / ms_total}},
            "isolated": {"ms_per_launch": (t32 + t32_even) / 2,
                         "achieved": bytes32 / ((t32 + t32_even) / 2 / 1e3) / 1e9,
                         "frac": bytes32 / ((t32 + t32_even) / 2 / 1e3) / 1e9 / peak,
                         "method": "one 20^3 x 40 field, mean of the odd and even half-sweep, L2 flushed by a "
                                   "256 MB memset before each launch"}}
    roof["kernel_ms"] = {"fp32_odd": t32, "fp32_even": t32_even, "fp64_odd_exact_solve": t64}
    # the same kernel inside a fix (no flush: each half-sweep's 138 MB working
    # set exceeds the 129 MB L2): FP32-phase time of N2 - N1 sweeps on a copy
    # of the warm field, both half-sweeps and the end-of-sweep kernel per sweep
    def fp32_phase_ms(n):
        Ui, Gi = U_warm.clone(), mcg.identity_gauge(dims, 1, mcg.F64, dev)
        pr_ = mcg.Params(tol=1e300, max_sweeps=n + 1, check_every=25, fp32_sweeps=n, fp32_tol=-1e300,
                         fp32_window=25, fp32_overrelax=OMEGA)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        mcg.mcg_fix(Ui, Gi, dims, pr_)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        return a0.elapsed_time(a1)
    n1, n2 = 100, 500
    fp32_phase_ms(n1)
    sweep_ms = (fp32_phase_ms(n2) - fp32_phase_ms(n1)) / (n2 - n1)
    roof["in_situ"] = {"ms_per_sweep": sweep_ms, "ms_per_launch": sweep_ms / 2,
                       "achieved": 2 * bytes32 / (sweep_ms / 1e3) / 1e9, "unit": "GB/s",
                       "frac": 2 * bytes32 / (sweep_ms / 1e3) / 1e9 / peak,
                       "method": "FP32 sweeps inside a fix, L2 not flushed (working set 138 MB > 129 MB L2); the "
                                 "end-of-sweep kernel counted in the sweep"}

    # Sec. III.A on the level-0 result: center decomposition (vortex-removed
    # and vortex-only fields) and on-axis Wilson loops of the three fields
    sec3d = None
    if not args.no_observables:
        Uf, Zf = U_out[0:1], Z_out[0:1]
        RT = (8, 8)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q2 = torch.cuda.Event(enable_timing=True)
        mcg.mcg_vortex_remove(Uf, Zf, dims)  # warm-up (scratch, module load)
        q0.record(stream)
        Ur, Zl = mcg.mcg_vortex_remove(Uf, Zf, dims)
        q1.record(stream)
        Ws = {name: mcg.mcg_wilson_loops(F, dims, *RT)[0] for name, F in
              (("full", Uf), ("vortex_removed", Ur), ("vortex_only", Zl))}
        q2.record(stream)
        offaxis = [(1, 1, 0), (2, 1, 0), (2, 2, 0), (1, 1, 1), (2, 1, 1), (2, 2, 1)]
        Wo = mcg.mcg_wilson_loops_offaxis(Uf, dims, offaxis, RT[1])[0]
        q3 = torch.cuda.Event(enable_timing=True)
        q3.record(stream)
        torch.cuda.synchronize(dev)
        vr_ms = q0.elapsed_time(q1)
        vr_bytes = 3 * V * 4 * 144 + V * 4  # read U and Z, write U' and Z (FP64 links)
        sec3d = {"field": "level 0 fixed field", "vortex_remove_ms": vr_ms,
                 "vortex_remove_GBps": vr_bytes / (vr_ms / 1e3) / 1e9,
                 "wilson_ms_3_fields": q1.elapsed_time(q2), "Rmax": RT[0], "Tmax": RT[1],
                 "W_RxT_diag": {k: [float(w[i, i]) for i in range(RT[0])] for k, w in Ws.items()},
                 "offaxis_vectors": offaxis, "offaxis_ms": q2.elapsed_time(q3),
                 "W_offaxis_T4": [float(Wo[v, 3]) for v in range(len(offaxis))]}
        del Ur, Zl

    # end to end through the public API: host canonical field in, results out.
    # Every step uploads its input field and reads back every level's center
    # sectors and gauge transform; the copies run on a copy stream with double
    # buffers, so step k's read-back and step k+1's upload overlap the compute
    # (the step itself synchronises on its own stream)
    barrier()
    copy_stream = torch.cuda.Stream(dev)
    canon_bufs = [canon_dev, torch.empty_like(canon_dev)]
    outs = [(U_out, G_out, Z_out), (mcg.empty_links(dims, nl, mcg.F64, dev), mcg.empty_gauge(dims, nl, mcg.F64, dev),
                                    torch.empty_like(Z_out))]
    z_hosts = [torch.empty((nl, V, 4), dtype=torch.int8).pin_memory() for _ in range(2)]
    g_hosts = [torch.empty(G_out.shape, dtype=G_out.dtype).pin_memory() for _ in range(2)]  # each level's Omega
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [None, None]
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    copy_stream.wait_event(h0)
    with torch.cuda.stream(copy_stream):
        canon_bufs[0].copy_(canon_pinned, non_blocking=True)
        ev_in[0].record(copy_stream)
    e2e_updates = 0
    for i in range(args.steps):
        b = i % 2
        stream.wait_event(ev_in[b])
        if i + 1 < args.steps:
            with torch.cuda.stream(copy_stream):
                canon_bufs[1 - b].copy_(canon_pinned, non_blocking=True)
                ev_in[1 - b].record(copy_stream)
        if ev_out[b] is not None:
            stream.wait_event(ev_out[b])  # step i-2's read-back of these outputs
        Ue = mcg.mcg_pack_links(canon_bufs[b], dims, mcg.F64)
        Uo, Go, Zo = outs[b]
        r2 = mcg.mcg_precondition_levels(Ue, dims, levels, mixed, rho=args.rho, eps=args.eps,
                                         smear_precision=mcg.F32, U_out=Uo, G_out=Go, Z_out=Zo)[3]
        Zc = mcg.mcg_unpack_center(Zo, dims)
        ready = torch.cuda.Event()
        ready.record(stream)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            z_hosts[b].copy_(Zc, non_blocking=True)
            g_hosts[b].copy_(Go, non_blocking=True)
            ev_out[b] = torch.cuda.Event()
            ev_out[b].record(copy_stream)
        Zc.record_stream(copy_stream)
        e2e_updates += sum(r["sweeps_smeared"] + r["sweeps_fixed"] for r in r2) * V
    stream.wait_stream(copy_stream)
    h1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(h0.elapsed_time(h1))
    e2e_value = sum_over_ranks(e2e_updates) / (e2e_ms / 1e3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, n, cores = oracle_sample(U_host, dims, args.cpu_seconds)
        v1, n1, _ = oracle_sample(U_host, dims, max(2.0, args.cpu_seconds / 4), threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} oracle FP64 MCG sweeps of the {dims[0]}x{dims[1]}x{dims[2]}x{dims[3]} workload field",
               "one_core": {"value": v1, "sample": f"{n1} sweeps on 1 thread"}}

    pipes = mcg.mcg_probe_peaks()  # after the timed region: denominators of the ALU-bound kernels
    mixed_err = None
    if rank == 0 and world == 1 and not args.no_mixed_error:
        mixed_err = mixed_error_block(args, mcg, U, dims, args.mixed_error_levels or levels, mixed, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": config_of(args, f"batched levels, FP32 smearing, FP32 sweeps (over-relaxed, omega="
                                          f"{mixed.fp32_overrelax}, until the 25-sweep mean dV_U < "
                                          f"{mixed.fp32_tol:g}; a field still running after "
                                          f"{mixed.fp32_restart} sweeps, or creeping for "
                                          f"{mixed.fp32_restart_creep}, restarts from "
                                          + ("a random gauge copy of " if mixed.fp32_restart_random else "")
                                          + f"its input with omega -+ k*"
                                          f"{mixed.fp32_restart_domega:g}"
                                          + ("; then plain FP32 sweeps to the same criterion" if mixed.fp32_plain_finish
                                             else "")
                                          + ") then FP64-class plain relaxation ("
                                          + ("double-float moves, local 4x4 solve in FP32, transform applied in "
                                             "FP64" if mixed.fp64_df else
                                             "local 4x4 solve in FP32, G normalised and applied in FP64")
                                          + ") to dV_U<1e-10 in FP64"),
                "ttc": {"mixed_ms_to_converged": ms, "plain_fp64": plain_info,
                        "sweeps": sw_all, "sweeps_fp32": sw32,
                        "V_fixed": [r["V_fixed"] for r in mixed_res],
                        "V_smeared": [r["V_smeared"] for r in mixed_res],
                        "vortex_density": [r["vortex_density"] for r in mixed_res],
                        "plaquette_in": mixed_res[0]["plaquette_in"],
                        "plaquette_out": [r["plaquette_out"] for r in mixed_res],
                        "converged": all(r["status"] == 0 for r in mixed_res),
                        "per_level": [{"n_smear": n, "sweeps_smeared": r["sweeps_smeared"],
                                       "sweeps_fixed": r["sweeps_fixed"], "sweeps_fp32": r["sweeps_fp32"],
                                       "fp32_restarts": r["fp32_restarts"],
                                       "converged": r["status"] == 0} for n, r in zip(levels, mixed_res)]},
                "roofline": roof, "cpu_baseline": cpu, "autotune": tuned,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": canon_pinned.numel() * 16,
                        "d2h_bytes_per_step": z_hosts[0].numel() + g_hosts[0].numel() * g_hosts[0].element_size(),
                        "d2h": "center sectors and gauge transform of every level",
                        "copies": "pinned host buffers, a copy stream and double device buffers: a step's read-back "
                                  "and the next step's upload overlap the compute",
                        "ms_per_step": e2e_ms / args.steps},
                "clocks": clk.summary(), "gpu_launches": launches, "sec3d": sec3d, "mixed_error": mixed_err,
                "measured_pipes": pipes}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
