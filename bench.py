"""Benchmark of the fused chi^2 + gradient evaluation.

Default workload: reactor8_1000x16384 -- 1000 bins in 0.5-15 MeV x 16384
Gauss-Legendre nodes x 8 baselines (131,072,000 probability evaluations per
step), parameters perturbed by +-5 %, Poisson chi^2, per-baseline spectra and
the four-parameter gradient.  One step = one evaluation of the whole chain
(parameter prep, fused phase/probability/weight/bin-sum kernel, chi^2 and
gradient epilogue) in the double-float-phase mixed precision.

Prints one JSON line (rank 0).  Under torchrun every rank evaluates its own
replica (its own pseudo-data seed): units are independent, there is no
data-path collective, and the timing is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1804_07682_gb300 import workloads as wl  # noqa: E402

METRIC = "χ²+grad evals/s and Gpoints/s vs plain FP64 GPU chain at ≤1e-6 rel err; % roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 issue peak: 152 SMs x 128 FP32 lanes per clock x 2070 MHz (maximum SM clock)
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def fp32_ops_general(nL: int, grad: bool, surv: bool) -> int:
    """Algorithmic FP32 operations per energy node of the any-channel node
    kernel: per (node, baseline) the phases reduced modulo pi and their
    sin/cos 38, angle addition 4, sin^2, sin cos and cos^2 of three phases 9,
    their weighted sums over the baselines 9 (18 with hi + lo weights for
    several baselines; none for one baseline, whose weight is exactly 1),
    with the gradient cos^2 - sin^2 3 and two more weighted sums per phase 6;
    per node the Kahan product-sums of 9 (15) values, 4 each.  Survival
    channels (alpha = beta) reduce the phases modulo pi/2 instead (11 each)
    with quadrant swaps (3 each): 10 more per (node, baseline)."""
    per_r = 51 + (18 if nL > 1 else 0) + (9 if grad else 0) + (10 if surv else 0)
    return nL * per_r + (60 if grad else 36)


def fp32_ops_per_node(nL: int, grad: bool, spec: bool) -> int:
    """Algorithmic FP32 operations (FMA = 1) of the fused kernel per energy node.

    Per (node, baseline): double-float phase and two-part reduction mod pi
    2 x 9, sin/cos polynomials 2 x 10 (u = r^2, degree-9 sine 5, degree-8
    cosine 4), angle addition 2, three squares, three weighted sums
    (38 + 2 + 3 + 3 = 46; 43 for one baseline, whose weight is exactly 1
    and needs no sums);
    with one or more baselines and no per-baseline sums the weights enter as
    hi + lo (3 more); gradient: cos of the sum 2, three sin*cos products and
    three weighted sums (8); spectra: P_r 3 + Kahan product-sum 4 (7).  Per
    node: combined P with hi + lo amplitudes 7 (+3 for hi + lo weights) and its
    Kahan product-sum 4; gradient: tangent combinations 10 + four Kahan
    product-sums 16.
    """
    omlo = nL > 1 and not spec
    per_r = (46 if nL > 1 else 43) + (3 if omlo else 0) + (8 if grad else 0) + (7 if spec else 0)
    per_node = 11 + (3 if omlo else 0) + (26 if grad else 0)
    return nL * per_r + per_node


# DRAM traffic of one launch of the benchmarked kernels from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), per mapping, valid only for
# the kernel sources it was taken with: reported as null once they change.
PROFILE_EVERY = 8
TRAFFIC_CAPTURE = {
    "split": {"sources_sha256": "4e84d90634a932986bddfc3627e81e2c61c0ee248b37d8a2b42cd44e71396f94",
              "bytes": 265113600 + 4114176},
    "slices": {"sources_sha256": "ee1c2edc308edbe2ecc5ca374d8666315fc1bb510abdc327df76998aaec7e7e2",
               "bytes": 268506880 + 4611584 + 8178176 + 0},
}
KERNEL_SOURCES = ["paper_1804_07682_gb300/csrc/common.cuh", "paper_1804_07682_gb300/csrc/fused.cuh",
                  "paper_1804_07682_gb300/csrc/epilogue.cuh", "paper_1804_07682_gb300/csrc/ff_consts.h",
                  "paper_1804_07682_gb300/csrc/slices.cu"]
KERNEL_NAMES = {"split": "k_fused_split", "slices": "k_fused_bins (slices) + k_slices_reduce",
                "bins": "k_fused_bins"}


def kernel_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        # the raw samples go to $BENCH_CLOCKS_DIR (if set) or the temporary directory
        import tempfile

        d = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, "bench_clocks_%d_%d.csv" % (index, os.getpid()))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() in ("active", "1")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend=backend)
        return dist
    return None


def reduce_max(dist, x, device):
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base: int, rank: int) -> int:
    """Pseudo-data seed of one replica: every rank fits its own Poisson draw."""
    return base + 1000 * rank


def replica_throughput(dist, ms_local: float, units_per_rank: float, world: int, device):
    """Whole-job throughput of independent replicas: the units all ranks
    processed divided by the slowest rank's time.  Returns (ms, units/s)."""
    ms = reduce_max(dist, ms_local, device)
    return ms, world * units_per_rank / (ms / 1e3)


# --------------------------------------------------------------- reference arm --
def reference_arm(args):
    """The oracle, as it stands, timed on the host cores.  Each step evaluates
    a bounded sample of the workload (a number of whole bins, every node and
    baseline, with the gradient) sized so that warm-up + timed steps take about
    a minute; the rate is scaled to one full evaluation."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle

    if world > 1:
        # the other ranks exit at once; the launcher's one-thread default is
        # for N busy ranks, so this rank takes every host core
        oracle.set_threads(os.cpu_count() or 1)

    w = wl.ALL[args.workload]()
    N = 1.0
    th = w.theta[0]

    def run(nb):
        return oracle.chain(w.edges[: nb + 1], w.nodes_per_bin, w.L, th, N, np.full(nb, 100.0), w.kind,
                            e_scale=w.e_scale)

    # per-bin time after the Gauss-Legendre rule is cached, on enough bins
    # that every host core has work ((baseline, bin) pairs are the oracle's
    # parallel loop); the sample keeps warm-up + timed steps near 90 s and
    # never drops below that many bins, so per-call overhead stays small
    nb_min = int(min(w.nbins, max(8, -(-2 * oracle.threads() // w.nL))))
    run(nb_min)
    t0 = time.perf_counter()
    run(nb_min)
    t_bin = max((time.perf_counter() - t0) / nb_min, 1e-6)
    budget = 90.0 / max(1, args.steps + args.warmup)
    nb = int(max(nb_min, min(w.nbins, budget / t_bin)))
    for _ in range(args.warmup):
        run(nb)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(nb)
    dt = (time.perf_counter() - t0) / args.steps
    frac = nb / w.nbins
    evals = frac / dt
    sample = "%d of %d bins per step (x%d nodes x%d baselines, with gradient), scaled to one full evaluation" % (
        nb, w.nbins, w.nodes_per_bin, w.nL)
    line = {"impl": "reference", "metric": METRIC, "value": evals, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / frac, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "bins": w.nbins, "nodes_per_bin": w.nodes_per_bin, "baselines": w.nL,
                       "points_per_eval": w.points_per_eval(), "bins_per_step": nb},
            "gpoints_per_s": evals * w.points_per_eval() / 1e9,
            "cpu_baseline": {"value": evals, "unit": "evals/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": evals, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- side workloads --
def side_workloads(api, torch, device, args):
    """The other workloads, each timed on its own after the main timed region:
    the 64 x 64 scan (4096 points, uneven grids, one graph-replayed launch),
    the same scan for nu_mu -> nu_e through the any-channel chain, the 16384
    pseudo-experiment fits (20 Levenberg-Marquardt iterations), the 10^4-node
    reactor chain, the differentiable chi^2 with 1000 nuisances, OscProb
    alone at the paper's Table 1 sizes (device, copies, staged, in place),
    OscProb for any channel, and the device pseudo-data.  Returns the results
    and the outputs the CPU-baseline leg checks against the oracle."""
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    # scan
    w = wl.scan_64x64_500bins()
    plan = api.Plan(w.edges, w.L, npts=w.npts, node_counts=w.node_counts, norm=1.0, e_scale=w.e_scale, prec=args.prec,
                    kind=w.kind)
    p = plan.params_tensor(w.theta)
    truth = plan.params_tensor(np.repeat(np.array(wl.TRUTH)[None, :], w.npts, axis=0))
    dummy = torch.ones(w.nbins, dtype=torch.float64, device=device)
    m = plan.eval(truth, dummy, grad=False, mu=True)["mu"][int(np.argmax(w.node_counts))]
    N = wl.TOTAL_EVENTS / float(m.sum())
    plan.close()
    plan = api.Plan(w.edges, w.L, npts=w.npts, node_counts=w.node_counts, norm=N, e_scale=w.e_scale, prec=args.prec,
                    kind=w.kind)
    data = torch.as_tensor(wl.poisson_data((m * N).cpu().numpy(), w.data_seed), device=device)
    plan.autotune(p, data, reps=3)
    plan.set_graph(True)
    o = {"chi2": torch.empty(w.npts, dtype=torch.float64, device=device),
         "grad": torch.empty(w.npts, 4, dtype=torch.float64, device=device)}
    for _ in range(3):
        plan.eval(p, data, grad=True, out=o)
    reps = 20
    torch.cuda.synchronize()
    plan.profile(False)
    a0, a1 = ev(), ev()
    a0.record(stream)
    for _ in range(reps):
        plan.eval(p, data, grad=True, out=o)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / reps
    pts = w.points_per_eval()
    ops = sum(fp32_ops_per_node(1, True, False) * w.nbins * int(n) for n in w.node_counts)
    check = {"scan": (w, N, data.cpu().numpy(), o["chi2"].cpu().numpy(), o["grad"].cpu().numpy())}
    out["scan_64x64_500bins"] = {"scans_per_s": 1e3 / ms, "ms_per_scan": ms, "chi2_grad_evals_per_s": w.npts * 1e3 / ms,
                                 "gpoints_per_s": pts / ms / 1e6, "points_per_scan": pts,
                                 "fp32_frac_of_issue_peak": ops / (ms * 1e-3) / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6),
                                 "tuning": plan.tuning, "graph": True}
    plan.close()
    # the same scan, chi^2 and gradient of all 4096 points, through the plain
    # FP64 chain (one kernel per transformation, points in chunks) and through
    # the all-double fused kernel; errors of the timed mixed path against them
    fp64 = {}
    for name, prec, plain in (("plain_fp64_chain", args.prec, True), ("fused_fp64", "fp64", False)):
        pl = api.Plan(w.edges, w.L, npts=w.npts, node_counts=w.node_counts, norm=N, e_scale=w.e_scale, prec=prec,
                      kind=w.kind, with_plain=plain)
        q = pl.params_tensor(w.theta)
        r = pl.eval(q, data, grad=True, plain=plain)
        torch.cuda.synchronize()
        n_rep = 3
        a0, a1 = ev(), ev()
        a0.record(stream)
        for _ in range(n_rep):
            pl.eval(q, data, grad=True, plain=plain, out=r)
        a1.record(stream)
        torch.cuda.synchronize()
        pl.status()
        ms64 = a0.elapsed_time(a1) / n_rep
        fp64[name] = {"ms_per_scan": ms64, "chi2_grad_evals_per_s": w.npts * 1e3 / ms64, "launches": pl.launches}
        c_ref, g_ref = r["chi2"].cpu().numpy(), r["grad"].cpu().numpy()
        c_mix, g_mix = check["scan"][3], check["scan"][4]
        fp64[name]["mixed_max_rel_err"] = {
            "chi2": float(np.max(np.abs(c_mix - c_ref) / np.abs(c_ref))),
            "grad_normwise": float(np.max(np.linalg.norm(g_mix - g_ref, axis=1) / np.linalg.norm(g_ref, axis=1)))}
        pl.close()
    out["scan_64x64_500bins"]["fp64_gpu"] = fp64
    # the same scan for nu_mu -> nu_e appearance through the any-channel chain:
    # (s2_13, dm2_32) on the same uneven grids, s2_23 = 0.545 and delta = 1.2 pi,
    # chi^2 and its gradient in all six parameters
    def six(t):
        t = np.atleast_2d(t)
        k = t.shape[0]
        return np.column_stack([t[:, 0], t[:, 1], np.full(k, 0.545), np.full(k, 1.2 * np.pi), t[:, 2], t[:, 3]])

    gkw = dict(npts=w.npts, node_counts=w.node_counts, e_scale=w.e_scale, prec=args.prec, kind=w.kind,
               channel=("mu", "e", False))
    plan = api.Plan(w.edges, w.L, norm=1.0, **gkw)
    m = plan.eval_general(plan.params_tensor(six(np.repeat(np.array(wl.TRUTH)[None, :], w.npts, axis=0))), dummy,
                          grad=False, mu=True)["mu"][int(np.argmax(w.node_counts))]
    Ng = wl.TOTAL_EVENTS / float(m.sum())
    plan.close()
    plan = api.Plan(w.edges, w.L, norm=Ng, **gkw)
    th6 = six(w.theta)
    pg = plan.params_tensor(th6)
    datag = torch.as_tensor(wl.poisson_data((m * Ng).cpu().numpy(), w.data_seed), device=device)
    plan.autotune(pg, datag, reps=3)
    og = {"chi2": torch.empty(w.npts, dtype=torch.float64, device=device),
          "grad": torch.empty(w.npts, 6, dtype=torch.float64, device=device)}
    for _ in range(3):
        plan.eval_general(pg, datag, grad=True, out=og)
    torch.cuda.synchronize()
    a0, a1 = ev(), ev()
    a0.record(stream)
    for _ in range(reps):
        plan.eval_general(pg, datag, grad=True, out=og)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / reps
    ops = sum(fp32_ops_general(1, True, False) * w.nbins * int(n) for n in w.node_counts)  # appearance
    check["scan_numu_nue"] = (w, Ng, datag.cpu().numpy(), og["chi2"].cpu().numpy(), og["grad"].cpu().numpy(), th6)
    out["scan_64x64_500bins_numu_nue"] = {
        "scans_per_s": 1e3 / ms, "ms_per_scan": ms, "chi2_grad_evals_per_s": w.npts * 1e3 / ms,
        "gpoints_per_s": pts / ms / 1e6,
        "fp32_frac_of_issue_peak": ops / (ms * 1e-3) / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6),
        "outputs": "chi2, d chi2 / d(s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32)", "tuning": plan.tuning}
    plan.close()
    # fits
    w = wl.fits_16384x1000()
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, npts=1, norm=1.0, prec=args.prec, kind=w.kind)
    m = plan.eval(plan.params_tensor(w.truth), torch.ones(w.nbins, dtype=torch.float64, device=device), grad=False,
                  mu=True)["mu"][0]
    N = wl.TOTAL_EVENTS / float(m.sum())
    plan.close()
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, npts=w.npts, norm=N, prec=args.prec, kind=w.kind,
                    max_datasets=w.npts)
    data = torch.as_tensor(wl.pseudo_datasets((m * N).cpu().numpy(), w.n_datasets, w.data_seed), device=device)
    p0 = plan.params_tensor(w.theta)
    p = p0.clone()
    plan.autotune(p, data, reps=1)
    c2 = torch.empty(w.npts, dtype=torch.float64, device=device)
    p.copy_(p0)
    plan.fit(p, data, iters=2, graph=True, chi2_out=c2)
    torch.cuda.synchronize()
    p.copy_(p0)
    a0, a1 = ev(), ev()
    a0.record(stream)
    plan.fit(p, data, iters=w.fit_iters, graph=True, chi2_out=c2)
    a1.record(stream)
    torch.cuda.synchronize()
    plan.status()
    ms = a0.elapsed_time(a1)
    pts = w.points_per_eval() * w.fit_iters
    check["fits"] = (w, N, data[0].cpu().numpy(), p[0].cpu().numpy(), c2[0].item())
    ops = fp32_ops_per_node(w.nL, True, False) * w.nbins * w.nodes_per_bin * w.npts * w.fit_iters
    out["fits_16384x1000"] = {"fits_per_s": w.npts * 1e3 / ms, "ms_per_batch": ms, "iterations": w.fit_iters,
                              "chi2_grad_evals_per_s": w.npts * w.fit_iters * 1e3 / ms, "gpoints_per_s": pts / ms / 1e6,
                              "fp32_frac_of_issue_peak": ops / (ms * 1e-3) / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6),
                              "median_best_chi2": float(c2.median()), "tuning": plan.tuning, "graph": True}
    plan.close()
    # against double precision on the same GPU: the plain FP64 chain's chi^2 +
    # gradient evaluations of 512 of the data sets (full size each, points in
    # chunks of 64: its rate per data set does not depend on how many are
    # evaluated), and all-double fused fits of 256 data sets (20 iterations)
    fp64 = {}
    k = 512
    pl = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, npts=k, norm=N, prec=args.prec, kind=w.kind,
                  max_datasets=k, with_plain=True)
    q, dk = p0[:k].contiguous(), data[:k].contiguous()
    r = pl.eval(q, dk, grad=True, plain=True)
    torch.cuda.synchronize()
    a0, a1 = ev(), ev()
    a0.record(stream)
    for _ in range(2):
        pl.eval(q, dk, grad=True, plain=True, out=r)
    a1.record(stream)
    torch.cuda.synchronize()
    pl.status()
    ms64 = a0.elapsed_time(a1) / 2
    plain_launches = pl.launches
    mixed = pl.eval(q, dk, grad=True)
    torch.cuda.synchronize()
    relc = float(((mixed["chi2"] - r["chi2"]).abs() / r["chi2"].abs()).max())
    relg = float(((mixed["grad"] - r["grad"]).norm(dim=1) / r["grad"].norm(dim=1)).max())
    fp64["plain_fp64_chain"] = {"datasets": k, "ms_per_eval": ms64, "chi2_grad_evals_per_s": k * 1e3 / ms64,
                                "launches": plain_launches,
                                "mixed_eval_max_rel_err": {"chi2": relc, "grad_normwise": relg}}
    pl.close()
    k = 256
    pl = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, npts=k, norm=N, prec="fp64", kind=w.kind,
                  max_datasets=k)
    q, dk = p0[:k].clone(), data[:k].contiguous()
    ck = torch.empty(k, dtype=torch.float64, device=device)
    pl.fit(q, dk, iters=2, graph=True, chi2_out=ck)
    q.copy_(p0[:k])
    torch.cuda.synchronize()
    a0, a1 = ev(), ev()
    a0.record(stream)
    pl.fit(q, dk, iters=w.fit_iters, graph=True, chi2_out=ck)
    a1.record(stream)
    torch.cuda.synchronize()
    pl.status()
    ms64 = a0.elapsed_time(a1)
    fp64["fused_fp64_fits"] = {
        "datasets": k, "ms_per_batch": ms64, "fits_per_s": k * 1e3 / ms64,
        "chi2_grad_evals_per_s": k * w.fit_iters * 1e3 / ms64,
        "mixed_fit_max_rel_err": {"best_chi2": float(((c2[:k] - ck).abs() / ck.abs()).max()),
                                  "best_params": float(((p[:k] - q).abs() / q.abs()).max())}}
    pl.close()
    out["fits_16384x1000"]["fp64_gpu"] = fp64
    # the 10^4-point reactor chain (latency-bound), all-double and mixed, graph-replayed
    w = wl.reactor_200x50()
    res = {}
    for prec in ("fp64", "ff"):
        plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=1.0, prec=prec, kind=w.kind)
        p = plan.params_tensor(w.theta)
        d = torch.full((w.nbins,), 500.0, dtype=torch.float64, device=device)
        o = {"chi2": torch.empty(1, dtype=torch.float64, device=device),
             "grad": torch.empty(1, 4, dtype=torch.float64, device=device)}
        plan.set_graph(True)
        plan.autotune(p, d, reps=50)
        for _ in range(20):
            plan.eval(p, d, grad=True, out=o)
        torch.cuda.synchronize()
        a0, a1 = ev(), ev()
        reps = 2000
        a0.record(stream)
        for _ in range(reps):
            plan.eval(p, d, grad=True, out=o)
        a1.record(stream)
        torch.cuda.synchronize()
        ms = a0.elapsed_time(a1) / reps
        res[prec] = {"evals_per_s": 1e3 / ms, "us_per_eval": ms * 1e3, "tuning": plan.tuning}
        plan.close()
    out["reactor_200x50"] = dict(res, note="10^4 nodes: launch-latency bound (graph replay of 2-3 kernels)")
    # differentiable chi2 with 1000 per-bin nuisances (1000 bins x 4096 nodes x
    # 8 baselines): chi2 and its hand-written adjoint d chi2 / d(theta, eta)
    # through the autograd Function (forward + backward), and the same
    # evaluation called directly
    w = wl.nuisance_1000x4096()
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=1.0, prec=args.prec, kind=w.kind)
    truth = plan.params_tensor(w.truth)
    m = plan.eval(truth, torch.ones(w.nbins, dtype=torch.float64, device=device), grad=False, mu=True)["mu"][0]
    N = wl.TOTAL_EVENTS / float(m.sum())
    plan.close()
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=N, prec=args.prec, kind=w.kind)
    data = torch.as_tensor(wl.poisson_data((m * N).cpu().numpy(), w.data_seed), device=device)
    plan.autotune(plan.params_tensor(w.theta), data, reps=5, grad=True)
    theta = torch.tensor(w.theta[0], dtype=torch.float64, device=device, requires_grad=True)
    eta = torch.tensor(w.eta, dtype=torch.float64, device=device, requires_grad=True)

    def ad_step():
        theta.grad = None
        eta.grad = None
        api.chi2(theta, plan, data, eta, w.sigma_eta).backward()

    pt, et = plan.params_tensor(w.theta), torch.as_tensor(w.eta, device=device)
    od = {"chi2": torch.empty(1, dtype=torch.float64, device=device),
          "grad": torch.empty(1, 4, dtype=torch.float64, device=device),
          "grad_eta": torch.empty(1, w.nbins, dtype=torch.float64, device=device)}

    def direct_step():
        plan.eval(pt, data, et, w.sigma_eta, grad=True, grad_eta=True, out=od)

    def ad_step_calling_thread():
        # PyTorch runs a CUDA backward on its per-device worker thread by
        # default (two cross-thread hand-offs per backward); with the engine's
        # multithreading off it runs on the calling thread
        with torch.autograd.set_multithreading_enabled(False):
            ad_step()

    res = {}
    for name, fn in (("autograd", ad_step), ("autograd_calling_thread", ad_step_calling_thread),
                     ("direct", direct_step)):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        a0, a1 = ev(), ev()
        a0.record(stream)
        for _ in range(100):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        res[name] = a0.elapsed_time(a1) / 100 * 1e3
    check["nuisance"] = (w, N, data.cpu().numpy(), od["chi2"][0].item(), od["grad"][0].cpu().numpy(),
                         od["grad_eta"][0].cpu().numpy())
    ops = fp32_ops_per_node(w.nL, True, False) * w.nbins * w.nodes_per_bin
    out["nuisance_1000x4096"] = {
        "evals_per_s_autograd": 1e6 / res["autograd"], "us_per_eval_autograd": res["autograd"],
        "us_per_eval_autograd_calling_thread": res["autograd_calling_thread"],
        "us_per_eval_direct": res["direct"], "gpoints_per_s": w.points_per_eval() / res["direct"] / 1e3,
        "fp32_frac_of_issue_peak": ops / (res["direct"] * 1e-6) / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6),
        "outputs": "chi2, d chi2 / d(4 oscillation parameters, 1000 nuisances)", "tuning": plan.tuning}
    plan.close()
    # the paper's Table 1 shape: bare OscProb in FP64 on 10^4 and 10^6 energies,
    # GPU compute only and with the host<->device transfers (the host side is
    # timed in the CPU-baseline leg)
    t1 = {}
    for n in (10 ** 4, 10 ** 6):
        E_h = torch.linspace(1.8, 12.0, n, dtype=torch.float64).pin_memory()
        P_h = torch.empty(1, n, dtype=torch.float64).pin_memory()
        E_d = E_h.to(device)
        for _ in range(5):
            api.oscprob(E_d, [52.5], wl.TRUTH, "fp64")
        torch.cuda.synchronize()
        reps = 200
        a0, a1 = ev(), ev()
        a0.record(stream)
        for _ in range(reps):
            api.oscprob(E_d, [52.5], wl.TRUTH, "fp64")
        a1.record(stream)
        torch.cuda.synchronize()
        gpu_ms = a0.elapsed_time(a1) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            e = E_h.to(device, non_blocking=True)
            P = api.oscprob(e, [52.5], wl.TRUTH, "fp64")
            P_h.copy_(P, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        gpu_xfer_ms = (time.perf_counter() - t0) * 1e3 / reps
        def host_ms(fn):
            for _ in range(5):
                fn()
            torch.cuda.current_stream().synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
                torch.cuda.current_stream().synchronize()
            return (time.perf_counter() - t0) * 1e3 / reps

        # host to host without copies (the kernel reads E and writes P in
        # pinned host memory over the host link), and through device staging
        # in chunks whose transfers overlap the evaluation
        row = {"gpu_compute_ms": gpu_ms, "gpu_with_transfer_ms": gpu_xfer_ms}
        for prec in ("fp64", "ff"):
            P_pin = torch.empty(1, n, dtype=torch.float64 if prec == "fp64" else torch.float32).pin_memory()
            key = "" if prec == "fp64" else "_ff"
            row["gpu_host_memory_in_place_ms" + key] = host_ms(
                lambda: api.oscprob(E_h, [52.5], wl.TRUTH, prec, out=P_pin))
            row["gpu_staged_chunks_ms" + key] = host_ms(
                lambda: api.oscprob_staged(E_h, [52.5], wl.TRUTH, prec, out=P_pin))
        t1[str(n)] = row
    out["oscprob_fp64_table1_shape"] = t1
    # any channel (general formula with the CP term): numu -> nue and numu ->
    # numu at 810 km on 10^6 energies in 0.5-5 GeV, FP64 and mixed
    gen = {}
    th_full = (wl.TRUTH[0], wl.TRUTH[1], 0.545, 1.2 * np.pi, wl.TRUTH[2], wl.TRUTH[3])
    E_d = torch.linspace(500.0, 5000.0, 10 ** 6, dtype=torch.float64, device=device)
    for a, b in (("mu", "e"), ("mu", "mu")):
        for prec in ("fp64", "ff"):
            for _ in range(5):
                api.oscprob_general(E_d, [810.0], th_full, a, b, prec=prec)
            torch.cuda.synchronize()
            reps = 200
            a0, a1 = ev(), ev()
            a0.record(stream)
            for _ in range(reps):
                api.oscprob_general(E_d, [810.0], th_full, a, b, prec=prec)
            a1.record(stream)
            torch.cuda.synchronize()
            ms = a0.elapsed_time(a1) / reps
            gen["%s->%s %s" % (a, b, prec)] = {"us": ms * 1e3, "gpoints_per_s": 1e6 / (ms * 1e-3) / 1e9}
    out["oscprob_any_channel_810km_1e6"] = gen
    # the fits workload's 16384 x 1000 Poisson pseudo-data drawn on the device
    wf = wl.fits_16384x1000()
    mu_f = np.linspace(20.0, 400.0, wf.nbins)
    api.poisson_datasets(mu_f, 16, 4)
    torch.cuda.synchronize()
    a0, a1 = ev(), ev()
    a0.record(stream)
    for _ in range(5):
        api.poisson_datasets(mu_f, wf.npts, 4)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / 5
    out["pseudo_data_16384x1000"] = {"ms": ms, "gsamples_per_s": wf.npts * wf.nbins / (ms * 1e-3) / 1e9,
                                     "mu_range": [20.0, 400.0]}
    return out, check


def fp32_probe(api, torch, device, index):
    """Measured FP32 pipe rate: the library's probe kernel (eight FMA chains per
    thread, eight 256-thread blocks per SM) over ~0.7 s of launches, CUDA events
    on the stream, the SM clock sampled meanwhile; FMA = one operation, as in
    the node kernels' counts.  Clocks are only read, never set."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, iters, reps = sms * 8, 1 << 18, 40
    out = torch.empty(1, dtype=torch.float32, device=device)
    api.fp32_probe(blocks, 1024, out)
    torch.cuda.synchronize()
    clk = Clocks(index)
    clk.start()
    time.sleep(0.2)
    stream = torch.cuda.current_stream()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    fmas = sum(api.fp32_probe(blocks, iters, out) for _ in range(reps))
    a1.record(stream)
    torch.cuda.synchronize()
    c = clk.stop()
    rate = fmas / (a0.elapsed_time(a1) * 1e-3)
    res = {"tops": rate / 1e12, "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons"), "samples": c.get("samples")}
    if c.get("sm_mhz"):
        res["fma_per_sm_per_clk"] = rate / (sms * c["sm_mhz"] * 1e6)
    return res


def short(x):
    """A float rounded to four significant digits (the summary at the end of the line)."""
    return None if x is None else float("%.4g" % x)


def fp64_summary(evals_per_s, plain, side, cpu):
    """The mixed path against double precision on the same GPU, per workload:
    the plain FP64 chain and the all-double fused kernel, with the mixed path's
    largest error against them; placed last on the line."""
    out = {}
    if plain is not None:
        e = plain["max_rel_err"]
        out["reactor8_1000x16384"] = {
            "mixed_evals_per_s": short(evals_per_s), "plain_fp64_evals_per_s": short(plain["evals_per_s"]),
            "x_plain": short(plain["speedup"]), "fused_fp64_evals_per_s": short(plain["fused_fp64"]["evals_per_s"]),
            "x_fused_fp64": short(plain["fused_fp64"]["speedup"]),
            "max_rel_err": {"chi2": short(e["chi2"]), "mu": short(e["mu"]), "spectra": short(e["spectra"])}}
    if side is not None:
        s = side["scan_64x64_500bins"]
        f = s["fp64_gpu"]
        out["scan_64x64_500bins"] = {
            "mixed_evals_per_s": short(s["chi2_grad_evals_per_s"]),
            "plain_fp64_evals_per_s": short(f["plain_fp64_chain"]["chi2_grad_evals_per_s"]),
            "x_plain": short(s["chi2_grad_evals_per_s"] / f["plain_fp64_chain"]["chi2_grad_evals_per_s"]),
            "fused_fp64_evals_per_s": short(f["fused_fp64"]["chi2_grad_evals_per_s"]),
            "x_fused_fp64": short(s["chi2_grad_evals_per_s"] / f["fused_fp64"]["chi2_grad_evals_per_s"]),
            "max_rel_err": {k: short(v) for k, v in f["plain_fp64_chain"]["mixed_max_rel_err"].items()}}
        s = side["fits_16384x1000"]
        f = s["fp64_gpu"]
        pc, ff = f["plain_fp64_chain"], f["fused_fp64_fits"]
        out["fits_16384x1000"] = {
            "mixed_evals_per_s": short(s["chi2_grad_evals_per_s"]),
            "plain_fp64_evals_per_s": short(pc["chi2_grad_evals_per_s"]),
            "x_plain": short(s["chi2_grad_evals_per_s"] / pc["chi2_grad_evals_per_s"]),
            "fused_fp64_fits_per_s": short(ff["fits_per_s"]), "mixed_fits_per_s": short(s["fits_per_s"]),
            "x_fused_fp64": short(s["fits_per_s"] / ff["fits_per_s"]),
            "max_rel_err": {"eval_chi2": short(pc["mixed_eval_max_rel_err"]["chi2"]),
                            "fit_chi2": short(ff["mixed_fit_max_rel_err"]["best_chi2"]),
                            "fit_params": short(ff["mixed_fit_max_rel_err"]["best_params"])}}
    return out


def cpu_side_errors(side, check):
    """CPU-baseline leg of the batched workloads: the oracle at sampled points
    of the scan, on the nuisance evaluation and on one fit; adds each
    workload's error against it."""
    import oracle

    rmax = lambda a, b: float(np.max(np.abs(np.asarray(a) - b) / np.abs(b)))
    nrel = lambda a, b: float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))
    w, N, d, c2, g = check["scan"]
    e = {"points": [0, 2049, 4095], "chi2": 0.0, "grad_normwise": 0.0}
    for p in e["points"]:
        r = oracle.chain(w.edges, int(w.node_counts[p]), w.L, w.theta[p], N, d, w.kind, e_scale=w.e_scale)
        e["chi2"] = max(e["chi2"], rmax(c2[p], r["chi2"]))
        e["grad_normwise"] = max(e["grad_normwise"], nrel(g[p], r["grad"][:4]))
    side["scan_64x64_500bins"]["error_vs_oracle"] = e
    w, N, d, c2, g, th6 = check["scan_numu_nue"]
    e = {"points": [0, 2049, 4095], "chi2": 0.0, "grad_normwise": 0.0}
    for p in e["points"]:
        r = oracle.chain_general(w.edges, int(w.node_counts[p]), w.L, th6[p], N, d, "mu", "e", False, w.kind,
                                 e_scale=w.e_scale)
        e["chi2"] = max(e["chi2"], rmax(c2[p], r["chi2"]))
        e["grad_normwise"] = max(e["grad_normwise"], nrel(g[p], r["grad"][:6]))
    side["scan_64x64_500bins_numu_nue"]["error_vs_oracle"] = e
    w, N, d, c2, g, ge = check["nuisance"]
    r = oracle.chain(w.edges, w.nodes_per_bin, w.L, w.theta[0], N, d, w.kind, eta=w.eta, sigma=w.sigma_eta)
    side["nuisance_1000x4096"]["error_vs_oracle"] = {
        "chi2": rmax(c2, r["chi2"]), "grad_normwise": nrel(g, r["grad"][:4]),
        "grad_eta_normwise": nrel(ge, r["grad"][4:])}
    w, N, d, pf, c2 = check["fits"]
    ev = lambda t: oracle.chain(w.edges, w.nodes_per_bin, w.L, t, N, d, w.kind)
    th, c2o, _ = oracle.fit_lm(ev, w.theta[0], iters=w.fit_iters)
    side["fits_16384x1000"]["error_vs_oracle"] = {
        "dataset": 0, "best_chi2": rmax(c2, c2o), "best_params": rmax(pf, th)}


def cpu_oscprob_table1(t1):
    """CPU-baseline leg of the Table 1 shape: the oracle's OscProb (FP64, all
    host cores) on the same 10^4 and 10^6 energies; adds the CPU/GPU ratios."""
    import oracle
    import torch

    for key, row in t1.items():
        n = int(key)
        En = torch.linspace(1.8, 12.0, n, dtype=torch.float64).numpy()
        oracle.pee(En, 52.5, wl.TRUTH)
        t0 = time.perf_counter()
        for _ in range(5):
            oracle.pee(En, 52.5, wl.TRUTH)
        cpu_ms = (time.perf_counter() - t0) * 1e3 / 5
        row.update({"cpu_oracle_ms": cpu_ms, "cpu_threads": oracle.threads(),
                    "cpu_over_gpu_with_transfer": cpu_ms / row["gpu_with_transfer_ms"],
                    "cpu_over_gpu_host_memory_in_place": cpu_ms / row["gpu_host_memory_in_place_ms"],
                    "cpu_over_gpu_staged_chunks": cpu_ms / row["gpu_staged_chunks_ms"],
                    "cpu_over_gpu_compute": cpu_ms / row["gpu_compute_ms"]})


# ---------------------------------------------------------------------- ours --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="reactor8_1000x16384")
    ap.add_argument("--prec", default="ff", choices=["ff", "f64phase", "fp64"])
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 chain comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default=None)
    ap.add_argument("--no-side", action="store_true", help="skip the scan and fit side measurements")
    ap.add_argument("--no-probe", action="store_true", help="skip the FP32 rate probe")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)

    import torch

    from paper_1804_07682_gb300 import api

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    device = torch.device("cuda", local)
    w = wl.ALL[args.workload]()
    if w.node_counts is not None or w.n_datasets > 1:
        raise SystemExit("bench.py times the single-point reactor workloads; use --workload reactor8_1000x16384")
    stream = torch.cuda.current_stream()

    # Configuration stage: plan, Asimov truth from the library itself (normalised
    # to 1e5 events), Poisson pseudo-data with a per-rank seed.
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=1.0, e_scale=w.e_scale, prec=args.prec,
                    kind=w.kind, with_plain=not args.no_plain)
    truth = plan.params_tensor(w.truth)
    dummy = torch.ones(w.nbins, dtype=torch.float64, device=device)
    m = plan.eval(truth, dummy, grad=False, mu=True)["mu"][0]
    N = wl.TOTAL_EVENTS / float(m.sum())
    plan.close()
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=N, e_scale=w.e_scale, prec=args.prec,
                    kind=w.kind, with_plain=not args.no_plain)
    mu_truth = (m * N).cpu().numpy()
    data_np = wl.poisson_data(mu_truth, replica_seed(w.data_seed, rank))
    data = torch.as_tensor(data_np, device=device)
    params = plan.params_tensor(w.theta)
    if args.tuning:
        plan.tuning = args.tuning
    elif not args.no_autotune:
        plan.autotune(params, data, reps=20, grad=True, spectra=True)
    out = {"chi2": torch.empty(1, dtype=torch.float64, device=device),
           "grad": torch.empty(1, 4, dtype=torch.float64, device=device),
           "spectra": torch.empty(1, w.nL, w.nbins, dtype=torch.float64, device=device)}

    def step():
        plan.eval(params, data, grad=True, spectra=True, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.status()
    launches_per_step = plan.launches

    # Timed region: K evaluations, events on the launching stream, kernel events inside the library.
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    # kernel events on every k-th evaluation (events between kernels hold back
    # the dependent launch, so the others run undisturbed), k <= 8 and at
    # least ten timed launches
    prof_every = max(1, min(PROFILE_EVERY, args.steps // 10))
    plan.profile(prof_every)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    kern_ms, kern_n = plan.profile_read()
    plan.profile(False)
    clk = clocks.stop()
    ms_total, evals_per_s = replica_throughput(dist, ms_total, args.steps, world, device)
    ms_step = ms_total / args.steps
    points = w.points_per_eval()
    kern_avg_ms = kern_ms / max(kern_n, 1)

    # roofline of the fused kernel (ALU-bound: FP32 issue)
    ops = fp32_ops_per_node(w.nL, True, True) * w.nbins * w.nodes_per_bin
    achieved_tops = ops / (kern_avg_ms * 1e-3) / 1e12
    peak_tops = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12
    pk, pk_src = peaks()
    hbm_bytes = 16 * w.nbins * w.nodes_per_bin
    mapping = plan.tuning.split()[0].split("=")[1]
    cap = TRAFFIC_CAPTURE.get(mapping, {})
    traffic = cap.get("bytes") if cap.get("sources_sha256") == kernel_sources_sha256() else None
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "TFLOP/s",
                "frac": achieved_tops / peak_tops, "traffic": traffic, "algorithmic_bytes": hbm_bytes,
                "kernel": KERNEL_NAMES.get(mapping, mapping) + " (double-float phase, 8 baselines, gradient + spectra)",
                "kernel_ms": kern_avg_ms, "ops_per_launch": ops,
                "timed_launches": kern_n, "timed_every": prof_every,
                "peak_note": "FP32 issue peak 152 SM x 128 lanes x 2070 MHz (FMA = 1 op)",
                "hbm_frac": hbm_bytes / (kern_avg_ms * 1e-3) / 1e9 / pk.get("hbm_gbs", 6800.0),
                "hbm_peak_src": pk_src}

    # epilogue only on the node sums the last evaluation kept (a change of the
    # data or of the nuisances costs no node pass)
    for _ in range(5):
        plan.eval_cached(data, grad=True, out={"chi2": out["chi2"], "grad": out["grad"]})
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(200):
        plan.eval_cached(data, grad=True, out={"chi2": out["chi2"], "grad": out["grad"]})
    c1.record(stream)
    torch.cuda.synchronize()
    epilogue_only = {"us_per_eval": c0.elapsed_time(c1) / 200 * 1e3,
                     "note": "gna_chain_eval_cached: new data or nuisances on the kept node sums, chi2 + gradient"}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    p_host = torch.as_tensor(w.theta.reshape(1, 4)).pin_memory().numpy()
    d_host = torch.as_tensor(data_np).pin_memory().numpy()
    c_host = torch.empty(1, dtype=torch.float64).pin_memory().numpy()
    g_host = torch.empty(1, 4, dtype=torch.float64).pin_memory().numpy()
    s_host = torch.empty(1, w.nL, w.nbins, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(10, args.steps)
    plan.set_graph(True)
    for _ in range(3):
        plan.eval_host(p_host, d_host, grad=True, chi2_out=c_host, grad_out=g_host, spectra_out=s_host)
    if dist is not None:
        dist.barrier()
    # every step copies its inputs in and its results out; step k + 1 is
    # enqueued (asynchronous host API) before step k's results are taken, so
    # the host's packing and unpacking overlap the device's work
    t0 = time.perf_counter()
    ticket = plan.eval_host_async(p_host, d_host, grad=True, spectra=True)
    for k in range(e2e_steps):
        nxt = plan.eval_host_async(p_host, d_host, grad=True, spectra=True) if k + 1 < e2e_steps else None
        plan.eval_host_wait(ticket, c_host, g_host, s_host)
        ticket = nxt
    e2e_ms, e2e_rate = replica_throughput(dist, (time.perf_counter() - t0) * 1e3, e2e_steps, world, device)
    plan.set_graph(False)
    e2e = {"value": e2e_rate, "unit": "evals/s", "h2d_bytes_per_step": p_host.nbytes + d_host.nbytes,
           "d2h_bytes_per_step": c_host.nbytes + g_host.nbytes + s_host.nbytes,
           "api": "Plan.eval_host_async / eval_host_wait (gna_chain_eval_host_async / _wait), two in flight"}

    # plain FP64 chain on the same GPU, and the error of the timed path against it
    plain = None
    if not args.no_plain:
        po = {"chi2": torch.empty(1, dtype=torch.float64, device=device),
              "grad": torch.empty(1, 4, dtype=torch.float64, device=device),
              "spectra": torch.empty(1, w.nL, w.nbins, dtype=torch.float64, device=device),
              "mu": torch.empty(1, w.nbins, dtype=torch.float64, device=device)}
        plan.eval(params, data, grad=True, spectra=True, mu=True, out=po, plain=True)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.plain_steps):
            plan.eval(params, data, grad=True, spectra=True, mu=True, out=po, plain=True)
        a1.record(stream)
        torch.cuda.synchronize()
        plain_ms = reduce_max(dist, a0.elapsed_time(a1) / args.plain_steps, device)
        mo = plan.eval(params, data, grad=True, spectra=True, mu=True)
        torch.cuda.synchronize()
        relerr = lambda a, b: float(((a - b).abs() / b.abs()).max())
        plain = {"evals_per_s": world * 1e3 / plain_ms, "ms_per_step": plain_ms,
                 "speedup": (world * 1e3 / plain_ms) and evals_per_s / (world * 1e3 / plain_ms),
                 "max_rel_err": {"chi2": relerr(mo["chi2"], po["chi2"]), "mu": relerr(mo["mu"], po["mu"]),
                                 "spectra": relerr(mo["spectra"], po["spectra"]),
                                 "grad_normwise": float((mo["grad"] - po["grad"]).norm() / po["grad"].norm())}}
        # and the all-double fused kernel on the same workload
        p64 = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=N, e_scale=w.e_scale, prec="fp64",
                       kind=w.kind)
        o64 = p64.eval(params, data, grad=True, spectra=True)
        torch.cuda.synchronize()
        a0.record(stream)
        for _ in range(args.plain_steps):
            p64.eval(params, data, grad=True, spectra=True, out=o64)
        a1.record(stream)
        torch.cuda.synchronize()
        p64.status()
        f64_ms = reduce_max(dist, a0.elapsed_time(a1) / args.plain_steps, device)
        plain["fused_fp64"] = {"evals_per_s": world * 1e3 / f64_ms, "ms_per_step": f64_ms,
                               "speedup": evals_per_s / (world * 1e3 / f64_ms),
                               "max_rel_err_chi2": relerr(mo["chi2"], o64["chi2"])}
        p64.close()

    # CPU baseline: the oracle, as it stands, on all host cores (rank 0 only):
    # one full evaluation (every bin, node and baseline, with the gradient)
    # after a one-bin call that builds and caches the Gauss-Legendre rule.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        oracle.chain(w.edges[:2], w.nodes_per_bin, w.L, w.theta[0], 1.0, np.full(1, 100.0), w.kind)
        t0 = time.perf_counter()
        ref = oracle.chain(w.edges, w.nodes_per_bin, w.L, w.theta[0], N, data_np, w.kind)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "evals/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": "one full evaluation (%d bins x %d nodes x %d baselines, with gradient) in %.2f s on %d threads"
                         % (w.nbins, w.nodes_per_bin, w.nL, dt, oracle.threads())}
        # the benchmarked path's error against that oracle evaluation, every output
        go = plan.eval(params, data, grad=True, spectra=True, mu=True)
        torch.cuda.synchronize()
        rmax = lambda a, b: float(np.max(np.abs(a - b) / np.abs(b)))
        g = go["grad"][0].cpu().numpy()
        cpu["gpu_error_vs_oracle"] = {
            "chi2": rmax(go["chi2"][0].item(), ref["chi2"]), "mu": rmax(go["mu"][0].cpu().numpy(), ref["mu"]),
            "spectra": rmax(go["spectra"][0].cpu().numpy(), ref["mu_rb"]),
            "grad_normwise": float(np.linalg.norm(g - ref["grad"][:4]) / np.linalg.norm(ref["grad"][:4]))}

    side, check = (None, None) if args.no_side else side_workloads(api, torch, device, args)
    if side is not None and cpu is not None:
        cpu_oscprob_table1(side["oscprob_fp64_table1_shape"])
        cpu_side_errors(side, check)

    # the FP32 pipe rate measured by the probe kernel: the roofline's second denominator
    probe = fp32_probe(api, torch, device, local) if not args.no_probe else None
    if probe is not None:
        roofline["measured_peak"] = probe["tops"]
        roofline["frac_of_measured"] = achieved_tops / probe["tops"]
        roofline["measured_peak_sm_mhz"] = probe["sm_mhz"]
        roofline["measured_peak_note"] = "FP32 FMA probe (gna_fp32_probe), CUDA events, SM clock sampled during it"

    if rank == 0:
        gpu_err = cpu.pop("gpu_error_vs_oracle", None) if cpu is not None else None
        line = {"metric": METRIC, "value": evals_per_s, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+ff-phase" if args.prec == "ff" else args.prec, "data": "synthetic",
                "config": {"workload": w.name, "bins": w.nbins, "nodes_per_bin": w.nodes_per_bin, "baselines": w.nL,
                           "points_per_eval": points, "outputs": "chi2, 4-parameter gradient, 8 per-baseline spectra",
                           "l2": "inputs larger than L2 (%d MB energy grid)" % (hbm_bytes >> 20),
                           "tuning": plan.tuning, "parallelism": "replicas" if world > 1 else "single"},
                "gpoints_per_s": evals_per_s * points / 1e9, "roofline": roofline, "plain_fp64_chain": plain,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches_per_step * args.steps,
                "epilogue_only": epilogue_only,
                "side_workloads": side,
                # last on the line: the mixed path against double precision on
                # this GPU, per workload, and the timed path's error against the oracle
                "fp32_probe": probe,
                "vs_fp64_gpu": fp64_summary(evals_per_s, plain, side, cpu),
                "gpu_error_vs_oracle": gpu_err}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
