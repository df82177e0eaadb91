"""Full-size parity: the five workloads at their real sizes, CUDA path (mixed
double-float-phase precision, the benchmarked configuration) vs the FP64
oracle.  The 8-baseline reactor workloads are compared whole (the oracle runs
on all host cores); the scan and the fits are compared on sampled points /
datasets that the oracle computes one by one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1804_07682_gb300 import workloads as wl
from refs import Case, chi2_err_bound, normrel, rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module")
def api():
    from paper_1804_07682_gb300 import api as _api
    return _api


@pytest.mark.parametrize("tuning", [None, "mapping=split block=256 nodes=32", "mapping=split block=128 nodes=128",
                                    "mapping=slices block=256 slice=216", "mapping=slices block=128 slice=108",
                                    "mapping=slices block=256 slice=1000"])
def test_reactor8_full(api, tuning):
    w = wl.reactor8_1000x16384()
    case = _cached("reactor8", lambda: Case(w))
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=case.N, prec="ff", kind=w.kind)
    if tuning:
        plan.tuning = tuning
    out = plan.eval(plan.params_tensor(w.theta), dev(case.data), grad=True, mu=True, spectra=True)
    torch.cuda.synchronize()
    plan.status()
    ref = _cached("reactor8_ref", lambda: case.oracle_point(0))
    assert abs(out["chi2"][0].item() - ref["chi2"]) <= 1e-6 * chi2_err_bound(ref, case.data, w.kind)
    assert rel(out["chi2"][0].item(), ref["chi2"]) < 1e-6
    assert rel(out["mu"][0].cpu().numpy(), ref["mu"]) < 1e-6
    assert rel(out["spectra"][0].cpu().numpy(), ref["mu_rb"]) < 1e-6
    assert normrel(out["grad"][0].cpu().numpy(), ref["grad"][:4]) < 1e-4
    plan.close()


def test_nuisance_full_with_autograd(api):
    w = wl.nuisance_1000x4096()
    case = Case(w)
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=case.N, prec="ff", kind=w.kind)
    theta = dev(w.theta[0]).requires_grad_(True)
    eta = dev(w.eta).requires_grad_(True)
    c = api.chi2(theta, plan, dev(case.data), eta, w.sigma_eta)
    c.backward()
    ref = case.oracle_point(0)
    assert abs(c.item() - ref["chi2"]) <= 1e-6 * chi2_err_bound(ref, case.data, w.kind)
    assert normrel(theta.grad.cpu().numpy(), ref["grad"][:4]) < 1e-4
    assert normrel(eta.grad.cpu().numpy(), ref["grad"][4:]) < 1e-4


def test_scan_full_sampled(api):
    w = wl.scan_64x64_500bins()
    case = Case(w)  # truth model at 524 nodes per bin
    plan = api.Plan(w.edges, w.L, npts=w.npts, node_counts=w.node_counts, norm=case.N, e_scale=w.e_scale,
                    prec="ff", kind=w.kind)
    plan.set_graph(True)
    out = plan.eval(plan.params_tensor(w.theta), dev(case.data), grad=True, mu=True)
    torch.cuda.synchronize()
    plan.status()
    chi2 = out["chi2"].cpu().numpy()
    # Delta chi2 surface: minimum near the truth point of the grid
    s13 = w.theta[:, 1].reshape(64, 64)
    d32 = w.theta[:, 3].reshape(64, 64)
    j = int(np.argmin(chi2))
    assert abs(w.theta[j, 1] / wl.TRUTH[1] - 1) < 0.1 and abs(w.theta[j, 3] / wl.TRUTH[3] - 1) < 0.05
    for p in [0, 1, 777, 2048, 4095, j]:
        ref = case.oracle_point(p)
        assert abs(chi2[p] - ref["chi2"]) <= 1e-6 * chi2_err_bound(ref, case.data, w.kind), p
        assert rel(out["mu"][p].cpu().numpy(), ref["mu"]) < 1e-6
        assert normrel(out["grad"][p].cpu().numpy(), ref["grad"][:4]) < 1e-4
    del s13, d32


def test_fits_full_sampled(api):
    w = wl.fits_16384x1000()
    case = Case(w)
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, npts=w.npts, norm=case.N, prec="ff", kind=w.kind,
                    max_datasets=w.npts)
    params = plan.params_tensor(w.theta).clone()
    data = dev(case.data)
    start = plan.eval(params, data, grad=False)["chi2"].cpu().numpy()
    params, chi2 = plan.fit(params, data, iters=20, graph=True)
    torch.cuda.synchronize()
    plan.status()
    P = params.cpu().numpy()
    C = chi2.cpu().numpy()
    assert np.all(np.isfinite(C)) and np.all(C > 0)
    # the best point of a Levenberg-Marquardt fit never has a larger chi2 than its start
    assert np.all(C <= start * (1 + 1e-12))
    assert np.mean(C) < np.mean(start)
    for j in [0, 9999]:
        ev = lambda t, j=j: oracle.chain(w.edges, w.nodes_per_bin, w.L, t, case.N, case.data[j], w.kind)
        th, c2, _ = oracle.fit_lm(ev, w.theta[j], iters=20)
        assert rel(C[j], c2) < 1e-6, (j, C[j], c2)
        assert rel(P[j], th) < 1e-3, (j, P[j], th)


_cache = {}


def _cached(key, fn):
    if key not in _cache:
        _cache[key] = fn()
    return _cache[key]


def test_pseudo_data_full_size_sampled(api):
    # the 16384 x 1000 pseudo-experiments of the fits workload drawn on the
    # device; sampled data sets (first, middle, last) against the oracle
    w = wl.fits_16384x1000()
    case = _cached("fits_case", lambda: Case(w))
    d = api.poisson_datasets(case.mu_truth, w.npts, 4)
    assert tuple(d.shape) == (w.npts, w.nbins)
    for j in (0, 8191, 16383):
        ref = oracle.pseudo_data(case.mu_truth, 1, 4, j0=j)[0]
        assert np.array_equal(d[j].cpu().numpy(), ref), j
    m = d.mean(0).cpu().numpy()
    assert np.abs(m - case.mu_truth).max() < 6 * np.sqrt(case.mu_truth.max() / w.npts) + 1e-9


def test_scan_numu_nue_full_sampled(api):
    # the 64 x 64 scan for nu_mu -> nu_e appearance through the any-channel
    # chain (s2_23 = 0.545, delta = 1.2 pi) on the 4096 uneven grids; sampled
    # points against the oracle, with the tuning the autotuner picks
    w = wl.scan_64x64_500bins()
    k = w.npts
    th6 = np.column_stack([w.theta[:, 0], w.theta[:, 1], np.full(k, 0.545), np.full(k, 1.2 * np.pi),
                           w.theta[:, 2], w.theta[:, 3]])
    truth = np.array([wl.TRUTH[0], wl.TRUTH[1], 0.545, 1.2 * np.pi, wl.TRUTH[2], wl.TRUTH[3]])
    n_t = int(np.max(w.node_counts))
    mu_rb, _ = oracle.binned_general(w.edges, n_t, w.L, truth, "mu", "e", False, w.e_scale)
    N = 1e5 / mu_rb[0].sum()
    data = wl.poisson_data(N * mu_rb[0], 13)
    plan = api.Plan(w.edges, w.L, npts=k, node_counts=w.node_counts, norm=N, e_scale=w.e_scale, prec="ff",
                    kind=w.kind, channel=("mu", "e", False))
    p = plan.params_tensor(th6)
    d = dev(data)
    o = {"chi2": torch.empty(k, dtype=torch.float64, device="cuda"),
         "grad": torch.empty(k, 6, dtype=torch.float64, device="cuda")}
    plan.autotune(p, d, reps=1)
    plan.eval_general(p, d, out=o)
    torch.cuda.synchronize()
    plan.status()
    chi2 = o["chi2"].cpu().numpy()
    g = o["grad"].cpu().numpy()
    for q in [0, 1, 777, 2048, 4095, int(np.argmin(chi2))]:
        ref = oracle.chain_general(w.edges, int(w.node_counts[q]), w.L, th6[q], N, data, "mu", "e", False, w.kind,
                                   e_scale=w.e_scale)
        assert abs(chi2[q] - ref["chi2"]) <= 1e-6 * chi2_err_bound(ref, data, w.kind), q
        assert normrel(g[q], ref["grad"][:6]) < 1e-4, q
    plan.close()
