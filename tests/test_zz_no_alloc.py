"""The allocation-free evaluation (gna_chain_eval_noalloc) against the FP64
oracle and against the plan-based evaluation (gna_chain_eval), through the C ABI.

gna_chain_eval_noalloc exists for callers that cannot allocate device memory
(a pool or arena they do not own, a host framework that forbids cudaMalloc);
it works in a fixed array inside the library that every call shares.  Two
calls in a row must both match, which also shows that each call starts from
cleared counters.  Baseline counts 2, 3 and 5 run the kernels built for 2, 4
and 8 baselines with zero-weight padding.  This file is collected last and is
self-contained, so it passes alone in a fresh process as well as after the
rest of the suite.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1804_07682_gb300 import workloads as wl
from refs import Case, check_chi2, normrel, rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

TOL = 1e-6   # mixed-precision tolerance of the parity tests (mu, chi^2)
GTOL = 1e-4  # gradient bound of the mixed-precision parity tests


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def node_arrays(w):
    """E and W on the bin-major Gauss-Legendre grid (numpy's leggauss rule)."""
    x, wt = np.polynomial.legendre.leggauss(w.nodes_per_bin)
    a, b = w.edges[:-1, None], w.edges[1:, None]
    half, mid = 0.5 * (b - a), 0.5 * (a + b)
    E = mid + half * x[None, :]
    Es = E * w.e_scale
    W = half * wt[None, :] * np.exp(0.87 - 0.16 * Es - 0.091 * Es * Es)
    return E, W


def baseline_case(nL, nbins=24, nodes=300, seed=0):
    rng = np.random.default_rng(100 + nL + seed)
    L = np.sort(rng.uniform(0.5, 60.0, nL))
    theta = np.array([wl.TRUTH]) * rng.uniform(0.97, 1.03, size=(1, 4))
    w = wl.Workload("noalloc_%dL" % nL, np.linspace(1.8, 9.0, nbins + 1), nodes, L, theta, wl.POISSON)
    return w, Case(w)


def run_noalloc(api, w, case, Lweight=None, grad=True, mu=True, calls=2):
    E, W = (dev(a) for a in node_arrays(w))
    params, data = dev(w.theta[:1]), dev(case.data)
    res = []
    for _ in range(calls):
        out = api.chi2_noalloc(E, W, w.L, params, data, case.N, kind=w.kind, Lweight=Lweight, grad=grad, mu=mu)
        torch.cuda.synchronize()
        res.append({k: v.cpu().numpy() for k, v in out.items()})
    return res


@pytest.mark.parametrize("name", ["reactor_200x50", "reactor8_40x3000"])
def test_noalloc_matches_oracle_and_plan_twice(name):
    from paper_1804_07682_gb300 import api

    w = wl.reactor_200x50() if name == "reactor_200x50" else wl.shrink(wl.reactor8_1000x16384(), nbins=40, nodes=3000)
    case = Case(w)
    ref = case.oracle_point(0)
    res = run_noalloc(api, w, case)
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=case.N, e_scale=w.e_scale, prec="ff", kind=w.kind)
    pl = plan.eval(dev(w.theta[:1]), dev(case.data), grad=True, mu=True)
    pl = {k: v[0].cpu().numpy() for k, v in pl.items()}
    plan.close()
    for r in res:
        check_chi2(float(r["chi2"][0]), ref, case.data, w.kind, TOL, tag="noalloc " + name)
        assert rel(r["mu"], ref["mu"]) < TOL
        assert normrel(r["grad"], ref["grad"][:4]) < GTOL
        # the same arithmetic as the plan's mixed path
        assert rel(r["chi2"][0], pl["chi2"]) < 2 * TOL and rel(r["mu"], pl["mu"]) < 2 * TOL
    assert np.array_equal(res[0]["chi2"], res[1]["chi2"])
    assert np.array_equal(res[0]["mu"], res[1]["mu"])
    assert np.array_equal(res[0]["grad"], res[1]["grad"])


@pytest.mark.parametrize("nL", [1, 2, 3, 5, 8])
def test_noalloc_baseline_counts(nL):
    # 2, 3 and 5 baselines run the 2-, 4- and 8-baseline kernels with
    # zero-weight slots; every output against the oracle, two calls in a row
    from paper_1804_07682_gb300 import api

    w, case = baseline_case(nL)
    ref = case.oracle_point(0)
    res = run_noalloc(api, w, case)
    for r in res:
        check_chi2(float(r["chi2"][0]), ref, case.data, w.kind, TOL, tag="noalloc nL=%d" % nL)
        assert rel(r["mu"], ref["mu"]) < TOL, nL
        assert normrel(r["grad"], ref["grad"][:4]) < GTOL, nL
    assert np.array_equal(res[0]["chi2"], res[1]["chi2"]) and np.array_equal(res[0]["mu"], res[1]["mu"])


def test_noalloc_explicit_weights_and_optional_outputs():
    # caller weights (normalised to sum 1 by the call), then chi^2 alone: no
    # gradient, no mu (both NULL at the C ABI)
    from paper_1804_07682_gb300 import api

    w, case = baseline_case(3, seed=7)
    Lw = np.array([0.5, 2.0, 1.5])
    om = Lw / Lw.sum()
    ref = oracle.chain(w.edges, w.nodes_per_bin, w.L, w.theta[0], case.N, case.data, w.kind, omega=om)
    (r,) = run_noalloc(api, w, case, Lweight=Lw, calls=1)
    check_chi2(float(r["chi2"][0]), ref, case.data, w.kind, TOL, tag="noalloc Lweight")
    assert rel(r["mu"], ref["mu"]) < TOL
    assert normrel(r["grad"], ref["grad"][:4]) < GTOL
    res = run_noalloc(api, w, case, Lweight=Lw, grad=False, mu=False)
    for q in res:
        assert set(q) == {"chi2"}
        assert q["chi2"][0] == r["chi2"][0]  # the same node sums and epilogue


def test_noalloc_refuses_memory_it_cannot_use():
    # at the C ABI: host memory, a misaligned pointer or a NULL output is
    # refused before anything is launched
    from paper_1804_07682_gb300 import _native as N

    w, case = baseline_case(1)
    E, W = (dev(a) for a in node_arrays(w))
    params, data = dev(w.theta[:1]), dev(case.data)
    chi2 = torch.empty(1, dtype=torch.float64, device="cuda")
    host = torch.as_tensor(node_arrays(w)[0]).pin_memory()
    Ls = np.ascontiguousarray(w.L)
    P = ctypes.POINTER(ctypes.c_double)
    vp = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)

    def call(E_, W_, d_, c_, lw=None):
        return N.lib().gna_chain_eval_noalloc(w.nbins, w.nodes_per_bin, E_, W_, Ls.ctypes.data_as(P), Ls.size,
                                              None if lw is None else lw.ctypes.data_as(P), vp(params),
                                              ctypes.c_double(case.N), w.kind, d_, c_, None, None, None)

    assert call(vp(E), vp(W), vp(data), vp(chi2)) == N.GNA_OK
    torch.cuda.synchronize()
    assert call(vp(host), vp(W), vp(data), vp(chi2)) == N.GNA_EINVAL
    assert call(vp(E, 4), vp(W), vp(data), vp(chi2)) == N.GNA_EINVAL
    assert call(vp(E), vp(W), vp(data), None) == N.GNA_EINVAL
    # baseline weights are normalised by their sum: zero or infinite ones are refused
    assert call(vp(E), vp(W), vp(data), vp(chi2), np.zeros(Ls.size)) == N.GNA_EINVAL
    assert call(vp(E), vp(W), vp(data), vp(chi2), np.full(Ls.size, np.inf)) == N.GNA_EINVAL


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1804_07682_gb300 import _native as N
    from paper_1804_07682_gb300 import api

    E = torch.ones(2049, 4, dtype=torch.float64, device="cuda")
    p = torch.zeros(1, 4, dtype=torch.float64, device="cuda")
    d = torch.ones(2049, dtype=torch.float64, device="cuda")
    with pytest.raises(N.GnaError) as e:
        api.chi2_noalloc(E, E, [1.0], p, d, 1.0)
    assert e.value.code == N.GNA_ESHAPE
    E2 = torch.ones(17, 1024 * 1024, dtype=torch.float64, device="cuda")  # 17 x 1024 tiles > 16384
    with pytest.raises(N.GnaError) as e:
        api.chi2_noalloc(E2, E2, [1.0], p, d[:17], 1.0)
    assert e.value.code == N.GNA_ESHAPE
