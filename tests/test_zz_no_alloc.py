"""The allocation-free evaluation (gna_chain_eval_noalloc) against the plan-based
one (gna_chain_eval), through the C ABI.

gna_chain_eval_noalloc exists for callers that cannot allocate device memory
(a pool or arena they do not own, a host framework that forbids cudaMalloc);
it works in a fixed array inside the library that every call shares.  Two
calls in a row must both match the plan-based result, which also shows that
each call starts from cleared counters.  This file is collected last and is
self-contained, so it passes alone in a fresh process as well as after the
rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_07682_gb300 import workloads as wl
from refs import Case, chi2_err_bound, normrel, rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

TOL = 1e-6   # mixed-precision tolerance of the parity tests (mu, scaled chi^2)
GTOL = 1e-4  # gradient sanity bound of the parity tests


def node_arrays(w):
    """E and W on the bin-major Gauss-Legendre grid (numpy's leggauss rule)."""
    x, wt = np.polynomial.legendre.leggauss(w.nodes_per_bin)
    a, b = w.edges[:-1, None], w.edges[1:, None]
    half, mid = 0.5 * (b - a), 0.5 * (a + b)
    E = mid + half * x[None, :]
    Es = E * w.e_scale
    W = half * wt[None, :] * np.exp(0.87 - 0.16 * Es - 0.091 * Es * Es)
    return E, W


@pytest.mark.parametrize("name", ["reactor_200x50", "reactor8_40x3000"])
def test_noalloc_matches_plan_twice(name):
    from paper_1804_07682_gb300 import api

    w = wl.reactor_200x50() if name == "reactor_200x50" else wl.shrink(wl.reactor8_1000x16384(), nbins=40, nodes=3000)
    case = Case(w)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    data = dev(case.data)
    params = dev(w.theta[:1])
    plan = api.Plan(w.edges, w.L, nodes_per_bin=w.nodes_per_bin, norm=case.N, e_scale=w.e_scale, prec="ff", kind=w.kind)
    ref = plan.eval(params, data, grad=True, mu=True)
    ref = {k: v[0].cpu().numpy() for k, v in ref.items()}
    E, W = node_arrays(w)
    E, W = dev(E), dev(W)
    results = []
    for _ in range(2):
        out = api.chi2_noalloc(E, W, w.L, params, data, case.N, kind=w.kind, grad=True, mu=True)
        torch.cuda.synchronize()
        results.append({k: v.cpu().numpy() for k, v in out.items()})
    scale = chi2_err_bound({"mu": ref["mu"], "chi2": float(ref["chi2"])}, case.data, w.kind)
    for r in results:
        assert abs(float(r["chi2"][0]) - float(ref["chi2"])) <= TOL * scale
        assert rel(r["mu"], ref["mu"]) < TOL
        assert normrel(r["grad"], ref["grad"]) < GTOL
    assert np.array_equal(results[0]["chi2"], results[1]["chi2"])
    assert np.array_equal(results[0]["mu"], results[1]["mu"])
    plan.close()


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
