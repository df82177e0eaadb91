"""Argument validation of the C ABI, on the host (no GPU needed): every check
below returns before the library touches a device, so a bad configuration is
refused with the documented status on any machine."""
import ctypes

import numpy as np
import pytest

OK, EINVAL, ESHAPE = 0, 1, 2
DBL = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def N():
    from paper_1804_07682_gb300 import _native, build

    build.build()
    return _native


def desc(N, **kw):
    edges = np.linspace(1.8, 8.0, 11)
    L = np.array([52.5, 53.1])
    d = dict(nbins=10, edges=edges, nodes_per_bin=8, npts=1, node_counts=None, nL=2, L=L, Lweight=None, norm=1.0,
             e_scale=1.0, prec=2, kind=1, max_datasets=0, flags=0, alpha=0, beta=0, anti=0)
    d.update(kw)
    keep = [d["edges"], d["L"], d["Lweight"], d["node_counts"]]
    D = N.GnaPlanDesc()
    D.nbins = d["nbins"]
    D.edges = d["edges"].ctypes.data_as(DBL) if d["edges"] is not None else None
    D.nodes_per_bin = d["nodes_per_bin"]
    D.npts = d["npts"]
    if d["node_counts"] is not None:
        D.node_counts = d["node_counts"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    D.nL = d["nL"]
    D.L = d["L"].ctypes.data_as(DBL) if d["L"] is not None else None
    if d["Lweight"] is not None:
        D.Lweight = d["Lweight"].ctypes.data_as(DBL)
    D.norm, D.e_scale, D.prec, D.kind = d["norm"], d["e_scale"], d["prec"], d["kind"]
    D.max_datasets, D.flags = d["max_datasets"], d["flags"]
    D.alpha, D.beta, D.anti = d["alpha"], d["beta"], d["anti"]
    return D, keep


@pytest.mark.parametrize("kw,code", [
    (dict(nbins=0), ESHAPE),
    (dict(npts=0), ESHAPE),
    (dict(nL=0), ESHAPE),
    (dict(nL=17), ESHAPE),
    (dict(edges=None), EINVAL),
    (dict(L=None), EINVAL),
    (dict(edges=np.array([1.8, 2.0, 2.0, 3.0, 4, 5, 6, 7, 8, 9, 10])), EINVAL),   # not strictly increasing
    (dict(edges=np.linspace(-1.0, 8.0, 11)), EINVAL),                             # E <= 0
    (dict(L=np.array([52.5, 0.0])), EINVAL),
    (dict(Lweight=np.array([1.0, -0.5])), EINVAL),
    (dict(Lweight=np.array([0.0, 0.0])), EINVAL),                                  # weights normalised by their sum
    (dict(Lweight=np.array([1.0, float("inf")])), EINVAL),
    (dict(L=np.array([52.5, float("inf")])), EINVAL),
    (dict(nodes_per_bin=0), ESHAPE),
    (dict(nodes_per_bin=65537), ESHAPE),
    (dict(npts=3, node_counts=np.array([4, 0, 9], dtype=np.int32)), ESHAPE),
    (dict(norm=0.0), EINVAL),
    (dict(norm=float("nan")), EINVAL),
    (dict(prec=3), EINVAL),
    (dict(kind=2), EINVAL),
    # any-channel plans: flavours 0..2, anti 0 or 1, up to 8 baselines, no
    # split mapping or plain chain
    (dict(flags=16, alpha=3), EINVAL),
    (dict(flags=16, beta=-1), EINVAL),
    (dict(flags=16, anti=2), EINVAL),
    (dict(flags=16 | 2), EINVAL),
    (dict(flags=16 | 1), EINVAL),
    (dict(flags=16, nL=9, L=np.linspace(1.0, 9.0, 9)), ESHAPE),
])
def test_plan_descriptor_is_checked_on_the_host(N, kw, code):
    D, keep = desc(N, **kw)
    out = ctypes.c_void_p(123)
    assert N.lib().gna_plan_create(ctypes.byref(out), ctypes.byref(D), None) == code
    assert out.value is None  # no plan is handed out on failure
    del keep


def test_oscprob_arguments(N):
    L = np.array([52.5])
    p = N.GnaOsc(0.307, 0.0218, 7.53e-5, 2.44e-3)
    f = N.lib().gna_oscprob_ee_staged
    Lp = L.ctypes.data_as(DBL)
    assert f(None, 0, Lp, 1, ctypes.byref(p), 0, None, 0, None) == OK      # nothing to do
    assert f(None, 10, Lp, 1, ctypes.byref(p), 0, None, -1, None) == ESHAPE  # chunk < 0
    assert f(None, -1, Lp, 1, ctypes.byref(p), 0, None, 0, None) == ESHAPE
    assert f(None, 10, Lp, 0, ctypes.byref(p), 0, None, 0, None) == ESHAPE
    assert f(None, 10, Lp, 1, ctypes.byref(p), 9, None, 0, None) == EINVAL  # unknown precision
    assert f(None, 10, Lp, 1, ctypes.byref(p), 0, None, 0, None) == EINVAL  # NULL buffers
    g = N.lib().gna_oscprob
    q = N.GnaOscFull(0.307, 0.0218, 0.545, 1.2 * np.pi, 7.53e-5, 2.44e-3)
    assert g(None, 0, Lp, 1, 1, 0, 0, ctypes.byref(q), 0, None, None) == OK
    assert g(None, 10, Lp, 1, 3, 0, 0, ctypes.byref(q), 0, None, None) == EINVAL  # flavour out of range
    assert g(None, 10, Lp, 1, 0, -1, 0, ctypes.byref(q), 0, None, None) == EINVAL
    bad = N.GnaOscFull(1.5, 0.0218, 0.545, 0.0, 7.53e-5, 2.44e-3)                # s2 > 1
    assert g(None, 10, Lp, 1, 1, 0, 0, ctypes.byref(bad), 0, None, None) == EINVAL
    assert g(None, 10, Lp, 17, 1, 0, 0, ctypes.byref(q), 0, None, None) == ESHAPE


def test_pseudo_data_arguments(N):
    f = N.lib().gna_poisson_datasets
    mu = np.array([3.0, 40.0])
    mp = mu.ctypes.data_as(DBL)
    assert f(mp, 0, 5, 1, ctypes.c_void_p(8), None) == ESHAPE
    assert f(mp, 2, -1, 1, ctypes.c_void_p(8), None) == ESHAPE
    assert f(None, 2, 5, 1, ctypes.c_void_p(8), None) == EINVAL
    assert f(mp, 2, 5, 1, None, None) == EINVAL
    for bad in (-1.0, 2e7, float("nan")):
        m2 = np.array([3.0, bad])
        assert f(m2.ctypes.data_as(DBL), 2, 5, 1, ctypes.c_void_p(8), None) == EINVAL
    assert f(mp, 2, 0, 1, None, None) == OK  # no data sets: validated, nothing drawn


def test_any_channel_calls_without_a_plan(N):
    o = N.GnaOutputs(None, None, None, None, None)
    assert N.lib().gna_chain_eval_general(None, None, None, 0.0, None, 0, ctypes.byref(o), None) == EINVAL
    assert N.lib().gna_plan_autotune_general(None, None, None, 0, ctypes.byref(o), 1, None) == EINVAL


def test_noalloc_wrapper_refuses_bad_arguments_before_any_launch():
    # chi2_noalloc checks dtypes, shapes and devices before it reaches the
    # library: a float32 or misshapen array, a short data row or output, or a
    # tensor off the device would otherwise be read or written out of bounds
    torch = pytest.importorskip("torch")
    from paper_1804_07682_gb300 import api

    f64 = torch.float64
    E = torch.ones(5, 7, dtype=f64)
    W = torch.ones(5, 7, dtype=f64)
    p = torch.zeros(1, 4, dtype=f64)
    d = torch.ones(5, dtype=f64)
    bad = {
        "E float32": dict(E=E.float()),
        "E 1-D": dict(E=torch.ones(35, dtype=f64)),
        "W float32": dict(W=W.float()),
        "W shaped unlike E": dict(W=torch.ones(5, 6, dtype=f64)),
        "params of 3": dict(params=torch.zeros(1, 3, dtype=f64)),
        "params float32": dict(params=p.float()),
        "data short": dict(data=torch.ones(4, dtype=f64)),
        "data float32": dict(data=d.float()),
        "Lweight per baseline": dict(L=[52.5, 30.0], Lweight=[1.0]),
        "out without chi2": dict(out={"grad": torch.empty(4, dtype=f64)}),
        "out mu short": dict(out={"chi2": torch.empty(1, dtype=f64), "mu": torch.empty(4, dtype=f64)}),
        "out grad short": dict(out={"chi2": torch.empty(1, dtype=f64), "grad": torch.empty(3, dtype=f64)}),
        "out chi2 empty": dict(out={"chi2": torch.empty(0, dtype=f64)}),
        "out unknown": dict(out={"chi2": torch.empty(1, dtype=f64), "spectra": torch.empty(5, dtype=f64)}),
    }
    for what, kw in bad.items():
        args = dict(E=E, W=W, L=[52.5], params=p, data=d, norm=1.0)
        args.update(kw)
        with pytest.raises(ValueError) as e:
            api.chi2_noalloc(**args)
        assert "CUDA" not in str(e.value), what  # refused for its dtype or shape, not its device
    # every dtype and shape right, but host tensors: refused for the device
    with pytest.raises(ValueError, match="CUDA tensors"):
        api.chi2_noalloc(E, W, [52.5], p, d, 1.0)


def test_grad_scale_refuses_bad_arguments(N):
    L = N.lib()
    s = ctypes.c_double(2.0)
    assert L.gna_grad_scale(None, 4, None, 0, None, None) == EINVAL  # no scale factor
    assert L.gna_grad_scale(None, 4, None, 0, ctypes.addressof(s), None) == EINVAL  # a = NULL, na = 4
    assert L.gna_grad_scale(None, 0, None, 3, ctypes.addressof(s), None) == EINVAL  # b = NULL, nb = 3
    buf = (ctypes.c_double * 4)()
    assert L.gna_grad_scale(ctypes.addressof(buf), -1, None, 0, ctypes.addressof(s), None) == EINVAL
    assert L.gna_grad_scale(ctypes.addressof(buf), 4, ctypes.addressof(buf), -2, ctypes.addressof(s), None) == EINVAL
    # host memory no device can reach (here: no GPU at all) is refused before any launch
    assert L.gna_grad_scale(ctypes.addressof(buf), 4, None, 0, ctypes.addressof(s), None) == EINVAL
    # nothing to scale: no launch, success
    assert L.gna_grad_scale(None, 0, None, 0, ctypes.addressof(s), None) == OK
