"""Oracle-side references for the parity tests: every input and expected
value here comes from the seeded generators and the FP64 oracle, never from
the CUDA path."""
from __future__ import annotations

import json
import os

import numpy as np

import oracle
from paper_1804_07682_gb300 import workloads as wl


class Case:
    """A workload instance with oracle-derived normalisation and data."""

    def __init__(self, w: wl.Workload, truth_nodes=None):
        self.w = w
        tn = truth_nodes if truth_nodes is not None else (w.nodes_per_bin or wl.SCAN_TRUTH_NODES)
        self.omega = oracle.baseline_weights(w.L)
        self.N = oracle.norm_for_total(w.edges, tn, w.L, w.truth, e_scale=w.e_scale)
        self.mu_truth = self.N * (self.omega @ oracle.binned(w.edges, tn, w.L, w.truth, w.e_scale))
        if w.n_datasets > 1:
            self.data = wl.pseudo_datasets(self.mu_truth, w.n_datasets, w.data_seed)
        else:
            self.data = wl.poisson_data(self.mu_truth, w.data_seed)

    def nodes_of(self, p):
        w = self.w
        return int(w.node_counts[p]) if w.node_counts is not None else w.nodes_per_bin

    def data_of(self, p):
        return self.data[p] if self.data.ndim == 2 else self.data

    def oracle_point(self, p, grad=True, theta=None):
        w = self.w
        th = w.theta[p] if theta is None else theta
        return oracle.chain(w.edges, self.nodes_of(p), w.L, th, self.N, self.data_of(p), w.kind, eta=w.eta,
                            sigma=w.sigma_eta, e_scale=w.e_scale, grad=grad)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def fit_sigma(r):
    """Statistical errors of the fitted parameters at an oracle evaluation r:
    the square roots of the diagonal of the inverse expected Fisher matrix
    sum_i (2 / mu_i) J_i J_i^T (the matrix the fitter's steps are built on)."""
    J = np.asarray(r["J"], dtype=np.float64)
    H = (J.T * (2.0 / np.asarray(r["mu"], dtype=np.float64))) @ J
    return np.sqrt(np.diag(np.linalg.inv(H)))


def normrel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def chi2_err_bound(ref, data, kind):
    """Scale of chi^2 errors implied by relative errors in mu: |d chi2| <=
    eps * sum_i |d chi2 / d mu_i| mu_i, so a 1e-6 gate on mu carries over to
    chi^2 as 1e-6 * max(chi2, sum_i |g_i| mu_i)."""
    mu = np.asarray(ref["mu"], dtype=np.float64)
    d = np.asarray(data, dtype=np.float64)
    g = (1 - d * d / (mu * mu)) if kind == 0 else 2 * (1 - d / mu)
    return max(abs(ref["chi2"]), float(np.sum(np.abs(g) * mu)))


_ERRLOG = os.environ.get("GNA_TEST_ERRLOG")


def log_err(tag, **vals):
    """Appends measured errors to the file named by $GNA_TEST_ERRLOG (if set),
    one JSON object per line, so that a test run can report the margins."""
    if not _ERRLOG:
        return
    with open(_ERRLOG, "a") as f:
        f.write(json.dumps(dict(tag=tag, **{k: float(v) for k, v in vals.items()})) + "\n")


def check_chi2(got, ref, data, kind, tol, tag="", plain=True):
    """chi^2 against the oracle at relative tolerance tol.  plain=False keeps
    only the scaled bound |d chi2| <= tol * max(chi2, sum_i |g_i| mu_i), for
    the cases whose chi^2 is small against that scale (a near-perfect fit of
    bins with very few nodes: their mixed-precision mu cannot average the
    per-node FP32 roundings down, and chi^2 amplifies them)."""
    r = abs(got - ref["chi2"]) / abs(ref["chi2"])
    scale = chi2_err_bound(ref, data, kind)
    log_err(tag, chi2_rel=r, chi2_scaled=abs(got - ref["chi2"]) / scale, amplification=scale / abs(ref["chi2"]))
    assert abs(got - ref["chi2"]) <= tol * scale, (tag, got, ref["chi2"], scale)
    if plain:
        assert r <= tol, (tag, "plain relative chi2", r, tol)
    return r
