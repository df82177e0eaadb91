"""Seeded synthetic workloads (inputs only; no step of the method lives here).

Five workloads, each named by what it is and its sizes:

* ``reactor_200x50``       200 bins in 1.8-12 MeV x 50 Gauss-Legendre nodes,
                           L = 52.5 km, Pearson chi^2, one parameter point.
* ``reactor8_1000x16384``  1000 bins in 0.5-15 MeV x 16384 nodes, 8 baselines
                           drawn in 0.5-60 km (weights 1/L^2), parameters
                           perturbed by +-5 %, Poisson chi^2.
* ``nuisance_1000x4096``   the same baselines and point at 4096 nodes/bin plus
                           1000 per-bin normalisation nuisances (sigma 2 %).
* ``scan_64x64_500bins``   64 x 64 grid in (sin^2 theta13, dm2_32), 500 bins in
                           0.5-5 GeV at L = 810 km, each point its own
                           Gauss-Legendre order (2^14..2^18 nodes in total,
                           log-uniform), spectrum evaluated with E in GeV.
* ``fits_16384x1000``      16384 Poisson pseudo-datasets of 1000 bins from the
                           8-baseline reactor model on 1000 x 262 nodes,
                           20 Levenberg-Marquardt iterations each.

Random draws (baselines, perturbations, nuisances, grid sizes, Poisson data)
come from ``numpy.random.default_rng(seed)``.  Poisson data need the expected
counts, which the caller supplies (the oracle in tests, the library itself in
the benchmark); this module only draws from them.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

# Oscillation parameters of the reference point (normal ordering):
# sin^2 theta12, sin^2 theta13, dm2_21 [eV^2], dm2_32 [eV^2].
TRUTH = (0.307, 0.0218, 7.53e-5, 2.44e-3)
TOTAL_EVENTS = 1e5
NUISANCE_SIGMA = 0.02

PEARSON = 0
POISSON = 1


@dataclass
class Workload:
    name: str
    edges: np.ndarray                 # [nbins+1] MeV
    nodes_per_bin: int                # Gauss-Legendre order (uniform grids)
    L: np.ndarray                     # [nL] km
    theta: np.ndarray                 # [npts, 4] evaluation points
    kind: int                         # PEARSON or POISSON
    truth: np.ndarray = field(default_factory=lambda: np.array(TRUTH))
    e_scale: float = 1.0              # spectrum evaluated at E_MeV * e_scale
    eta: Optional[np.ndarray] = None  # [nbins] nuisance values
    sigma_eta: float = 0.0
    node_counts: Optional[np.ndarray] = None  # [npts] per-point orders (uneven grids)
    data_seed: int = 0
    n_datasets: int = 1               # pseudo-datasets (fits)
    fit_iters: int = 0

    @property
    def nbins(self) -> int:
        return self.edges.size - 1

    @property
    def npts(self) -> int:
        return self.theta.shape[0]

    @property
    def nL(self) -> int:
        return self.L.size

    def points_per_eval(self) -> int:
        """Probability evaluations (node x baseline x parameter point) per eval."""
        if self.node_counts is not None:
            return int(self.nbins * self.node_counts.sum() * self.nL)
        return int(self.nbins * self.nodes_per_bin * self.nL * self.npts)


def _reactor8_draws():
    rng = np.random.default_rng(1)
    L = rng.uniform(0.5, 60.0, 8)
    u = rng.uniform(-0.05, 0.05, 4)
    return L, np.array(TRUTH) * (1.0 + u)


def reactor_200x50() -> Workload:
    return Workload("reactor_200x50", np.linspace(1.8, 12.0, 201), 50, np.array([52.5]),
                    np.array([TRUTH]), PEARSON, data_seed=0)


def reactor8_1000x16384() -> Workload:
    L, theta = _reactor8_draws()
    return Workload("reactor8_1000x16384", np.linspace(0.5, 15.0, 1001), 16384, L, theta[None, :],
                    POISSON, data_seed=11)


def nuisance_1000x4096() -> Workload:
    L, theta = _reactor8_draws()
    eta = np.random.default_rng(2).normal(0.0, NUISANCE_SIGMA, 1000)
    return Workload("nuisance_1000x4096", np.linspace(0.5, 15.0, 1001), 4096, L, theta[None, :],
                    POISSON, eta=eta, sigma_eta=NUISANCE_SIGMA, data_seed=12)


def scan_grid(n13=64, n32=64):
    s13 = np.linspace(0.015, 0.03, n13)
    dm32 = np.linspace(2.3e-3, 2.6e-3, n32)
    S, D = np.meshgrid(s13, dm32, indexing="ij")
    th = np.empty((n13 * n32, 4))
    th[:, 0] = TRUTH[0]
    th[:, 1] = S.ravel()
    th[:, 2] = TRUTH[2]
    th[:, 3] = D.ravel()
    return th


def scan_node_counts(npts: int, nbins: int = 500, seed: int = 3) -> np.ndarray:
    """Per-point Gauss-Legendre order: N_p = 2^U(14,18) nodes in total."""
    rng = np.random.default_rng(seed)
    Np = 2.0 ** rng.uniform(14.0, 18.0, npts)
    return np.maximum(1, np.rint(Np / nbins)).astype(np.int64)


SCAN_TRUTH_NODES = 524  # round(2^18 / 500): the order of the scan's truth model


def scan_64x64_500bins(n13=64, n32=64) -> Workload:
    th = scan_grid(n13, n32)
    counts = scan_node_counts(th.shape[0])
    return Workload("scan_64x64_500bins", np.linspace(500.0, 5000.0, 501), 0, np.array([810.0]), th, POISSON,
                    e_scale=1e-3, node_counts=counts, data_seed=13)


def fits_16384x1000(n_datasets=16384) -> Workload:
    L, theta = _reactor8_draws()
    th = np.repeat(theta[None, :], n_datasets, axis=0)
    return Workload("fits_16384x1000", np.linspace(0.5, 15.0, 1001), 262, L, th, POISSON, data_seed=4,
                    n_datasets=n_datasets, fit_iters=20)


ALL = {
    "reactor_200x50": reactor_200x50,
    "reactor8_1000x16384": reactor8_1000x16384,
    "nuisance_1000x4096": nuisance_1000x4096,
    "scan_64x64_500bins": scan_64x64_500bins,
    "fits_16384x1000": fits_16384x1000,
}


def shrink(w: Workload, nbins: Optional[int] = None, nodes: Optional[int] = None, npts: Optional[int] = None,
           nL: Optional[int] = None) -> Workload:
    """A smaller copy of a workload with the same structure (for parity tests)."""
    edges = w.edges
    if nbins is not None:
        edges = np.linspace(w.edges[0], w.edges[-1], nbins + 1)
    theta = w.theta if npts is None else w.theta[:npts]
    counts = w.node_counts if (w.node_counts is None or npts is None) else w.node_counts[:npts]
    eta = w.eta if (w.eta is None or nbins is None) else w.eta[:nbins]
    L = w.L if nL is None else w.L[:nL]
    return replace(w, edges=edges, nodes_per_bin=w.nodes_per_bin if nodes is None else nodes, theta=theta,
                   node_counts=counts, eta=eta, L=L,
                   n_datasets=min(w.n_datasets, theta.shape[0]))


def poisson_data(mu: np.ndarray, seed: int) -> np.ndarray:
    """Poisson draws with means mu (any shape), as float64."""
    return np.random.default_rng(seed).poisson(np.asarray(mu, dtype=np.float64)).astype(np.float64)


def pseudo_datasets(mu: np.ndarray, n: int, seed: int) -> np.ndarray:
    """n Poisson pseudo-datasets [n][nbins] drawn around one expected spectrum."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(mu, dtype=np.float64)[None, :], size=(n, mu.size)).astype(np.float64)
