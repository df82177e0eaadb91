"""The library's host-side mixing matrix (gna_pmns, built from the written-out
elements of R23 U13(delta) R12) against the oracle's (products of the three
rotation matrices): two independent constructions of the same matrix.  CPU only."""
import numpy as np
import pytest

import oracle

CASES = [(0.307, 0.0218, 0.545, 1.2 * np.pi), (0.3, 0.02, 0.5, 0.0), (0.0, 0.0, 0.0, 0.7), (1.0, 1.0, 1.0, -2.1),
         (0.25, 0.1, 0.6, np.pi / 2)]


@pytest.fixture(scope="module")
def api():
    from paper_1804_07682_gb300 import api as _api
    from paper_1804_07682_gb300 import build

    build.build()
    return _api


@pytest.mark.parametrize("s12,s13,s23,delta", CASES)
def test_pmns_matches_oracle(api, s12, s13, s23, delta):
    U = api.pmns((s12, s13, s23, delta, 7.5e-5, 2.4e-3))
    ref = oracle.pmns(s12, s13, s23, delta)
    assert np.abs(U - ref).max() < 1e-15
    assert np.abs(U @ U.conj().T - np.eye(3)).max() < 1e-15


def test_pmns_rejects_bad_angles(api):
    from paper_1804_07682_gb300 import _native as N

    with pytest.raises(N.GnaError):
        api.pmns((1.5, 0.02, 0.5, 0.0, 7.5e-5, 2.4e-3))
