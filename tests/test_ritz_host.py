"""Condition-number estimates from PCG coefficients (Sec. 4.5): the
library's host routines against the oracle's tridiagonal matrix and numpy's
dense symmetric eigensolver.  No GPU: these are host functions."""
import numpy as np
import pytest

from oracle import spectrum


@pytest.fixture(scope="module")
def spai(spai_lib):
    return spai_lib


@pytest.mark.parametrize("k", [1, 2, 7, 60, 450])
def test_ritz_extremes_and_kaporin_match_dense(spai, k):
    rng = np.random.default_rng(k)
    alpha = rng.uniform(0.05, 2.0, size=k)
    beta = rng.uniform(0.01, 0.99, size=max(k - 1, 0))
    t = spectrum.lanczos_tridiagonal(alpha, beta)
    lam = np.linalg.eigvalsh(t)
    lo, hi = spai.ritz_extremes(alpha, beta)
    assert lo == pytest.approx(lam[0], rel=1e-12, abs=1e-14 * abs(lam).max())
    assert hi == pytest.approx(lam[-1], rel=1e-12)
    if lam[0] > 0:
        m = min(k, 400)
        th, v = np.linalg.eigh(spectrum.lanczos_tridiagonal(alpha[:m], beta[: m - 1]))
        w = v[0] ** 2
        want = (w @ th) / np.exp(w @ np.log(th))
        assert spai.ritz_kaporin(alpha, beta) == pytest.approx(want, rel=1e-8)


def test_ritz_rejects_bad_coefficients(spai):
    with pytest.raises(spai.SpaiError):
        spai.ritz_extremes([1.0, -1.0], [0.5])
    with pytest.raises(spai.SpaiError):
        spai.ritz_kaporin([], [])
