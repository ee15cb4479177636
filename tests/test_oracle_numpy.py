"""A second, independently written implementation of the oracle's
definitions in vectorised NumPy (no shared code, no C): the recurrence
matrix by broadcasting and the run lengths of every diagonal and column by
differencing padded 0/1 arrays.  It must reproduce the C oracle's three
histograms and recurrence count exactly for series of up to 2,000 points,
every norm and several Theiler windows."""
import numpy as np
import pytest

import oracle
import synth


def _matrix(s, m, tau, eps, norm, w):
    n = len(s) - (m - 1) * tau
    X = np.stack([s[k * tau:k * tau + n] for k in range(m)], axis=1)
    D = X[:, None, :] - X[None, :, :]
    if norm == 0:
        d = np.abs(D).max(axis=2)
    elif norm == 2:
        d = np.zeros((n, n))
        for k in range(m):              # left to right, as the definition adds
            d = d + np.abs(D[:, :, k])
    else:
        d = np.zeros((n, n))
        for k in range(m):
            d = d + D[:, :, k] * D[:, :, k]
        d = np.sqrt(d)
    i, j = np.indices((n, n))
    return (d <= eps) & (np.abs(i - j) >= w)


def _runs(lines, n):
    """Histogram of the lengths of the runs of 1s in each 1-D 0/1 array."""
    h = np.zeros(n + 1, np.uint64)
    for a in lines:
        p = np.concatenate([[0], a.astype(np.int8), [0]])
        dd = np.diff(p)
        lengths = np.nonzero(dd == -1)[0] - np.nonzero(dd == 1)[0]
        np.add.at(h, lengths, 1)
    return h


def _histograms(R):
    n = R.shape[0]
    diags = [np.diagonal(R, k) for k in range(-(n - 1), n)]
    cols = [R[:, j] for j in range(n)]
    return _runs(diags, n), _runs(cols, n), _runs([~c for c in cols], n), int(R.sum())


@pytest.mark.parametrize("gen,N", [("logistic", 600), ("ar1", 1200), ("lorenz", 2000)])
@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 3])
def test_numpy_reimplementation_matches(gen, N, norm, w):
    s = {"logistic": lambda: synth.logistic(N, 4), "ar1": lambda: synth.ar1(N, 5, 0.9),
         "lorenz": lambda: synth.lorenz_x(N, 6)}[gen]()
    m, tau, eps = 3, 2, (0.08 if gen == "logistic" else 0.5)
    R = _matrix(s, m, tau, eps, norm, w)
    hd, hv, hw, rp = _histograms(R)
    r = oracle.rqa(s, oracle.Settings(m=m, tau=tau, eps=eps, norm=norm, theiler=w))
    assert r["rp"] == rp
    assert np.array_equal(r["hd"], hd)
    assert np.array_equal(r["hv"], hv)
    assert np.array_equal(r["hw"], hw)
