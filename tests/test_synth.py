"""Synthetic input generators (host side, CPU): the power-law sparse matrix
that stands in for a web graph is a valid CSR (strictly increasing columns
within each row, no repeats, values in (0, 1]), is fixed by its seed, and has
the skew it is meant to have (hub columns far above the mean degree, and
empty rows and columns)."""
import numpy as np
import pytest

from paper_1609_09154_gb300 import synth

torch = pytest.importorskip("torch")


def _csr(m, n, nnz, seed):
    rp, ci, v = synth.sparse_powerlaw_torch(m, n, nnz, seed=seed, device="cpu")
    return rp.numpy(), ci.numpy(), v.numpy()


def test_powerlaw_csr_is_valid():
    m, n = 5000, 4000
    rp, ci, v = _csr(m, n, 60000, seed=5)
    assert rp.dtype == np.int64 and ci.dtype == np.int32 and v.dtype == np.float32
    assert rp[0] == 0 and rp[-1] == ci.size == v.size and (np.diff(rp) >= 0).all()
    assert ci.min() >= 0 and ci.max() < n
    for r in range(m):
        row = ci[rp[r]:rp[r + 1]]
        assert (np.diff(row) > 0).all()  # sorted, no repeated position
    assert (v > 0).all() and (v <= 1).all()


def test_powerlaw_is_fixed_by_its_seed():
    a = _csr(3000, 2000, 30000, seed=7)
    b = _csr(3000, 2000, 30000, seed=7)
    c = _csr(3000, 2000, 30000, seed=8)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[1], c[1])


def test_powerlaw_degrees_are_skewed():
    m, n, nnz = 20000, 15000, 200000
    rp, ci, _ = _csr(m, n, nnz, seed=9)
    col = np.bincount(ci, minlength=n)
    row = np.diff(rp)
    assert col.max() > 100 * col.mean()  # hub columns (degree ~ rank^-0.7)
    assert row.max() > 20 * row.mean()   # heavy rows (degree ~ rank^-0.5)
    assert (col == 0).any() and (row == 0).any()
    # repeats dropped: fewer positions than draws, but most draws kept
    assert 0.8 * nnz < ci.size <= nnz
