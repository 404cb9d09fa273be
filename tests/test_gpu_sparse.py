"""Sparse A (CSR) through the C ABI against the FP64 oracle's CSR code path.

Inputs: uniformly placed nonzeros with values in (0, 1] (the recipe of the
sparse workload), rounded to FP32 for both sides.  Tolerances as for the
dense FP32 path: products within 2 K u (|A| |B|) with K the number of
nonzeros in the row/column; whole FP32 runs within 1e-6 in the relative
residual."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module")
def ax():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf

    return aunmf.Handle()


def sparse_problem(m, n, density, k, seed):
    indptr, indices, data = synth.sparse_uniform(m, n, density, seed=seed)
    data = data.astype(np.float32).astype(np.float64)
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return (indptr, indices, data), r32(W0), r32(H0)


def dev_csr(csr, shape):
    from paper_1609_09154_gb300 import aunmf

    indptr, indices, data = csr
    t = (torch.as_tensor(indptr, device="cuda"), torch.as_tensor(indices, device="cuda"),
         torch.as_tensor(data.astype(np.float32), device="cuda"))
    return aunmf.csr_matrix(*t, shape), t


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,n,density,k", [(3000, 2000, 0.01, 50), (500, 700, 0.05, 1),
                                            (257, 33, 0.3, 100), (64, 4000, 0.002, 17),
                                            (900, 600, 0.02, 300)])
def test_sparse_products(ax, m, n, density, k):
    csr, W, H = sparse_problem(m, n, density, k, seed=m + k)
    M, keep = dev_csr(csr, (m, n))
    S = sp.csr_matrix((csr[2], csr[1], csr[0]), shape=(m, n))
    Mo = orc.Matrix(csr=csr, shape=(m, n))
    PW = host(ax.aht(M, dev(H)))
    PH = host(ax.wta(M, dev(W)))
    absS = abs(S)
    nz_row = np.diff(csr[0]).max()
    nz_col = np.bincount(csr[1], minlength=n).max()
    tol_w = 2 * max(nz_row, 1) * U32 * (absS @ np.abs(H).T) + 1e-30
    tol_h = 2 * max(nz_col, 1) * U32 * (np.abs(W).T @ absS) + 1e-30
    assert (np.abs(PW - orc.aht(Mo, H)) <= tol_w).all()
    assert (np.abs(PH - orc.wta(Mo, W)) <= tol_h).all()


@pytest.mark.parametrize("algo", ["mu", "hals", "abpp"])
def test_sparse_run_matches_oracle(ax, algo):
    m, n, k = 4000, 3000, 20
    csr, W0, H0 = sparse_problem(m, n, 0.01, k, seed=77)
    M, keep = dev_csr(csr, (m, n))
    ref = orc.nmf_run(orc.Matrix(csr=csr, shape=(m, n)), k, algo, 30, W0, H0)
    assert ref["rc"] == 0
    W, H, rel, info = ax.run(M, k, algo, 30, dev(W0), dev(H0))
    assert np.all(np.abs(rel - ref["relres"]) <= 1e-6), np.abs(rel - ref["relres"]).max()


def test_sparse_empty_rows_and_columns(ax):
    """Rows and columns without nonzeros (an all-zero row of A gives a zero
    row of A H^T; MU keeps it zero, HALS/ABPP project it to zero)."""
    m, n, k = 300, 200, 5
    csr, W0, H0 = sparse_problem(m, n, 0.02, k, seed=4)
    indptr, indices, data = csr
    keep_rows = np.arange(m) % 7 != 0
    S = sp.csr_matrix((data, indices, indptr), shape=(m, n)).toarray()
    S[~keep_rows] = 0.0
    S[:, ::9] = 0.0
    S = sp.csr_matrix(S)
    csr2 = (S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    M, keep = dev_csr(csr2, (m, n))
    for algo in ("mu", "hals", "abpp"):
        ref = orc.nmf_run(orc.Matrix(csr=csr2, shape=(m, n)), k, algo, 10, W0, H0)
        W, H, rel, info = ax.run(M, k, algo, 10, dev(W0), dev(H0))
        assert np.all(np.abs(rel - ref["relres"]) <= 1e-6)


def test_sparse_run_deterministic(ax):
    m, n, k = 5000, 4000, 16
    csr, W0, H0 = sparse_problem(m, n, 0.005, k, seed=8)
    M, keep = dev_csr(csr, (m, n))
    W1, H1, r1, _ = ax.run(M, k, "hals", 10, dev(W0), dev(H0))
    W2, H2, r2, _ = ax.run(M, k, "hals", 10, dev(W0), dev(H0))
    assert torch.equal(W1, W2) and torch.equal(H1, H2) and np.array_equal(r1, r2)


def powerlaw_problem(m, n, nnz, k, seed):
    """Power-law row and column degrees (hub columns with thousands of
    entries next to empty ones), from the same generator as the large sparse
    benchmark, on the CPU."""
    rp, ci, v = synth.sparse_powerlaw_torch(m, n, nnz, seed=seed, device="cpu")
    csr = (rp.numpy().astype(np.int64), ci.numpy().astype(np.int32),
           v.numpy().astype(np.float32).astype(np.float64))
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return csr, r32(W0), r32(H0)


@pytest.mark.parametrize("m,n,nnz,k", [(20000, 15000, 200000, 50), (3000, 50000, 150000, 17)])
def test_sparse_powerlaw_products(ax, m, n, nnz, k):
    """Both products on skewed degrees: W^T A goes through the CSC copy, whose
    columns (a radix sort by column of the CSR order) must list their rows in
    ascending order for the sums to come out as the oracle's."""
    csr, W, H = powerlaw_problem(m, n, nnz, k, seed=m + nnz)
    assert np.bincount(csr[1], minlength=n).max() > 50 * csr[1].size / n  # a hub column
    M, keep = dev_csr(csr, (m, n))
    S = sp.csr_matrix((csr[2], csr[1], csr[0]), shape=(m, n))
    Mo = orc.Matrix(csr=csr, shape=(m, n))
    PW = host(ax.aht(M, dev(H)))
    PH = host(ax.wta(M, dev(W)))
    absS = abs(S)
    nz_row = np.diff(csr[0]).max()
    nz_col = np.bincount(csr[1], minlength=n).max()
    tol_w = 2 * max(nz_row, 1) * U32 * (absS @ np.abs(H).T) + 1e-30
    tol_h = 2 * max(nz_col, 1) * U32 * (np.abs(W).T @ absS) + 1e-30
    assert (np.abs(PW - orc.aht(Mo, H)) <= tol_w).all()
    assert (np.abs(PH - orc.wta(Mo, W)) <= tol_h).all()


@pytest.mark.parametrize("algo", ["mu", "hals"])
def test_sparse_powerlaw_run_matches_oracle(ax, algo):
    m, n, k = 20000, 15000, 20
    csr, W0, H0 = powerlaw_problem(m, n, 200000, k, seed=91)
    M, keep = dev_csr(csr, (m, n))
    ref = orc.nmf_run(orc.Matrix(csr=csr, shape=(m, n)), k, algo, 20, W0, H0)
    assert ref["rc"] == 0
    W, H, rel, info = ax.run(M, k, algo, 20, dev(W0), dev(H0))
    assert np.all(np.abs(rel - ref["relres"]) <= 1e-6), np.abs(rel - ref["relres"]).max()


def test_sparse_long_rows_are_split(ax):
    """A row of 7000 and a column of 9000 nonzeros, longer than the 4096 a
    warp takes alone: both products split them into chunks over several warps
    (partials added in chunk order).  Products entry by entry and a HALS run
    against the oracle, and the run is repeatable bit for bit."""
    m, n, k = 9000, 7000, 24
    S = sp.random(m, n, density=0.002, format="lil", random_state=12, dtype=np.float64)
    g = np.random.default_rng(12)
    S[37, :] = g.random(n) + 0.01
    S[:, 4242] = (g.random(m) + 0.01)[:, None]
    S = S.tocsr()
    S.sort_indices()
    csr = (S.indptr.astype(np.int64), S.indices.astype(np.int32),
           S.data.astype(np.float32).astype(np.float64))
    W0, H0 = synth.init_factors(m, n, k, seed=12)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    W0, H0 = r32(W0), r32(H0)
    M, keep = dev_csr(csr, (m, n))
    Mo = orc.Matrix(csr=csr, shape=(m, n))
    absS = abs(sp.csr_matrix((csr[2], csr[1], csr[0]), shape=(m, n)))
    tol_w = 2 * n * U32 * (absS @ np.abs(H0).T) + 1e-30
    tol_h = 2 * m * U32 * (np.abs(W0).T @ absS) + 1e-30
    assert (np.abs(host(ax.aht(M, dev(H0))) - orc.aht(Mo, H0)) <= tol_w).all()
    assert (np.abs(host(ax.wta(M, dev(W0))) - orc.wta(Mo, W0)) <= tol_h).all()
    ref = orc.nmf_run(Mo, k, "hals", 10, W0, H0)
    W1, H1, r1, _ = ax.run(M, k, "hals", 10, dev(W0), dev(H0))
    W2, H2, r2, _ = ax.run(M, k, "hals", 10, dev(W0), dev(H0))
    assert np.all(np.abs(r1 - ref["relres"]) <= 1e-6), np.abs(r1 - ref["relres"]).max()
    assert torch.equal(W1, W2) and torch.equal(H1, H2) and np.array_equal(r1, r2)


def test_gather_probe_runs_and_checks_its_arguments():
    """The gather-roof kernel (a measurement, not a step of the method) runs
    on a product's index stream and rejects a leading dimension that is not
    a multiple of 4 or a rank above 64, launching nothing then."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf

    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    idx = torch.randint(0, 5000, (100_003,), device="cuda", dtype=torch.int32, generator=g)
    X = torch.rand((5000, 52), device="cuda", generator=g)
    sink = torch.zeros(1, device="cuda")
    aunmf.probe_gather(idx, X, 50, sink)
    torch.cuda.synchronize()
    assert float(sink) == 0.0
    with pytest.raises(aunmf.AunmfError) as e:
        aunmf.probe_gather(idx, torch.rand((5000, 50), device="cuda"), 50, sink)
    assert e.value.code == aunmf.E_INVAL
    with pytest.raises(aunmf.AunmfError) as e:
        aunmf.probe_gather(idx, torch.rand((5000, 68), device="cuda"), 65, sink)
    assert e.value.code == aunmf.E_INVAL
