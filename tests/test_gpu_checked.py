"""The checked build, libaunmf_check.so (-DAUNMF_CHECK): device code tests
every index it takes from data -- CSR / CSC structure and sorted positions,
gathered factor rows, BPP index lists, batched work items, TMA coordinates
-- records the site of a failing test and skips the access (see
aunmf_check_status in include/aunmf.h).  It stands in for a memory checker.

Each case runs a whole AU-NMF call through the checked library on the shapes
the parity tests use (ragged tiles, long sparse rows split into chunks, wide
ranks, batched problems), asserts that no check fired, and that the result
is the normal build's (the checks change no arithmetic: same bar as the
oracle parity, 1e-6 in the relative residual)."""
import numpy as np
import pytest

from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf, build

    build.build(check=True)
    aunmf.load(checked=True)
    assert aunmf.check_status(checked=True) == 0
    hc, hn = aunmf.Handle(checked=True), aunmf.Handle()
    yield aunmf, hc, hn
    hc.close()
    hn.close()


def dev(x, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=dtype), device="cuda")


def dense(m, n, k, seed):
    A, _, _ = synth.dense_lowrank(m, n, k, seed=seed)
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    return dev(A), dev(W0), dev(H0)


def _same(libs, run):
    aunmf, hc, hn = libs
    _, _, rc, ic = run(hc)
    assert aunmf.check_status(checked=True) == 0
    _, _, rn, _ = run(hn)
    assert np.abs(rc - rn).max() <= 1e-6
    return ic


@pytest.mark.parametrize("prec,k", [("fp32", 40), ("fp32", 20), ("tf32", 50), ("bf16", 50),
                                    ("tf32", 300)])
def test_checked_dense_hals(libs, prec, k):
    A = dense(700, 520, min(k, 50), seed=k)[0]
    W0, H0 = (dev(x) for x in synth.init_factors(700, 520, k, seed=k))
    _same(libs, lambda h: h.run(A, k, "hals", 4, W0, H0, prec=prec))


@pytest.mark.parametrize("prec,cold", [("fp32", False), ("tf32", False), ("fp32", True)])
def test_checked_dense_abpp(libs, prec, cold):
    A, W0, H0 = dense(1200, 900, 24, seed=31)
    _same(libs, lambda h: h.run(A, 24, "abpp", 5, W0, H0, prec=prec, bpp_cold_start=cold))


def test_checked_sparse_with_long_rows(libs):
    aunmf = libs[0]
    m, n, k = 300, 30000, 16
    indptr, indices, data = synth.sparse_uniform(m, n, 0.01, seed=5)
    # two rows past the chunking threshold (4096 nonzeros)
    rows = [np.sort(np.random.default_rng(1).choice(n, 6000, replace=False)),
            np.sort(np.random.default_rng(2).choice(n, 9000, replace=False))]
    lens = np.diff(indptr)
    cols = np.split(indices, np.cumsum(lens)[:-1])
    cols[7], cols[123] = rows[0].astype(np.int32), rows[1].astype(np.int32)
    lens = np.array([len(c) for c in cols])
    indptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    indices = np.concatenate(cols).astype(np.int32)
    data = np.random.default_rng(3).uniform(0.1, 1.0, indices.size).astype(np.float32)
    t = (dev(indptr, np.int64), dev(indices, np.int32), dev(data))
    M = aunmf.csr_matrix(*t, (m, n))
    W0, H0 = synth.init_factors(m, n, k, seed=6)
    W0, H0 = dev(W0), dev(H0)
    _same(libs, lambda h: h.run(M, k, "hals", 4, W0, H0, validate=True))


def test_checked_batched(libs):
    aunmf, hc, hn = libs
    ks = [8, 24, 40]
    probs = [dense(500 + 77 * i, 380 + 45 * i, k, seed=70 + i) for i, k in enumerate(ks)]
    As = [p[0] for p in probs]
    H0s = [p[2] for p in probs]
    _, _, rc, _ = hc.run_batched(As, ks, 4, H0s, prec="tf32")
    assert aunmf.check_status(checked=True) == 0
    _, _, rn, _ = hn.run_batched(As, ks, 4, H0s, prec="tf32")
    assert np.abs(rc - rn).max() <= 1e-6
