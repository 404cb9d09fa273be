"""Run options through the C ABI: input validation (aunmf_options.validate)
and BPP cold starts (aunmf_options.bpp_cold_start).

Validation (Sec. 2 poses NMF for A >= 0; the updates of Sec. 4 keep the
factors nonnegative from a nonnegative start): every malformed input here is
one that the validation kernels reject before any other kernel reads it --
a negative, NaN or infinite entry, or a CSR structure with a row pointer out
of order or range or a column index out of [0, n) or not increasing within
its row.  Valid input runs exactly as without the check.

Cold start (Sec. 4.3, SolveBPP): the NNLS problem of each row has one
solution when its Gram is positive definite, so starting every solve from
x = 0 reaches the same factors as the warm start (to the solver's rounding),
with more exchanges."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf

    return aunmf


def dev(x, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=dtype), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def problem(m, n, k, seed):
    A, _, _ = synth.dense_lowrank(m, n, k, seed=seed)
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return r32(A), r32(W0), r32(H0)


def _expect_inval(lib, fn):
    with pytest.raises(lib.AunmfError) as e:
        fn()
    assert e.value.code == lib.E_INVAL, (e.value.code, str(e.value))


@pytest.mark.parametrize("algo", ["hals", "abpp"])
def test_validate_passes_valid_input_unchanged(lib, algo):
    A, W0, H0 = problem(700, 500, 12, seed=3)
    h = lib.Handle()
    Ad = dev(A)
    W1, H1, r1, _ = h.run(Ad, 12, algo, 5, dev(W0), dev(H0))
    W2, H2, r2, _ = h.run(Ad, 12, algo, 5, dev(W0), dev(H0), validate=True)
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(host(W1), host(W2))
    np.testing.assert_array_equal(host(H1), host(H2))
    h.close()


@pytest.mark.parametrize("bad", [-1e-3, np.nan, np.inf])
def test_validate_rejects_a_bad_entry_of_A(lib, bad):
    A, W0, H0 = problem(300, 200, 8, seed=4)
    A[123, 77] = bad
    h = lib.Handle()
    _expect_inval(lib, lambda: h.run(dev(A), 8, "hals", 3, dev(W0), dev(H0), validate=True))
    # a pinned-host A through aunmf_run_host is checked the same way
    _expect_inval(lib, lambda: h.run_host(A.astype(np.float32), 8, "hals", 3,
                                          W0.astype(np.float32), H0.astype(np.float32),
                                          validate=True))
    h.close()


def test_validate_rejects_bad_factors(lib):
    A, W0, H0 = problem(300, 200, 8, seed=5)
    h = lib.Handle()
    Hb = H0.copy()
    Hb[3, 150] = -0.5
    _expect_inval(lib, lambda: h.run(dev(A), 8, "mu", 3, dev(W0), dev(Hb), validate=True))
    Wb = W0.copy()
    Wb[10, 2] = np.nan
    _expect_inval(lib, lambda: h.run(dev(A), 8, "hals", 3, dev(Wb), dev(H0), validate=True))
    # ABPP does not read W0 (Alg. 1 initialises only H), so W0 is not checked
    W, H, rel, _ = h.run(dev(A), 8, "abpp", 3, dev(Wb), dev(H0), validate=True)
    ref = orc.nmf_run(A, 8, "abpp", 3, np.zeros_like(W0), H0)["relres"]
    assert np.abs(rel - ref).max() <= 1e-6
    h.close()


def _csr(m, n, density, seed):
    indptr, indices, data = synth.sparse_uniform(m, n, density, seed=seed)
    return (np.asarray(indptr, np.int64).copy(), np.asarray(indices, np.int32).copy(),
            np.asarray(data, np.float32).copy())


def _run_csr(lib, h, csr, m, n, k, validate=True):
    indptr, indices, data = csr
    t = (dev(indptr, np.int64), dev(indices, np.int32), dev(data))
    M = lib.csr_matrix(*t, (m, n))
    W0, H0 = synth.init_factors(m, n, k, seed=9)
    return h.run(M, k, "hals", 3, dev(W0), dev(H0), validate=validate)


def _first_row_with(indptr, count):
    lens = np.diff(indptr)
    return int(np.argmax(lens >= count))


@pytest.mark.parametrize("defect", ["column_past_n", "negative_column", "unsorted_row",
                                    "duplicate_column", "rowptr_decreasing", "rowptr_end",
                                    "negative_value"])
def test_validate_rejects_a_malformed_csr(lib, defect):
    m, n = 400, 300
    csr = _csr(m, n, 0.02, seed=11)
    indptr, indices, data = csr
    r = _first_row_with(indptr, 3)
    p = int(indptr[r])
    if defect == "column_past_n":
        indices[p + 2] = n
    elif defect == "negative_column":
        indices[p] = -1
    elif defect == "unsorted_row":
        indices[p], indices[p + 1] = indices[p + 1], indices[p]
    elif defect == "duplicate_column":
        indices[p + 1] = indices[p]
    elif defect == "rowptr_decreasing":
        indptr[r + 1] = indptr[r] - 1
    elif defect == "rowptr_end":
        indptr[m] = indptr[m] - 1
    elif defect == "negative_value":
        data[p] = -1.0
    h = lib.Handle()
    _expect_inval(lib, lambda: _run_csr(lib, h, (indptr, indices, data), m, n, 6))
    # the same handle then runs a well-formed matrix
    W, H, rel, _ = _run_csr(lib, h, _csr(m, n, 0.02, seed=11), m, n, 6)
    assert np.isfinite(rel).all()
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_bpp_cold_start_reaches_the_warm_start_factors(lib, prec):
    A, W0, H0 = problem(900, 700, 16, seed=21)
    h = lib.Handle()
    Ad = dev(A)
    Ww, Hw, rw, iw = h.run(Ad, 16, "abpp", 8, dev(W0), dev(H0), prec=prec)
    Wc, Hc, rc, ic = h.run(Ad, 16, "abpp", 8, dev(W0), dev(H0), prec=prec, bpp_cold_start=True)
    # the same NNLS solutions, so the same iterates up to the solver's rounding
    assert np.abs(rw - rc).max() <= 1e-6
    assert np.linalg.norm(host(Wc) - host(Ww)) <= 1e-4 * np.linalg.norm(host(Ww))
    assert np.linalg.norm(host(Hc) - host(Hw)) <= 1e-4 * np.linalg.norm(host(Hw))
    assert ic["bpp_pivots"] > iw["bpp_pivots"]  # the warm start saves exchanges
    if prec == "fp32":
        ref = orc.nmf_run(A, 16, "abpp", 8, np.zeros_like(W0), H0)["relres"]
        assert np.abs(rc - ref).max() <= 1e-6
    h.close()


def test_batched_options(lib):
    ks = [8, 16, 24]
    probs = [problem(600 + 83 * i, 450 + 51 * i, k, seed=60 + i) for i, k in enumerate(ks)]
    As = [dev(A) for A, _, _ in probs]
    H0s = [dev(H0) for _, _, H0 in probs]
    h = lib.Handle()
    _, _, rel_w, info_w = h.run_batched(As, ks, 6, H0s, prec="tf32")
    _, _, rel_c, info_c = h.run_batched(As, ks, 6, H0s, prec="tf32", bpp_cold_start=True,
                                        validate=True)
    assert np.abs(rel_w - rel_c).max() <= 1e-5
    assert info_c["bpp_pivots"] > info_w["bpp_pivots"]
    bad = probs[1][0].copy()
    bad[5, 5] = -2.0
    As_bad = [As[0], dev(bad), As[2]]
    _expect_inval(lib, lambda: h.run_batched(As_bad, ks, 6, H0s, prec="tf32", validate=True))
    h.close()
