"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by
step from identical inputs and over whole runs.

Inputs are drawn in FP64 by the seeded generators, rounded once to FP32, and
that FP32 data is what both sides see (the oracle promotes it to FP64).

Tolerances (derived from the arithmetic, FP32 unit roundoff u = 2^-24):
  * products with A and Grams: a K-term FP32 dot product carries an error of
    at most ~K u sum_t |a_t b_t|; the test allows 2 K u (|A| |B|).
  * MU: one k-term dot + a division per entry: rtol 1e-5.
  * HALS: k sequential coordinate steps, each with a k-term dot: 1e-4 of the
    entry plus 1e-5 of the largest entry.
  * BPP runs in FP64 on both sides and rounds to FP32 at the end: 2 ulp.
  * whole runs, FP32 path: relative residual within 1e-6 of the oracle's;
    on degenerate shapes whose fit is nearly exact the trace form's own
    rounding (~4u in relres^2) is added to the bar (test_edge_shapes).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ax():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf

    return aunmf.Handle()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def problem(m, n, k, seed, rank=None):
    A, _, _ = synth.dense_lowrank(m, n, rank or k, seed=seed)
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return r32(A), r32(W0), r32(H0)


def assert_product(got, ref, absprod, K, extra_rel=0.0):
    tol = (2 * K * U32 + extra_rel) * absprod + 1e-30
    err = np.abs(got - ref)
    bad = err > tol
    assert not bad.any(), f"max err/tol {np.max(err / tol):.3g} at {np.argwhere(bad)[:3]}"


# shapes spanning several 128-row tiles with ragged tails, and k across the
# 16 / 32 / 64-wide product tiles, the thread-per-row updates' padded widths
# (16, 32, 48, 56, 64 for k <= 64) and the warp-per-row updates above 64 (up to
# 12 and 16 entries per lane at k = 300 and 512)
SHAPES = [(300, 200, 10), (517, 389, 50), (129, 1031, 33), (64, 48, 1), (700, 260, 100),
          (257, 300, 24), (200, 150, 64), (600, 520, 300), (420, 380, 512)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_gram(ax, m, n, k):
    A, W, H = problem(m, n, k, seed=m)
    GW = host(ax.gram_w(dev(W)))
    GH = host(ax.gram_h(dev(H)))
    assert_product(GW, orc.gram_w(W), np.abs(W).T @ np.abs(W), m)
    assert_product(GH, orc.gram_h(H), np.abs(H) @ np.abs(H).T, n)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_products_fp32(ax, m, n, k):
    A, W, H = problem(m, n, k, seed=m + 1)
    PW = host(ax.aht(dev(A), dev(H)))
    PH = host(ax.wta(dev(A), dev(W)))
    assert_product(PW, orc.aht(A, H), np.abs(A) @ np.abs(H).T, n)
    assert_product(PH, orc.wta(A, W), np.abs(W).T @ np.abs(A), m)


@pytest.mark.parametrize("m,n,k", [(300, 9000, 50), (9000, 300, 20)])
def test_products_fp32_long_contraction(ax, m, n, k):
    """Few output tiles and a long contraction: the FP32 product splits K
    into up to 4 ranges (each with its own compensated sums) and adds the
    partials in split order."""
    A, W, H = problem(m, n, k, seed=m + 7)
    PW = host(ax.aht(dev(A), dev(H)))
    PH = host(ax.wta(dev(A), dev(W)))
    assert_product(PW, orc.aht(A, H), np.abs(A) @ np.abs(H).T, n)
    assert_product(PH, orc.wta(A, W), np.abs(W).T @ np.abs(A), m)


@pytest.mark.parametrize("m,n,k", [(40, 1000, 33), (1000, 40, 33), (513, 260, 64), (256, 256, 65),
                                   (2048, 4, 40)])
def test_products_fp32_tma_edges(ax, m, n, k):
    """The TMA-fed FP32 form (k > 32, rows 16-byte aligned) at its edges: an
    output tile mostly past M (40 rows of 256), a contraction shorter than
    one 16-deep step or one 128-long slab (K = 40, K = 4), exactly one tile
    (256 x 256), N = 33 (one column past 32) and 65 (a second column tile of
    one column), and M = 513 (one row into a third tile)."""
    A, W, H = problem(m, n, k, seed=m * 7 + n + k)
    PW = host(ax.aht(dev(A), dev(H)))
    PH = host(ax.wta(dev(A), dev(W)))
    assert_product(PW, orc.aht(A, H), np.abs(A) @ np.abs(H).T, n)
    assert_product(PH, orc.wta(A, W), np.abs(W).T @ np.abs(A), m)


@pytest.mark.parametrize("k", [24, 50])
def test_products_fp32_padded_rows(ax, k):
    """A in a buffer with padded rows (lda = 204 > n = 201), with K tails (201
    and 333 are not multiples of the 16-deep K step).  k = 24: the register-
    staged form takes the float4 tile loads (16-byte aligned rows), and for
    W^T A an output edge (M = 201) whose last group of four rows is partly
    outside A.  k = 50: the TMA-fed form, whose tensor map strides by lda and
    zero-fills past the matrix's n (not lda) columns and m rows."""
    A, W, H = problem(333, 201, k, seed=5)
    big = np.zeros((333, 204))
    big[:, :201] = A
    Abig = dev(big)
    from paper_1609_09154_gb300 import aunmf

    M = aunmf.Matrix(333, 201, Abig.data_ptr(), 204, None, None, None, 0)
    PW = host(ax.aht(M, dev(H)))
    PH = host(ax.wta(M, dev(W)))
    assert_product(PW, orc.aht(A, H), np.abs(A) @ np.abs(H).T, 201)
    assert_product(PH, orc.wta(A, W), np.abs(W).T @ np.abs(A), 333)


@pytest.mark.parametrize("rows,k", [(400_003, 50), (350_001, 33), (320_000, 64), (330_017, 8)])
def test_gram_many_rows(ax, rows, k):
    """Factors with >= 16 x 128 rows per SM take the 8 x 8-tile Gram (rows
    staged as contiguous spans, ~64-row slabs folded into Kahan sums, the
    row groups' sums added in order).  Its error is at most (L + 2 + ngrp) u
    |X|^T |X| for slabs of L ~ 64 rows and ngrp = 256 // tiles row groups
    (FP32 sums of L terms, Kahan's fold, the groups' sum), far inside the
    generic 2 rows u bar; the ragged row counts end in partial stages."""
    rng = np.random.default_rng(rows + k)
    X = rng.random((rows, k)).astype(np.float32).astype(np.float64)
    G = host(ax.gram_w(dev(X)))
    ref = orc.gram_w(X)
    nt = (k + 7) // 8
    ngrp = 256 // (nt * (nt + 1) // 2)
    absprod = np.abs(X).T @ np.abs(X)
    tol = (64 + 2 + ngrp) * U32 * absprod
    err = np.abs(G - ref)
    assert (err <= tol).all(), f"max err/tol {np.max(err / tol):.3g}"
    np.testing.assert_array_equal(G, G.T)


@pytest.mark.parametrize("rows,k", [(5003, 128), (3001, 300), (2100, 512), (1500, 96)])
def test_gram_wide_ranks(ax, rows, k):
    """k >= 96 (a multiple of 4) on >= 1024 rows: X^T X on the TMA-fed FP32
    product kernel, the whole square in Kahan-compensated slabs of 128 rows
    over K splits whose partials are added in FP64.  Error at most (128 + 4)
    u |X|^T |X| (slab sums, Kahan's fold, the splits); the square comes out
    exactly symmetric (entries (i, j) and (j, i) take the same FMAs in the
    same order)."""
    rng = np.random.default_rng(rows + k)
    X = rng.random((rows, k)).astype(np.float32).astype(np.float64)
    G = host(ax.gram_w(dev(X)))
    ref = orc.gram_w(X)
    tol = (128 + 4) * U32 * (np.abs(X).T @ np.abs(X))
    err = np.abs(G - ref)
    assert (err <= tol).all(), f"max err/tol {np.max(err / tol):.3g}"
    np.testing.assert_array_equal(G, G.T)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_mu_updates(ax, m, n, k):
    A, W, H = problem(m, n, k, seed=m + 2)
    PW = (A @ H.T).astype(np.float32).astype(np.float64)
    GH = (H @ H.T).astype(np.float32).astype(np.float64)
    Wg = dev(W)
    ax.update_w("mu", Wg, dev(PW), dev(GH))
    np.testing.assert_allclose(host(Wg), orc.mu_update_w(W, PW, GH), rtol=1e-5, atol=0)
    PH = (W.T @ A).astype(np.float32).astype(np.float64)
    GW = (W.T @ W).astype(np.float32).astype(np.float64)
    Hg = dev(H)
    ax.update_h("mu", Hg, dev(PH), dev(GW))
    np.testing.assert_allclose(host(Hg), orc.mu_update_h(H, PH, GW), rtol=1e-5, atol=0)


def assert_sweep(got, ref, k):
    """HALS sweep (Eq. halsupdate, k coordinates in order) in FP32 against
    FP64: each coordinate step is a k-term dot product whose rounding (~k u
    of its terms) carries into every later coordinate, so the bar grows
    with k above 64."""
    scale = max(1.0, k / 64.0)
    tol = scale * (1e-4 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    err = np.abs(got - ref)
    assert (err <= tol).all(), f"max err/tol {np.max(err / tol):.3g}"


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_hals_updates(ax, m, n, k):
    A, W, H = problem(m, n, k, seed=m + 3)
    PW = (A @ H.T).astype(np.float32).astype(np.float64)
    GH = (H @ H.T).astype(np.float32).astype(np.float64)
    Wg, Hg = dev(W), dev(H)
    ax.update_w("hals", Wg, dev(PW), dev(GH), Hg)
    Wr, Hr = orc.hals_update_w(W, PW, GH, H)
    assert_sweep(host(Wg), Wr, k)
    assert_sweep(host(Hg), Hr, k)
    W1 = host(Wg)
    PH = (W1.T @ A).astype(np.float32).astype(np.float64)
    GW = (W1.T @ W1).astype(np.float32).astype(np.float64)
    H1 = host(Hg)
    Hg2 = dev(H1)
    ax.update_h("hals", Hg2, dev(PH), dev(GW))
    assert_sweep(host(Hg2), orc.hals_update_h(H1, PH, GW), k)


def assert_bpp(got, ref):
    tol = 2 * 2.0 ** -23 * np.abs(ref) + 1e-9 * np.abs(ref).max()
    err = np.abs(got - ref)
    assert (err <= tol).all(), f"max err/tol {np.max(err / tol):.3g}"


@pytest.mark.parametrize("m,n,k", [(300, 200, 10), (517, 389, 50), (129, 1031, 33), (64, 48, 1),
                                   (90, 70, 64)])
def test_bpp_updates(ax, m, n, k):
    A, W, H = problem(m, n, k, seed=m + 4)
    PW = (A @ H.T).astype(np.float32).astype(np.float64)
    GH = (H @ H.T).astype(np.float32).astype(np.float64)
    Wg = dev(np.zeros_like(W))
    ax.update_w("abpp", Wg, dev(PW), dev(GH))
    Wr, rc = orc.bpp_update_w(PW, GH)
    assert rc >= 0
    assert_bpp(host(Wg), Wr)
    PH = (W.T @ A).astype(np.float32).astype(np.float64)
    GW = (W.T @ W).astype(np.float32).astype(np.float64)
    Hg = dev(np.zeros_like(H))
    ax.update_h("abpp", Hg, dev(PH), dev(GW))
    Hr, rc = orc.bpp_update_h(PH, GW)
    assert rc >= 0
    assert_bpp(host(Hg), Hr)


def test_nls_bpp_kkt_and_bruteforce_small(ax):
    """Batched NLS entry point on random well-posed systems: matches the oracle
    and satisfies the KKT conditions (Eq. KKT)."""
    g = np.random.default_rng(5)
    for k in (1, 3, 17, 40, 64):
        C = g.random((3 * k + 5, k)).astype(np.float32).astype(np.float64)
        B = g.normal(size=(3 * k + 5, 257)) + 0.3
        G = (C.T @ C).astype(np.float32).astype(np.float64)
        R = (C.T @ B).T.astype(np.float32).astype(np.float64)  # 257 x k
        X, piv, nc = ax.nls_bpp(dev(G), dev(R))
        X = host(X)
        assert nc == 0
        for r in range(R.shape[0]):
            xr, rc = orc.bpp_solve(G, R[r])
            assert rc >= 0
            assert_bpp(X[r], xr)


def test_nls_bpp_zero_column(ax):
    """A zero column of C (zero Gram diagonal): that entry stays 0 (reading
    R4) and the rest matches the oracle."""
    g = np.random.default_rng(8)
    for k in (5, 40):
        C = g.random((3 * k, k))
        C[:, k // 2] = 0.0
        B = g.random((3 * k, 64))
        G = (C.T @ C).astype(np.float32).astype(np.float64)
        R = (C.T @ B).T.astype(np.float32).astype(np.float64)
        X, piv, nc = ax.nls_bpp(dev(G), dev(R))
        X = host(X)
        assert nc == 0 and np.all(X[:, k // 2] == 0.0)
        for r in range(R.shape[0]):
            xr, rc = orc.bpp_solve(G, R[r])
            assert rc >= 0
            assert_bpp(X[r], xr)


def test_update_abpp_reports_numeric_failure(ax):
    """An ABPP step whose Gram is not positive definite (here indefinite)
    reports AUNMF_E_NUMERIC after synchronising, instead of returning OK
    with rows left unsolved; the oracle rejects the same system."""
    from paper_1609_09154_gb300 import aunmf

    k = 4
    G = np.array([[1.0, 2.0, 0.0, 0.0], [2.0, 1.0, 0.0, 0.0],
                  [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]])  # eigenvalues -1, 1, 1, 3
    R = np.full((8, k), 1.0)
    _, rc = orc.bpp_solve(G, R[0])
    assert rc < 0
    W = dev(np.zeros((8, k)))
    with pytest.raises(aunmf.AunmfError) as e:
        ax.update_w("abpp", W, dev(R), dev(G))
    assert e.value.code == aunmf.E_NUMERIC
    Ht = dev(np.zeros((k, 8)))
    with pytest.raises(aunmf.AunmfError) as e:
        ax.update_h("abpp", Ht, dev(R.T), dev(G))
    assert e.value.code == aunmf.E_NUMERIC


def test_relres_step(ax):
    A, W, H = problem(433, 377, 12, seed=9)
    got = ax.relres(dev(A), dev(W), dev(H))
    assert got == pytest.approx(orc.relres_direct(A, W, H), rel=1e-5)


# ------------------------------------------------------------------ whole runs
@pytest.fixture(scope="module")
def config_small():
    """Dense 2,000 x 1,500, planted rank 10 + |N(0, 0.01^2)|, k = 10."""
    return problem(2000, 1500, 10, seed=2024)


@pytest.fixture(scope="module")
def oracle_runs(config_small):
    A, W0, H0 = config_small
    return {a: orc.nmf_run(A, 10, a, 30, W0, H0) for a in ("mu", "hals", "abpp")}


@pytest.mark.parametrize("algo", ["mu", "hals", "abpp"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_run_matches_oracle_fp32(ax, config_small, oracle_runs, algo, use_graph):
    A, W0, H0 = config_small
    W, H, rel, info = ax.run(dev(A), 10, algo, 30, dev(W0), dev(H0), use_graph=use_graph)
    ref = oracle_runs[algo]
    assert ref["rc"] == 0
    assert np.all(np.abs(rel - ref["relres"]) <= 1e-6), np.abs(rel - ref["relres"]).max()
    Wh, Hh = host(W), host(H)
    assert (Wh >= 0).all() and (Hh >= 0).all()
    # the device residual agrees with the oracle's direct residual of the GPU factors
    assert rel[-1] == pytest.approx(orc.relres_direct(A, Wh, Hh), abs=1e-6)
    if algo == "abpp":
        assert info["bpp_nonconverged"] == 0 and info["bpp_pivots"] > 0


def test_run_is_deterministic_and_resumable(ax, config_small):
    A, W0, H0 = config_small
    Ad = dev(A)
    W1, H1, r1, _ = ax.run(Ad, 10, "hals", 30, dev(W0), dev(H0))
    W2, H2, r2, _ = ax.run(Ad, 10, "hals", 30, dev(W0), dev(H0))
    assert torch.equal(W1, W2) and torch.equal(H1, H2) and np.array_equal(r1, r2)
    Wa, Ha, ra, _ = ax.run(Ad, 10, "hals", 15, dev(W0), dev(H0))
    Wb, Hb, rb, _ = ax.run(Ad, 10, "hals", 15, Wa, Ha)
    assert torch.equal(Wb, W1) and torch.equal(Hb, H1)
    assert np.array_equal(np.concatenate([ra, rb]), r1)


@pytest.mark.parametrize("m,n,k,algo", [(1, 1, 1, "mu"), (3, 700, 2, "hals"), (700, 3, 3, "abpp"),
                                        (257, 129, 1, "hals"), (150, 90, 64, "abpp")])
def test_edge_shapes(ax, m, n, k, algo):
    """Degenerate shapes (1 x 1, a rank above one side, k = 1, k = 64 on
    150 x 90) over 5 iterations.  The device residual is the trace form
    relres^2 = (||A||^2 - 2 <P_H, H> + <G_W, G_H>) / ||A||^2 built from FP32
    products and Grams.  Their stored entries carry a relative rounding of
    u / 2 each (u = 2^-24; the compensated sums keep the accumulation error
    at that size), and at a close fit <P_H, H> and <G_W, G_H> are each about
    ||A||^2, so relres^2 is off by at most ~4u in absolute terms and relres
    by sqrt(r^2 + 4u) - r, r the oracle's value: 4.9e-4 at an exact fit (the
    1 x 1 case, r ~ 1e-15), 3.5e-5 at r = 0.0034 (k = 64 on 150 x 90),
    1.4e-6 at r = 0.083.  The bar is 1e-6 plus that, and no BPP solve may
    stop at its pivot cap."""
    A, W0, H0 = problem(m, n, k, seed=m * 7 + n)
    ref = orc.nmf_run(A, k, algo, 5, W0, H0)
    assert ref["rc"] == 0
    W, H, rel, info = ax.run(dev(A), k, algo, 5, dev(W0), dev(H0))
    r = ref["relres"]
    bar = 1e-6 + (np.sqrt(r * r + 4 * U32) - r)
    assert np.all(np.abs(rel - r) <= bar), (rel - r, bar)
    assert info["bpp_nonconverged"] == 0


def test_zero_iterations_and_invalid_arguments(ax):
    from paper_1609_09154_gb300 import aunmf

    A, W0, H0 = problem(40, 30, 4, seed=1)
    W, H, rel, _ = ax.run(dev(A), 4, "mu", 0, dev(W0), dev(H0))
    np.testing.assert_array_equal(host(W), W0.astype(np.float32))
    np.testing.assert_array_equal(host(H), H0.astype(np.float32))
    with pytest.raises(aunmf.AunmfError) as e:
        ax.run(dev(A), 0, "mu", 3, dev(W0), dev(H0))
    assert e.value.code == aunmf.E_INVAL
    with pytest.raises(aunmf.AunmfError) as e:
        ax.run(dev(A), 65, "abpp", 3, dev(np.ones((40, 65))), dev(np.ones((65, 30))))
    assert e.value.code == aunmf.E_INVAL
    with pytest.raises(aunmf.AunmfError) as e:
        ax.run(dev(A), aunmf.K_MAX + 1, "hals", 1, dev(np.ones((40, aunmf.K_MAX + 1))),
               dev(np.ones((aunmf.K_MAX + 1, 30))))
    assert e.value.code == aunmf.E_INVAL


def test_run_host_matches_device_run(ax, config_small):
    A, W0, H0 = config_small
    f = lambda x: np.ascontiguousarray(x, dtype=np.float32)  # noqa: E731
    Wh, Hh, rel_h, _ = ax.run_host(f(A), 10, "mu", 10, f(W0), f(H0))
    Wd, Hd, rel_d, _ = ax.run(dev(A), 10, "mu", 10, dev(W0), dev(H0))
    np.testing.assert_array_equal(Wh, Wd.cpu().numpy())
    np.testing.assert_array_equal(rel_h, rel_d)
