"""Pins for the FP64 oracle: each test checks the oracle against something other
than itself -- a hand derivation, a closed form, an invariant the paper states,
a brute-force enumeration or an independent library routine -- so that a
dropped term, a sign error or a transposed operand in the oracle fails here.

CPU only (no GPU marker)."""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _frac_matrix(nd):
    return np.array([[float(Fraction(a, b)) for a, b in row] for row in nd])


# ------------------------------------------------------------------ Gram / products
def test_gram_and_products_vs_numpy():
    """Alg. 1 lines 3-4: the oracle's loops against numpy's BLAS products."""
    g = np.random.default_rng(1)
    A = g.random((37, 23))
    W = g.random((37, 5))
    H = g.random((5, 23))
    np.testing.assert_allclose(orc.gram_w(W), W.T @ W, rtol=1e-13)
    np.testing.assert_allclose(orc.gram_h(H), H @ H.T, rtol=1e-13)
    np.testing.assert_allclose(orc.aht(A, H), A @ H.T, rtol=1e-13)
    np.testing.assert_allclose(orc.wta(A, W), W.T @ A, rtol=1e-13)


def test_gram_w_equals_gram_h_of_transpose():
    g = np.random.default_rng(2)
    W = g.random((41, 7))
    np.testing.assert_allclose(orc.gram_w(W), orc.gram_h(W.T), rtol=1e-14)


def test_sparse_products_match_dense_and_scipy():
    """Sec. 5.2.1 sparse products: the CSR loops against the dense loops on the
    densified matrix and against scipy.sparse."""
    sp = pytest.importorskip("scipy.sparse")
    indptr, indices, data = synth.sparse_uniform(53, 31, 0.15, seed=3)
    S = sp.csr_matrix((data, indices, indptr), shape=(53, 31))
    D = S.toarray()
    W0, H0 = synth.init_factors(53, 31, 6, seed=3)
    Ms = orc.Matrix(csr=(indptr, indices, data), shape=(53, 31))
    np.testing.assert_allclose(orc.aht(Ms, H0), orc.aht(D, H0), rtol=1e-13)
    np.testing.assert_allclose(orc.wta(Ms, W0), orc.wta(D, W0), rtol=1e-13)
    np.testing.assert_allclose(orc.aht(Ms, H0), S @ H0.T, rtol=1e-13)
    np.testing.assert_allclose(orc.wta(Ms, W0), (S.T @ W0).T, rtol=1e-13)
    np.testing.assert_allclose(orc.norm2_a(Ms), (D * D).sum(), rtol=1e-13)


# ------------------------------------------------------------------ MU
@pytest.mark.parametrize("fixture", ["mu_step_2x2.json"])
def test_mu_hand_derived_step(fixture):
    """Eq. (muupdate), one W then one H update, hand-derived in exact fractions."""
    d = json.load(open(os.path.join(GOLD, fixture)))
    A, W, H = (np.array(d[x], float) for x in ("A", "W0", "H0"))
    GH = orc.gram_h(H)
    PW = orc.aht(A, H)
    W1 = orc.mu_update_w(W, PW, GH, eps=0.0)
    np.testing.assert_allclose(W1, _frac_matrix(d["W1_num_den"]), rtol=1e-15, atol=0)
    H1 = orc.mu_update_h(H, orc.wta(A, W1), orc.gram_w(W1), eps=0.0)
    np.testing.assert_allclose(H1, _frac_matrix(d["H1_num_den"]), rtol=1e-15, atol=0)


def test_mu_rank1_run_and_relres():
    """Alg. 1 driver + Sec. 6.2 relative error on a hand-derived k=1 example."""
    d = json.load(open(os.path.join(GOLD, "mu_step_rank1.json")))
    A, W, H = (np.array(d[x], float) for x in ("A", "W0", "H0"))
    out = orc.nmf_run(A, 1, "mu", 1, W, H, mu_eps=0.0)
    assert out["rc"] == 0
    np.testing.assert_allclose(out["W"], np.array(d["W1"]), rtol=1e-15)
    np.testing.assert_allclose(out["H"], np.array(d["H1"]), rtol=1e-15)
    a, b = d["relres1_squared_num_den"]
    assert out["relres"][0] == pytest.approx(np.sqrt(a / b), rel=1e-15)


def test_mu_exact_factorisation_is_fixed_point():
    """With A = W H exactly, A H^T = W H H^T and W^T A = W^T W H, so every MU
    ratio is 1 (Eq. muupdate)."""
    A, Ws, Hs = synth.dense_lowrank(30, 20, 4, seed=5, noise=False)
    out = orc.nmf_run(A, 4, "mu", 3, Ws, Hs, mu_eps=0.0)
    np.testing.assert_allclose(out["W"], Ws, rtol=1e-12)
    np.testing.assert_allclose(out["H"], Hs, rtol=1e-12)
    assert np.all(out["relres"] < 1e-14)


# ------------------------------------------------------------------ HALS
def _hals_w_from_objective(A, W, H):
    """Each column of W set to the exact minimiser of ||A - W H||_F over that
    column alone, in order (Eq. hals_obj), computed from A itself -- no Gram
    matrix, no A H^T -- then unit-normalised with H's rows scaled (reading R3)."""
    W = W.copy()
    H = H.copy()
    k = W.shape[1]
    for i in range(k):
        R = A - W @ H + np.outer(W[:, i], H[i])  # residual without term i
        hh = H[i] @ H[i]
        if hh > 0:
            W[:, i] = np.maximum(0.0, R @ H[i] / hh)
    for i in range(k):
        s = np.linalg.norm(W[:, i])
        if s > 0:
            W[:, i] /= s
            H[i] *= s
    return W, H


def _hals_h_from_objective(A, W, H):
    H = H.copy()
    for i in range(H.shape[0]):
        R = A - W @ H + np.outer(W[:, i], H[i])
        ww = W[:, i] @ W[:, i]
        if ww > 0:
            H[i] = np.maximum(0.0, W[:, i] @ R / ww)
    return H


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hals_updates_are_exact_coordinate_minimisers(seed):
    """Eq. (halsupdate) with readings R2/R3 against block-coordinate minimisation
    of the objective (Eq. hals_obj) written from A directly."""
    A, _, _ = synth.dense_lowrank(40, 30, 5, seed=seed)
    W0, H0 = synth.init_factors(40, 30, 6, seed=seed)
    W1, H1 = orc.hals_update_w(W0, orc.aht(A, H0), orc.gram_h(H0), H0)
    Wr, Hr = _hals_w_from_objective(A, W0, H0)
    np.testing.assert_allclose(W1, Wr, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(H1, Hr, rtol=1e-11, atol=1e-13)
    H2 = orc.hals_update_h(H1, orc.wta(A, W1), orc.gram_w(W1))
    np.testing.assert_allclose(H2, _hals_h_from_objective(A, W1, H1), rtol=1e-11, atol=1e-13)


def test_hals_normalisation_keeps_wh_and_unit_columns():
    """Reading R3: compensated normalisation leaves W H unchanged (the W sweep
    with unit-norm output columns)."""
    A, _, _ = synth.dense_lowrank(35, 25, 4, seed=9)
    W0, H0 = synth.init_factors(35, 25, 4, seed=9)
    Wu = W0.copy()
    GH, PW = orc.gram_h(H0), orc.aht(A, H0)
    # the unnormalised sweep, obtained from the objective-based reference
    Wn, Hn = orc.hals_update_w(W0, PW, GH, H0)
    np.testing.assert_allclose(np.linalg.norm(Wn, axis=0), 1.0, rtol=1e-13)
    Wref, Href = _hals_w_from_objective(A, Wu, H0)
    np.testing.assert_allclose(Wn @ Hn, Wref @ Href, rtol=1e-11)


def test_hals_in_sweep_normalisation_equivalence():
    """Normalising each column right after its update (the paper's placement),
    with h_i compensated and H H^T, A H^T recomputed, gives the same W, H as
    the oracle's after-sweep normalisation (reading R3)."""
    A, _, _ = synth.dense_lowrank(30, 22, 3, seed=4)
    W, H = synth.init_factors(30, 22, 5, seed=4)
    W = W.copy(); H = H.copy()
    Wo, Ho = orc.hals_update_w(W, orc.aht(A, H), orc.gram_h(H), H)
    for i in range(W.shape[1]):
        GH = H @ H.T
        PW = A @ H.T
        if GH[i, i] > 0:
            W[:, i] = np.maximum(0.0, W[:, i] + (PW[:, i] - W @ GH[:, i]) / GH[i, i])
        s = np.linalg.norm(W[:, i])
        if s > 0:
            W[:, i] /= s
            H[i] *= s
    np.testing.assert_allclose(Wo, W, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(Ho, H, rtol=1e-11, atol=1e-14)


def test_hals_zero_diagonal_leaves_column():
    """Reading R2: a zero row of H gives (H H^T)_ii = 0 and leaves w^i as is."""
    A, _, _ = synth.dense_lowrank(12, 9, 2, seed=1)
    W0, H0 = synth.init_factors(12, 9, 3, seed=1)
    H0[1] = 0.0
    W1, _ = orc.hals_update_w(W0, orc.aht(A, H0), orc.gram_h(H0), None)
    np.testing.assert_allclose(W1[:, 1], W0[:, 1] / np.linalg.norm(W0[:, 1]), rtol=1e-14)


# ------------------------------------------------------------------ BPP / NLS
def _nls_bruteforce(G, r):
    """Enumerate all 2^k passive sets; return the unique one meeting the KKT
    conditions (Eq. KKT) with strictly positive passive values."""
    k = len(r)
    best = None
    for mask in itertools.product([0, 1], repeat=k):
        F = [i for i in range(k) if mask[i]]
        x = np.zeros(k)
        if F:
            x[F] = np.linalg.solve(G[np.ix_(F, F)], r[F])
        y = G @ x - r
        if np.all(x >= -1e-12) and np.all(y >= -1e-12):
            if best is None or np.abs(x - best).max() > 1e-9:
                assert best is None, "KKT point not unique"
                best = x
    return best


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_bpp_matches_bruteforce_and_scipy_nnls(k):
    """Sec. 4.3: SolveBPP against exhaustive passive-set enumeration and against
    Lawson-Hanson NNLS on C, b (a different algorithm, working on C itself)."""
    from scipy.optimize import nnls

    g = np.random.default_rng(100 + k)
    for trial in range(20):
        C = g.normal(size=(k + 4, k))
        b = g.normal(size=k + 4)
        G, r = C.T @ C, C.T @ b
        x, rc = orc.bpp_solve(G, r)
        assert rc >= 0
        np.testing.assert_allclose(x, _nls_bruteforce(G, r), rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(x, nnls(C, b)[0], rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("k", [10, 30, 50])
def test_bpp_kkt_conditions(k):
    """Eq. (KKT): y = Gx - r >= 0, x >= 0, x_i y_i = 0 at the returned point."""
    g = np.random.default_rng(k)
    for trial in range(10):
        C = g.random((3 * k, k))
        b = g.normal(size=3 * k) + 0.2
        G, r = C.T @ C, C.T @ b
        x, rc = orc.bpp_solve(G, r)
        assert rc >= 0
        y = G @ x - r
        scale = np.abs(r).max()
        assert np.all(x >= 0)
        assert np.all(y >= -1e-10 * scale)
        assert np.all(np.abs(x * y) <= 1e-10 * scale * (1 + x.max()))


def test_bpp_k1_is_scalar_projection():
    """k = 1 reduces to x = max(0, r / g)."""
    for g_, r_ in [(2.0, 3.0), (2.0, -3.0), (0.5, 0.0), (4.0, 1e-300)]:
        x, rc = orc.bpp_solve(np.array([[g_]]), np.array([r_]))
        assert rc >= 0 and x[0] == pytest.approx(max(0.0, r_ / g_), rel=4e-16, abs=0)


def test_bpp_updates_are_rowwise_and_columnwise_nnls():
    """SolveBPP(HH^T, (AH^T)^T) gives the rows of W and SolveBPP(W^TW, W^TA)
    the columns of H (Sec. 4.3): each against scipy NNLS on the original
    least-squares problem min ||H^T x - a_r|| / min ||W x - a^c||."""
    from scipy.optimize import nnls

    A, _, _ = synth.dense_lowrank(25, 18, 3, seed=8)
    W0, H0 = synth.init_factors(25, 18, 4, seed=8)
    W, rc = orc.bpp_update_w(orc.aht(A, H0), orc.gram_h(H0))
    assert rc >= 0
    for r in range(A.shape[0]):
        np.testing.assert_allclose(W[r], nnls(H0.T, A[r])[0], rtol=1e-8, atol=1e-10)
    H, rc = orc.bpp_update_h(orc.wta(A, W0), orc.gram_w(W0))
    assert rc >= 0
    for c in range(A.shape[1]):
        np.testing.assert_allclose(H[:, c], nnls(W0, A[:, c])[0], rtol=1e-8, atol=1e-10)


def test_bpp_indefinite_gram_reports_error():
    """A Gram matrix that is not positive semidefinite has no NLS problem
    behind it: the passive-set Cholesky meets a non-positive pivot."""
    G = np.array([[1.0, 2.0], [2.0, 1.0]])
    x, rc = orc.bpp_solve(G, np.array([1.0, 1.0]))
    assert rc == orc.E_NUMERIC


def test_bpp_zero_column_stays_active():
    """Reading R4: a zero column of C (zero Gram diagonal) leaves its x
    undetermined; the index stays active (x = 0) and the rest is the NNLS
    solution of the other columns (scipy NNLS on C agrees)."""
    from scipy.optimize import nnls

    g = np.random.default_rng(3)
    C = g.random((9, 4))
    C[:, 2] = 0.0
    b = g.random(9)
    G, r = C.T @ C, C.T @ b
    x, rc = orc.bpp_solve(G, r)
    assert rc >= 0 and x[2] == 0.0
    np.testing.assert_allclose(x, nnls(C, b)[0], rtol=1e-9, atol=1e-12)
    y = G @ x - r
    assert np.all(y >= -1e-12) and np.all(np.abs(x * y) <= 1e-12)


# ------------------------------------------------------------------ whole runs
@pytest.mark.parametrize("algo", ["mu", "hals", "abpp"])
@pytest.mark.parametrize("seed", [0, 1])
def test_relative_error_is_monotone(algo, seed):
    """Sec. 6.2: the relative error decreases monotonically (Lee-Seung for MU;
    exact block-coordinate steps for HALS and ABPP)."""
    A, _, _ = synth.dense_lowrank(60, 45, 4, seed=seed)
    W0, H0 = synth.init_factors(60, 45, 5, seed=seed)
    out = orc.nmf_run(A, 5, algo, 30, W0, H0)
    assert out["rc"] == 0
    rel = out["relres"]
    assert np.all(np.diff(rel) <= 1e-12 * rel[:-1])
    assert np.all(out["W"] >= 0) and np.all(out["H"] >= 0)


@pytest.mark.parametrize("algo,iters,tol", [("hals", 2000, 1e-4), ("abpp", 1000, 1e-6)])
def test_planted_noise_free_recovery(algo, iters, tol):
    """A = W* H* with k equal to the planted rank: the residual goes to ~0
    (ABPP solves each subproblem exactly and converges fast; HALS converges
    linearly, so it gets a looser bar at the same budget)."""
    hits = 0
    for seed in range(4):
        A, _, _ = synth.dense_lowrank(50, 40, 3, seed=seed, noise=False)
        W0, H0 = synth.init_factors(50, 40, 3, seed=seed)
        out = orc.nmf_run(A, 3, algo, iters, W0, H0)
        assert out["rc"] == 0
        hits += out["relres"][-1] < tol
    assert hits >= 3


def test_exact_factorisation_is_fixed_point_for_abpp_and_hals():
    A, Ws, Hs = synth.dense_lowrank(30, 20, 4, seed=6, noise=False)
    out = orc.nmf_run(A, 4, "abpp", 2, None, Hs)
    np.testing.assert_allclose(out["W"] @ out["H"], A, rtol=1e-10)
    np.testing.assert_allclose(out["W"], Ws, rtol=1e-9)
    out = orc.nmf_run(A, 4, "hals", 2, Ws, Hs)
    np.testing.assert_allclose(out["W"] @ out["H"], A, rtol=1e-10)
    assert out["relres"][-1] < 1e-12


def test_k1_hals_equals_abpp():
    """k = 1: the HALS coordinate step and the NLS solve are the same scalar
    projection, so one W-update agrees (up to HALS's normalisation)."""
    A, _, _ = synth.dense_lowrank(20, 15, 2, seed=3)
    W0, H0 = synth.init_factors(20, 15, 1, seed=3)
    GH, PW = orc.gram_h(H0), orc.aht(A, H0)
    Wb, rc = orc.bpp_update_w(PW, GH)
    Wh, Hh = orc.hals_update_w(W0, PW, GH, H0)
    np.testing.assert_allclose(Wh * np.linalg.norm(Wb), Wb, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ residual / loss
def test_trace_expansion_equals_direct_residual():
    """||A-WH||^2 = ||A||^2 - 2<W^T A, H> + <W^T W, H H^T> (the identity the GPU
    path uses) against the entry-by-entry residual."""
    A, _, _ = synth.dense_lowrank(33, 27, 4, seed=11)
    W, H = synth.init_factors(33, 27, 5, seed=11)
    d = orc.relres_direct(A, W, H)
    t = orc.relres_trace(orc.norm2_a(A), orc.wta(A, W), H, orc.gram_w(W), orc.gram_h(H))
    assert t == pytest.approx(d, rel=1e-12)
    assert d == pytest.approx(np.linalg.norm(A - W @ H) / np.linalg.norm(A), rel=1e-13)


def test_loss_gradient_central_differences():
    """0.5||A-WH||^2: gradient against central finite differences in FP64
    (step 1e-6) and zero at an exact factorisation."""
    A, _, _ = synth.dense_lowrank(9, 7, 2, seed=12)
    W, H = synth.init_factors(9, 7, 3, seed=12)
    loss, dW, dH = orc.loss_grad(A, W, H)
    assert loss == pytest.approx(0.5 * np.sum((A - W @ H) ** 2), rel=1e-13)
    h = 1e-6
    for (i, j) in [(0, 0), (4, 2), (8, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (orc.loss_grad(A, Wp, H)[0] - orc.loss_grad(A, Wm, H)[0]) / (2 * h)
        assert dW[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for (i, j) in [(0, 0), (2, 6), (1, 3)]:
        Hp, Hm = H.copy(), H.copy()
        Hp[i, j] += h
        Hm[i, j] -= h
        fd = (orc.loss_grad(A, W, Hp)[0] - orc.loss_grad(A, W, Hm)[0]) / (2 * h)
        assert dH[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    A0, Ws, Hs = synth.dense_lowrank(9, 7, 2, seed=12, noise=False)
    l0, g1, g2 = orc.loss_grad(A0, Ws, Hs)
    assert l0 < 1e-25 and np.abs(g1).max() < 1e-12 and np.abs(g2).max() < 1e-12


def test_sparse_run_matches_dense_run():
    """The driver on CSR input follows the same iterates as on the densified
    matrix (the two product code paths differ)."""
    indptr, indices, data = synth.sparse_uniform(40, 30, 0.2, seed=13)
    sp = pytest.importorskip("scipy.sparse")
    D = sp.csr_matrix((data, indices, indptr), shape=(40, 30)).toarray()
    W0, H0 = synth.init_factors(40, 30, 4, seed=13)
    Ms = orc.Matrix(csr=(indptr, indices, data), shape=(40, 30))
    for algo in ("mu", "hals", "abpp"):
        a = orc.nmf_run(Ms, 4, algo, 10, W0, H0)
        b = orc.nmf_run(D, 4, algo, 10, W0, H0)
        np.testing.assert_allclose(a["relres"], b["relres"], rtol=1e-10)


def test_sampled_gradient_rows_and_columns_match_full_gradient():
    """or_grad_w_row / or_grad_h_col (used at sizes where the full gradient is
    too costly) against or_loss_grad, and the gradient against the closed form
    (WH - A) H^T, W^T (WH - A) written with numpy."""
    A, _, _ = synth.dense_lowrank(23, 19, 3, seed=21)
    W, H = synth.init_factors(23, 19, 4, seed=21)
    _, dW, dH = orc.loss_grad(A, W, H)
    np.testing.assert_allclose(orc.grad_w_rows(A, W, H, [0, 7, 22]), dW[[0, 7, 22]], rtol=1e-12)
    np.testing.assert_allclose(orc.grad_h_cols(A, W, H, [0, 5, 18]), dH[:, [0, 5, 18]].T, rtol=1e-12)
    R = W @ H - A
    np.testing.assert_allclose(dW, R @ H.T, rtol=1e-12)
    np.testing.assert_allclose(dH, W.T @ R, rtol=1e-12)
    assert orc.resid2(A, W, H) == pytest.approx(np.sum(R * R), rel=1e-13)


# ------------------------------------------------------------------ HALS as printed (R9)
def _orthogonal_rows(k, n, norms, seed):
    """k x n with mutually orthogonal rows of the given norms (H H^T diagonal)."""
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, k)))
    return np.asarray(norms)[:, None] * q.T


def test_hals_printed_w_closed_form_with_diagonal_gram():
    """With H H^T = D diagonal the columns decouple, and the printed rule
    (no division by D_ii, then normalisation) gives column i = the unit
    vector along [(1 - D_ii) w^i + (A H^T)^i]_+ in closed form; the exact
    coordinate step (reading R2) would give [(A H^T)^i / D_ii]_+ instead."""
    A, _, _ = synth.dense_lowrank(30, 24, 4, seed=21)
    W0, _ = synth.init_factors(30, 24, 4, seed=21)
    d = np.array([0.5, 2.0, 1.0, 3.5])
    H = _orthogonal_rows(4, 24, np.sqrt(d), seed=21)
    GH = H @ H.T
    assert np.abs(GH - np.diag(d)).max() < 1e-12
    PW = A @ H.T
    W1 = orc.hals_update_w_printed(W0, PW, GH)
    zero = 0
    for i in range(4):
        v = np.maximum(0.0, (1.0 - d[i]) * W0[:, i] + PW[:, i])
        s = np.linalg.norm(v)
        if s == 0.0:  # the step empties the column, which then stays zero
            zero += 1
            np.testing.assert_array_equal(W1[:, i], 0.0)
        else:
            np.testing.assert_allclose(W1[:, i], v / s, rtol=1e-11, atol=1e-13)
    assert zero == 1  # D_33 = 3.5 overshoots: (1 - 3.5) w + p < 0 here


def test_hals_printed_w_satisfies_its_recurrence():
    """The printed sweep normalises each column before the next is updated:
    column i of the result is the unit vector along
    [w0^i + p^i - sum_{l < i} W1^l G_li - sum_{l >= i} W0^l G_li]_+, i.e. the
    later columns see the earlier ones already normalised (checked on the
    output, with a Gram matrix that couples every pair of columns)."""
    A, _, _ = synth.dense_lowrank(25, 20, 3, seed=22)
    W0, H = synth.init_factors(25, 20, 5, seed=22)
    GH, PW = H @ H.T, A @ H.T
    W1 = orc.hals_update_w_printed(W0, PW, GH)
    np.testing.assert_allclose(np.linalg.norm(W1, axis=0), 1.0, rtol=1e-13)
    for i in range(5):
        v = W0[:, i] + PW[:, i] - W1[:, :i] @ GH[:i, i] - W0[:, i:] @ GH[i:, i]
        v = np.maximum(0.0, v)
        np.testing.assert_allclose(W1[:, i], v / np.linalg.norm(v), rtol=1e-10, atol=1e-13)
    # and it differs from normalising after the sweep
    Wa = W0.copy()
    for i in range(5):
        Wa[:, i] = np.maximum(0.0, Wa[:, i] + PW[:, i] - Wa @ GH[:, i])
    Wa /= np.linalg.norm(Wa, axis=0)
    assert np.abs(Wa - W1).max() > 1e-3


def test_hals_printed_h_equals_exact_step_for_unit_columns():
    """With unit-norm columns of W, (W^T W)_ii = 1 and the printed H rule is
    the exact coordinate minimiser (reading R2's rule, pinned above)."""
    A, _, _ = synth.dense_lowrank(30, 26, 4, seed=23)
    W, H = synth.init_factors(30, 26, 4, seed=23)
    W = W / np.linalg.norm(W, axis=0)
    PH, GW = W.T @ A, W.T @ W
    np.testing.assert_allclose(orc.hals_update_h_printed(H, PH, GW),
                               orc.hals_update_h(H, PH, GW), rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ projected gradient (R10)
def _products(A, W, H):
    return H @ H.T, A @ H.T, W.T @ W, W.T @ A


def test_pgrad_interior_equals_gradient_norm():
    """For W, H > 0 the projection keeps every entry: the measure is the norm
    of the gradient of 0.5 ||A - WH||^2 (pinned by finite differences)."""
    A, _, _ = synth.dense_lowrank(20, 16, 3, seed=24)
    W, H = synth.init_factors(20, 16, 4, seed=24)
    W, H = W + 0.1, H + 0.1
    _, dW, dH = orc.loss_grad(A, W, H)
    want = np.sqrt(np.sum(dW ** 2) + np.sum(dH ** 2))
    assert orc.pgrad(W, H, *_products(A, W, H)) == pytest.approx(want, rel=1e-12)


def test_pgrad_vanishes_at_an_nnls_solution():
    """W from an exact NLS solve for fixed H meets the KKT conditions: the
    W block of the projected gradient is zero (the zero entries' positive
    gradient is projected away, the positive entries' gradient is zero)."""
    A, _, _ = synth.dense_lowrank(30, 25, 4, seed=25)
    _, H = synth.init_factors(30, 25, 4, seed=25)
    W, rc = orc.bpp_update_w(A @ H.T, H @ H.T)
    assert rc >= 0
    assert (W == 0).any() and (W > 0).any()
    GH, PW = H @ H.T, A @ H.T
    Hz = np.zeros_like(H)  # no H block
    assert orc.pgrad(W, Hz, GH, PW, W.T @ W, np.zeros_like(H)) < 1e-10 * np.abs(PW).max()
    # the raw gradient is not zero there: the projection is doing the work
    g = W @ GH - PW
    assert np.abs(g[W == 0]).max() > 1e-3


def test_pgrad_hand_case_with_zero_entries_of_both_signs():
    """Hand-derived 2 x 2 case, k = 2, whose factors have zero entries with a
    negative and with a positive gradient (reading R10: min(0, g) where the
    entry is 0, g where it is > 0).

    H = [[1, 0], [1, 1]], A = [[3, 0], [0, 0]], W = [[0, 1], [1, 0]]:
      H H^T = [[1, 1], [1, 2]], A H^T = [[3, 3], [0, 0]],
      W^T W = I,                 W^T A = [[0, 0], [3, 0]].
      grad_W = W H H^T - A H^T = [[-2, -1], [1, 1]]
        W_00 = 0, g = -2 -> -2 (kept: negative at a zero entry)
        W_01 = 1, g = -1 -> -1;  W_10 = 1, g = 1 -> 1
        W_11 = 0, g = +1 ->  0 (projected away)           sum of squares 6
      grad_H = W^T W H - W^T A = [[1, 0], [-2, 1]]
        H_00 = 1 -> 1, H_01 = 0 with g = 0 -> 0, H_10 = 1 -> -2, H_11 = 1 -> 1
                                                          sum of squares 6
    so the measure is sqrt(12).  Dropping the negative gradient at a zero
    entry (keeping g only where x > 0) gives sqrt(8); keeping max(0, g)
    there gives sqrt(9); no projection gives sqrt(13).  The transposed
    problem (A^T, H^T, W^T) has the same measure and sends the W entries
    through the loop over H, so both loops see both kinds of zero entry."""
    H = np.array([[1.0, 0.0], [1.0, 1.0]])
    A = np.array([[3.0, 0.0], [0.0, 0.0]])
    W = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert orc.pgrad(W, H, *_products(A, W, H)) == pytest.approx(np.sqrt(12.0), rel=1e-15)
    assert orc.pgrad(H.T, W.T, *_products(A.T, H.T, W.T)) == pytest.approx(np.sqrt(12.0),
                                                                           rel=1e-15)


def test_stop_rule_stops_at_the_first_iteration_below_tolerance():
    """stop_tol: the run ends after the first iteration whose starting state
    has a projected gradient <= stop_tol times the initial one (reading R10);
    stop_tol >= 1 ends after one iteration, and the tracked sequence of a
    full run gives the stopping iteration."""
    A, _, _ = synth.dense_lowrank(40, 30, 4, seed=26)
    W0, H0 = synth.init_factors(40, 30, 4, seed=26)
    assert orc.nmf_run(A, 4, "hals", 10, W0, H0, stop_tol=1.0)["iters_done"] == 1
    full = orc.nmf_run(A, 4, "hals", 40, W0, H0, track_pgrad=True)
    pg = full["pgrad"]
    assert full["iters_done"] == 40 and pg[-1] < 0.05 * pg[0]
    tol = 0.5 * (pg[5] + pg[6]) / pg[0] if pg[6] < pg[5] else None
    assert tol is not None
    first = int(np.argmax(pg <= tol * pg[0]))
    run = orc.nmf_run(A, 4, "hals", 40, W0, H0, stop_tol=tol)
    assert run["iters_done"] == first + 1
    # the same iterates (to the rounding of the threaded residual sums)
    np.testing.assert_allclose(run["relres"], full["relres"][: first + 1], rtol=1e-13)


def test_hals_printed_run_keeps_unit_columns_and_finite_iterates():
    """The printed rule (a step of 1 instead of 1 / (H H^T)_ii) still keeps
    W's columns at unit norm and the iterates finite over a run."""
    A, _, _ = synth.dense_lowrank(40, 30, 4, seed=27)
    W0, H0 = synth.init_factors(40, 30, 4, seed=27)
    r = orc.nmf_run(A, 4, "hals", 30, W0, H0, hals_variant=1)
    assert r["rc"] == 0 and np.isfinite(r["relres"]).all() and np.isfinite(r["H"]).all()
    norms = np.linalg.norm(r["W"], axis=0)
    np.testing.assert_allclose(norms[norms > 0], 1.0, rtol=1e-12)
