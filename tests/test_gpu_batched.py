"""Batched ABPP (aunmf_run_batched): many uneven problems advanced together
with one launch per phase, against the single-problem path and the oracle.

Each problem is checked against aunmf_run on the same inputs (the same
arithmetic, but the single path splits long products and Gram sums
differently, and each exact NLS solve passes such rounding differences on
scaled by the conditioning of the Gram matrix: the bar on the factors'
relative residual is 1e-5 for TF32 and 5e-5 for BF16 products, with
m, n >= 500 >> k as in the batched workload), the reported trace-form
residual against the factors' own FP64 residual (after the term that the
rounding of A contributes, computed here: relres^2 within 8e-7, twice the
bound on the relative bias that the tensor core's truncating accumulation
leaves in <W^T A, H> with 2-K-block chains, <= 3e-7 measured; at
relres ~ 2e-3 that is ~1e-4 in relres), and against the
FP64 oracle at the mixed-precision bar (1e-3) after 30 iterations (TF32:
at every iteration; BF16 rounds A itself, so its trajectory may leave the
oracle's by more than the bar mid-descent and is compared at the end)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ax():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf

    return aunmf.Handle()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def rounded(A, prec):
    """A (FP32 values) rounded as the tensor-core products read it: BF16 to
    nearest even, TF32 to nearest with ties away from zero."""
    a32 = np.ascontiguousarray(A, dtype=np.float32)
    if prec == "bf16":
        return torch.from_numpy(a32).to(torch.bfloat16).to(torch.float64).numpy()
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = ((bits + 0x1000) & ~np.uint64(0x1FFF)).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64)


def expected_reported(A, W, H, prec, direct):
    """The trace form with the rounded copy A~ = A + d and the constant term
    ||A||^2 + 2 <d, A> measures ||A - WH||^2 + 2 <d, A - WH>: the second
    term is the part of the rounding noise that the fitted WH absorbs (about
    k (m + n) / (m n) of ||d||^2; ~1e-6 ||A||^2 for BF16 on the small
    problems here, ~1e-9 on the large workloads)."""
    d = rounded(A, prec) - A
    extra = 2.0 * float((d * (A - W @ H)).sum()) / float((A * A).sum())
    return float(np.sqrt(max(0.0, direct * direct + extra)))


def batch(seed, count, lo=500, hi=900):
    """Uneven problems: m, n uniform in [lo, hi], k from {8, 16, 32, 64},
    planted rank k + noise."""
    g = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        m, n = (int(x) for x in g.integers(lo, hi + 1, size=2))
        k = int(g.choice([8, 16, 32, 64]))
        A, _, _ = synth.dense_lowrank(m, n, k, seed=seed * 1000 + i)
        _, H0 = synth.init_factors(m, n, k, seed=seed * 1000 + i)
        probs.append((A.astype(np.float32).astype(np.float64), H0.astype(np.float32).astype(np.float64), k))
    return probs


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_batched_matches_single_and_oracle(ax, prec):
    """Per problem: the factors' FP64 residual (oracle, entry by entry) equals
    the single path's (1e-5 TF32, 5e-5 BF16); the reported residual matches
    it (squared, 8e-7, after the rounding term) and is within 1e-3 of the
    oracle's own run after 30 iterations."""
    same_bar = 1e-5 if prec == "tf32" else 5e-5
    iters = 30
    probs = batch(11, 7)
    As = [dev(A) for A, _, _ in probs]
    H0s = [dev(H0) for _, H0, _ in probs]
    ks = [k for _, _, k in probs]
    Ws, Hs, rel, info = ax.run_batched(As, ks, iters, H0s, prec=prec)
    assert info["bpp_nonconverged"] == 0 and info["bpp_numeric"] == 0
    assert info["tuned_bpp_warps"] > 0 and info["tuned_bpp_rows"] > 0
    # the grouped products' pipeline depth, autotuned on the first call
    assert info["tuned_gemm_stages_aht"] >= 2 and info["tuned_gemm_stages_wta"] >= 2
    host = lambda t: t.cpu().numpy().astype(np.float64)  # noqa: E731
    for p, (A, H0, k) in enumerate(probs):
        W1, H1, r1, _ = ax.run(As[p], k, "abpp", iters, dev(np.zeros((A.shape[0], k))), H0s[p],
                               prec=prec)
        db = orc.relres_direct(A, host(Ws[p]), host(Hs[p]))
        ds = orc.relres_direct(A, host(W1), host(H1))
        assert abs(db - ds) <= same_bar, (p, db, ds)
        want = expected_reported(A, host(Ws[p]), host(Hs[p]), prec, db)
        assert abs(rel[p][-1] ** 2 - want ** 2) <= 8e-7, (p, rel[p][-1], want, db)
        ref = orc.nmf_run(A, k, "abpp", iters, None, H0)
        assert abs(rel[p][-1] - ref["relres"][-1]) <= 1e-3
        if prec == "tf32":
            assert np.abs(rel[p] - ref["relres"]).max() <= 1e-3
        assert bool((Ws[p] >= 0).all()) and bool((Hs[p] >= 0).all())


def test_batched_deterministic_graph_and_eager(ax):
    probs = batch(12, 5)
    As = [dev(A) for A, _, _ in probs]
    H0s = [dev(H0) for _, H0, _ in probs]
    ks = [k for _, _, k in probs]
    W1, H1, r1, _ = ax.run_batched(As, ks, 6, H0s, use_graph=True)
    W2, H2, r2, _ = ax.run_batched(As, ks, 6, H0s, use_graph=False)
    assert np.array_equal(r1, r2)
    for a, b in zip(W1 + H1, W2 + H2):
        assert torch.equal(a, b)


def test_batched_rejects_unsupported(ax):
    from paper_1609_09154_gb300 import aunmf

    A = dev(np.ones((50, 40)))
    with pytest.raises(aunmf.AunmfError) as e:
        ax.run_batched([A], [65], 2, [dev(np.ones((65, 40)))])
    assert e.value.code == aunmf.E_INVAL
    with pytest.raises(aunmf.AunmfError) as e:
        ax.run_batched([A], [4], 2, [dev(np.ones((4, 40)))], prec="fp32")
    assert e.value.code == aunmf.E_UNSUPPORTED


def test_abpp_ill_conditioned_factor_keeps_gram_definite(ax):
    """ABPP's factors on uniform low-rank data can reach cond(W^T W) ~ 1e9
    (a 2522 x 5235, k = 32 instance of the batched recipe does at its second
    W update).  A Gram summed in FP32 is then indefinite and the FP64
    Cholesky of the passive set fails; the library forms ABPP's Grams to
    ~FP64 accuracy.  The TF32 run must complete, and match the FP32 run."""
    m, n, k, seed = 2522, 5235, 32, 1609 + 31 * 128
    A, _, _ = synth.dense_lowrank_torch(m, n, k, seed=seed, device="cuda")
    _, H0 = synth.init_factors_torch(m, n, k, seed=seed, device="cuda")
    Z = torch.zeros((m, k), device="cuda")
    rels = {}
    for prec in ("tf32", "fp32"):
        W, H, rel, info = ax.run(A, k, "abpp", 5, Z, H0, prec=prec)
        assert info["bpp_numeric"] == 0
        # at cond(G) ~ 1e9 the solves go through G^-1 with a refinement step,
        # so (almost) no row needs the full-size fallback
        assert 0 <= info["bpp_redone"] <= 0.01 * 5 * (m + n)
        rels[prec] = rel
    assert np.abs(rels["tf32"] - rels["fp32"]).max() <= 1e-3
    # the factor really is ill-conditioned: after the second W update its
    # Gram's smallest eigenvalue is below FP32's resolution of the largest
    W2, _, _, _ = ax.run(A, k, "abpp", 2, Z, H0, prec="tf32")
    Wd = W2.double()
    ev = torch.linalg.eigvalsh(Wd.T @ Wd)
    assert float(ev[0] / ev[-1]) < 2.0 ** -24
