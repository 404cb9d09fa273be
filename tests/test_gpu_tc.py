"""Tensor-core (tcgen05) products with A against the FP64 oracle, and whole
mixed-precision runs.

Tolerances (from the arithmetic):
  * TF32: each operand keeps 10 explicit mantissa bits (relative error below
    2^-10 whichever way the hardware drops the low bits), so a product term is
    off by < 2^-9 relative; with FP32 accumulation the test allows
    (2^-9 + 2 K u) (|X| |Y|^T).
  * BF16: both operands rounded to nearest with 7 explicit bits (2^-8
    relative each): (2^-7 + 2 K u) (|X| |Y|^T).
  * whole runs in mixed precision: relative residual within 1e-3 of the
    oracle's after 30 iterations from the same start.
"""
import functools

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
torch = pytest.importorskip("torch")
REL = {"tf32": 2.0 ** -9, "bf16": 2.0 ** -7}


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


def problem(m, n, k, seed):
    A, _, _ = synth.dense_lowrank(m, n, min(k, 20), seed=seed)
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return r32(A), r32(W0), r32(H0)


def check(got, ref, absprod, K, prec):
    tol = (REL[prec] + 2 * K * U32) * absprod + 1e-30
    err = np.abs(got - ref)
    assert (err <= tol).all(), f"max err/tol {np.max(err / tol):.3g} at {np.argwhere(err > tol)[:4]}"


# ragged M and K, k across the MMA N steps (16 .. 256), single and double
# TMEM buffering (N <= 128 vs > 128), one and several units per CTA and K
# splits; partial sums in shared memory (k <= ~160) or in the per-CTA global
# accumulator (k = 256, 300, 384, 512, over several K chunks), and products
# wider than one MMA (k > 256: two column blocks in one launch)
SHAPES = [(300, 200, 10), (517, 389, 50), (1031, 129, 33), (64, 48, 1), (700, 260, 100),
          (257, 1000, 129), (600, 520, 256), (40000, 3000, 50), (2100, 70000, 16),
          (600, 520, 300), (1500, 1300, 512), (700, 9000, 384)]


@functools.lru_cache(maxsize=None)
def oracle_products(m, n, k):
    """The oracle's A H^T and W^T A (FP64) for the shape's problem, shared by
    the TF32 and BF16 cases."""
    A, W, H = problem(m, n, k, seed=m + n + k)
    return orc.aht(A, H), orc.wta(A, W)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_products_tensor_cores(ax, m, n, k, prec):
    A, W, H = problem(m, n, k, seed=m + n + k)
    Ad = dev(A)
    PW = host(ax.aht(Ad, dev(H), prec=prec))
    PH = host(ax.wta(Ad, dev(W), prec=prec))
    ref_aht, ref_wta = oracle_products(m, n, k)
    check(PW, ref_aht, np.abs(A) @ np.abs(H).T, n, prec)
    check(PH, ref_wta, np.abs(W).T @ np.abs(A), m, prec)


@pytest.mark.parametrize("algo,prec", [("hals", "tf32"), ("mu", "bf16"), ("hals", "fp32")])
def test_wide_rank_run_matches_oracle(ax, algo, prec):
    """k = 300, above one MMA's N: the tensor-core products run as two column
    blocks of C, the updates hold 12 entries of a row per lane.  Relative
    residual against the oracle's run from the same start at every one of
    10 iterations: 1e-3 for the mixed forms, 1e-6 for FP32."""
    m, n, k, iters = 1200, 900, 300, 10
    A, _, _ = synth.dense_lowrank(m, n, 40, seed=77)
    W0, H0 = synth.init_factors(m, n, k, seed=77)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    A, W0, H0 = r32(A), r32(W0), r32(H0)
    W, H, rel, _ = ax.run(dev(A), k, algo, iters, dev(W0), dev(H0), prec=prec)
    ref = orc.nmf_run(A, k, algo, iters, W0, H0)["relres"]
    bar = 1e-6 if prec == "fp32" else 1e-3
    assert np.abs(rel - ref).max() <= bar, (rel, ref)
    assert (host(W) >= 0).all() and (host(H) >= 0).all()


def test_products_tensor_cores_padded_lda(ax):
    """A with a leading dimension that is not a multiple of 4 (copied to
    16-byte-aligned rows before TMA)."""
    A, W, H = problem(333, 201, 24, seed=3)
    big = np.zeros((333, 203))
    big[:, :201] = A
    Abig = dev(big)
    Av = Abig[:, :201]
    from paper_1609_09154_gb300 import aunmf

    M = aunmf.Matrix(333, 201, Av.data_ptr(), 203, None, None, None, 0)
    PW = host(ax.aht(M, dev(H), prec="tf32"))
    check(PW, orc.aht(A, H), np.abs(A) @ np.abs(H).T, 201, "tf32")


def test_tensor_core_products_deterministic(ax):
    A, W, H = problem(40000, 3000, 50, seed=5)
    Ad, Hd = dev(A), dev(H)
    p1 = ax.aht(Ad, Hd, prec="tf32")
    p2 = ax.aht(Ad, Hd, prec="tf32")
    assert torch.equal(p1, p2)


@pytest.fixture(scope="module")
def config_small():
    A, _, _ = synth.dense_lowrank(2000, 1500, 10, seed=2024)
    W0, H0 = synth.init_factors(2000, 1500, 10, seed=2024)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return r32(A), r32(W0), r32(H0)


@pytest.fixture(scope="module")
def oracle_runs(config_small):
    A, W0, H0 = config_small
    return {a: orc.nmf_run(A, 10, a, 30, W0, H0) for a in ("mu", "hals", "abpp")}


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("algo", ["mu", "hals", "abpp"])
def test_mixed_run_within_1e3_of_oracle(ax, config_small, oracle_runs, algo, prec):
    A, W0, H0 = config_small
    W, H, rel, info = ax.run(dev(A), 10, algo, 30, dev(W0), dev(H0), prec=prec)
    ref = oracle_runs[algo]["relres"]
    assert np.abs(rel[-1] - ref[-1]) <= 1e-3, (rel[-1], ref[-1])
    assert np.all(np.abs(rel - ref) <= 1e-3)
    assert (host(W) >= 0).all() and (host(H) >= 0).all()


def test_mixed_run_with_and_without_graph_identical(ax, config_small):
    A, W0, H0 = config_small
    Ad = dev(A)
    W1, H1, r1, _ = ax.run(Ad, 10, "hals", 12, dev(W0), dev(H0), prec="tf32", use_graph=True)
    W2, H2, r2, _ = ax.run(Ad, 10, "hals", 12, dev(W0), dev(H0), prec="tf32", use_graph=False)
    assert torch.equal(W1, W2) and torch.equal(H1, H2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_reported_residual_matches_direct(ax, prec):
    """The reported relres (trace form, Sec. 5) equals the FP64 residual of
    the returned factors computed entry by entry, on a product with a long
    contraction (W^T A sums over m = 40000 rows).  The tensor core rounds
    each MMA's addition into its FP32 accumulator toward zero, which biases
    a long accumulation chain low (~-3e-5 relative here without restarts)
    and moves the trace-form residual by ~bias / relres (~1e-3); the kernel
    restarts the chain every 2 K blocks and rounds the sums of chains to
    nearest, and the constant term carries the rounding of A itself.  The
    bar, 1e-4, is 10x what the residual bias of 2-block chains (<= 3e-7
    relative in <W^T A, H>) moves it by at relres ~ 0.03."""
    m, n, k = 40000, 1000, 32
    A, W0, H0 = problem(m, n, k, seed=77)
    W, H, rel, _ = ax.run(dev(A), k, "hals", 5, dev(W0), dev(H0), prec=prec)
    direct = orc.relres_direct(A, host(W), host(H))
    assert abs(rel[-1] - direct) <= 1e-4, (rel[-1], direct)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_run_host_reads_pinned_a_directly(ax, config_small, prec):
    """aunmf_run_host with A in page-locked host memory and a tensor-core
    form: the layout pass reads A over the host link (no staging copy); the
    result equals the device-buffer run bit for bit (same rounded copies,
    same kernels), and so does a pageable A (copied first) and a pinned A
    with padded rows (lda > n)."""
    A, W0, H0 = config_small
    f = lambda x: np.ascontiguousarray(x, dtype=np.float32)  # noqa: E731
    Wd, Hd, rel_d, _ = ax.run(dev(A), 10, "hals", 8, dev(W0), dev(H0), prec=prec)
    pinned = torch.from_numpy(f(A)).pin_memory()
    wide = torch.zeros((A.shape[0], A.shape[1] + 4), dtype=torch.float32).pin_memory()
    wide[:, :A.shape[1]] = pinned
    for Ah in (pinned.numpy(), f(A), wide.numpy()[:, :A.shape[1]]):
        Wh, Hh, rel_h, _ = ax.run_host(Ah, 10, "hals", 8, f(W0), f(H0), prec=prec)
        np.testing.assert_array_equal(rel_h, rel_d)
        np.testing.assert_array_equal(Wh, Wd.cpu().numpy())
        np.testing.assert_array_equal(Hh, Hd.cpu().numpy())
