"""0.5 ||A - WH||_F^2 and its gradient through the C ABI (aunmf_loss_fwd /
aunmf_loss_bwd) and the torch.autograd.Function, against the FP64 oracle.

Tolerances: the loss is an FP64 reduction of FP32 products, relative 1e-5 on
random (unfitted) factors; gradient entries g (X G - P) carry the FP32 error
of a K-term product in each term: 2 K u (|X||G| + |A||F|) elementwise.
The oracle's gradient is itself pinned to FP64 central differences
(tests/test_oracle_pins.py); here the GPU gradient is also checked directly
against FP64 central differences of the oracle's loss."""
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
    A, _, _ = synth.dense_lowrank(m, n, rank or min(k, 20), seed=seed)
    W, H = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return r32(A), r32(W), r32(H)


def grad_tols(A, W, H):
    m, n = A.shape
    aW, aH, aA = np.abs(W), np.abs(H), np.abs(A)
    tw = 2 * max(m, n) * U32 * (aW @ (aH @ aH.T) + aA @ aH.T) + 1e-30
    th = 2 * max(m, n) * U32 * ((aW.T @ aW) @ aH + aW.T @ aA) + 1e-30
    return tw, th


@pytest.mark.parametrize("m,n,k", [(300, 200, 10), (517, 389, 50), (700, 260, 100)])
def test_loss_and_gradient_match_oracle(ax, m, n, k):
    A, W, H = problem(m, n, k, seed=m + k)
    loss_ref, dW_ref, dH_ref = orc.loss_grad(A, W, H)
    Ad, Wd, Hd = dev(A), dev(W), dev(H)
    loss, wta = ax.loss_fwd(Ad, Wd, Hd)
    assert float(loss.detach()) == pytest.approx(loss_ref, rel=1e-5)
    dW, dH = ax.loss_bwd(Ad, Wd, Hd, wta=wta)
    tw, th = grad_tols(A, W, H)
    assert (np.abs(host(dW) - dW_ref) <= tw).all()
    assert (np.abs(host(dH) - dH_ref) <= th).all()
    dW2, dH2 = ax.loss_bwd(Ad, Wd, Hd)  # without the saved W^T A
    assert torch.equal(dW, dW2) and torch.equal(dH, dH2)


def test_gradient_against_fp64_central_differences(ax):
    """GPU gradient entries against (L(x+h) - L(x-h)) / 2h of the FP64 oracle
    loss, h = 1e-6."""
    A, W, H = problem(40, 30, 5, seed=7)
    dW, dH = ax.loss_bwd(dev(A), dev(W), dev(H))
    dW, dH = host(dW), host(dH)
    h = 1e-6
    for (i, j) in [(0, 0), (17, 3), (39, 4)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (orc.loss_grad(A, Wp, H)[0] - orc.loss_grad(A, Wm, H)[0]) / (2 * h)
        assert dW[i, j] == pytest.approx(fd, rel=1e-4, abs=1e-4)
    for (i, j) in [(0, 0), (2, 17), (4, 29)]:
        Hp, Hm = H.copy(), H.copy()
        Hp[i, j] += h
        Hm[i, j] -= h
        fd = (orc.loss_grad(A, W, Hp)[0] - orc.loss_grad(A, W, Hm)[0]) / (2 * h)
        assert dH[i, j] == pytest.approx(fd, rel=1e-4, abs=1e-4)


def test_autograd_function(ax):
    from paper_1609_09154_gb300.autograd import nmf_loss

    A, W, H = problem(257, 129, 16, seed=3)
    Ad = dev(A)
    Wd = dev(W).requires_grad_(True)
    Hd = dev(H).requires_grad_(True)
    loss = nmf_loss(Ad, Wd, Hd)
    (3.0 * loss).backward()
    loss_ref, dW_ref, dH_ref = orc.loss_grad(A, W, H)
    assert float(loss.detach()) == pytest.approx(loss_ref, rel=1e-5)
    tw, th = grad_tols(A, W, H)
    assert (np.abs(host(Wd.grad) - 3.0 * dW_ref) <= 3.0 * tw).all()
    assert (np.abs(host(Hd.grad) - 3.0 * dH_ref) <= 3.0 * th).all()


def test_autograd_function_on_a_side_stream(ax):
    """nmf_loss called under another torch stream runs its kernels on that
    stream (the handle is rebound to torch's current stream at every call):
    inputs made on the side stream, loss and gradients read after it, equal
    bit for bit to the same call on the default stream."""
    from paper_1609_09154_gb300.autograd import nmf_loss

    A, W, H = problem(2000, 1500, 32, seed=13)

    def grads():
        Ad = dev(A)
        Wd = dev(W).requires_grad_(True)
        Hd = dev(H).requires_grad_(True)
        loss = nmf_loss(Ad, Wd, Hd)
        loss.backward()
        return loss.detach().clone(), Wd.grad.clone(), Hd.grad.clone()

    ref = grads()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        got = grads()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_loss_mixed_precision(ax, prec):
    A, W, H = problem(700, 520, 50, seed=9)
    loss_ref, dW_ref, dH_ref = orc.loss_grad(A, W, H)
    Ad, Wd, Hd = dev(A), dev(W), dev(H)
    loss, wta = ax.loss_fwd(Ad, Wd, Hd, prec=prec)
    assert float(loss) == pytest.approx(loss_ref, rel=1e-3)
    dW, dH = ax.loss_bwd(Ad, Wd, Hd, wta=wta, prec=prec)
    rel = 2.0 ** -9 if prec == "tf32" else 2.0 ** -7
    aW, aH, aA = np.abs(W), np.abs(H), np.abs(A)
    tw = rel * (aW @ (aH @ aH.T) + aA @ aH.T)
    assert (np.abs(host(dW) - dW_ref) <= tw).all()


def test_loss_full_size_sampled(ax):
    """The differentiable-loss workload: dense 20,000 x 10,000, planted rank
    100 + noise, k = 100.  Loss against the oracle's entrywise residual;
    gradient rows / columns sampled (first, last, random) against the
    oracle's one-row / one-column definitions."""
    m, n, k = 20_000, 10_000, 100
    A, _, _ = synth.dense_lowrank(m, n, k, seed=2016)
    A = A.astype(np.float32).astype(np.float64)
    W, H = synth.init_factors(m, n, k, seed=2016)
    W, H = W.astype(np.float32).astype(np.float64) * 0.2, H.astype(np.float32).astype(np.float64) * 0.2
    W, H = W.astype(np.float32).astype(np.float64), H.astype(np.float32).astype(np.float64)
    Ad, Wd, Hd = dev(A), dev(W), dev(H)
    loss, wta = ax.loss_fwd(Ad, Wd, Hd)
    dW, dH = ax.loss_bwd(Ad, Wd, Hd, wta=wta)
    ref = 0.5 * orc.resid2(A, W, H)
    assert float(loss) == pytest.approx(ref, rel=1e-5)
    g = np.random.default_rng(0)
    rows = [0, m - 1] + list(g.integers(0, m, 6))
    cols = [0, n - 1] + list(g.integers(0, n, 6))
    gw = orc.grad_w_rows(A, W, H, rows)
    gh = orc.grad_h_cols(A, W, H, cols)
    dWh, dHh = host(dW), host(dH)
    aW, aH, aA = np.abs(W), np.abs(H), np.abs(A)
    GHa = aH @ aH.T
    for t, r in enumerate(rows):
        tol = 2 * n * U32 * (aW[r] @ GHa + aA[r] @ aH.T) + 1e-30
        assert (np.abs(dWh[r] - gw[t]) <= tol).all()
    GWa = aW.T @ aW
    for t, c in enumerate(cols):
        tol = 2 * m * U32 * (GWa @ aH[:, c] + aW.T @ aA[:, c]) + 1e-30
        assert (np.abs(dHh[:, c] - gh[t]) <= tol).all()
