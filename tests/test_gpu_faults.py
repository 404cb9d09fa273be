"""Failure paths through the C ABI, made without faulting or hanging the GPU.

aunmf_test_inject withholds one signal so that a bounded device wait runs out
(a flag that nothing sets), with a wait limit of a few milliseconds:
  * the tensor-core product's MMA warp never signals that its first
    accumulator chunk is ready, so the epilogue's mbarrier wait runs out; the
    kernel waits for its own copies and MMAs in flight, frees its tensor
    memory and returns, and aunmf_run / aunmf_run_batched return
    AUNMF_E_TIMEOUT;
  * the FP32 product's producer warp never signals that the first stage of A
    is in shared memory, so the consumer warps' mbarrier wait runs out;
    aunmf_run and aunmf_relres return AUNMF_E_TIMEOUT;
  * block 0 of the printed HALS sweep never arrives at the first grid
    barrier, and every block's bounded wait gives up;
  * workspace allocations fail (cudaMalloc is not called): AUNMF_E_NOMEM.
After each, the same handle runs a normal call that matches the oracle, so
the context and the handle are still usable (and the tensor memory was
freed: a kernel that could not allocate it would not finish)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WAIT_MS = 5.0


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1609_09154_gb300 import aunmf

    yield aunmf
    aunmf.test_inject(aunmf.INJECT_NONE)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def problem(m, n, k, seed):
    A, _, _ = synth.dense_lowrank(m, n, k, seed=seed)
    W0, H0 = synth.init_factors(m, n, k, seed=seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    return r32(A), r32(W0), r32(H0)


@pytest.fixture(scope="module")
def small():
    A, W0, H0 = problem(2000, 1500, 10, seed=2024)
    return A, W0, H0, {a: orc.nmf_run(A, 10, a, 6, W0, H0)["relres"] for a in ("hals", "abpp")}


def _expect(lib, code, fn):
    with pytest.raises(lib.AunmfError) as e:
        fn()
    assert e.value.code == code, (e.value.code, str(e.value))


@pytest.mark.parametrize("use_graph", [True, False])
def test_tensor_core_wait_runs_out_then_handle_recovers(lib, small, use_graph):
    A, W0, H0, ref = small
    h = lib.Handle()
    Ad = dev(A)
    assert lib.test_inject(lib.INJECT_TC_WAIT, WAIT_MS) == lib.OK
    try:
        _expect(lib, lib.E_TIMEOUT, lambda: h.run(Ad, 10, "hals", 6, dev(W0), dev(H0),
                                                  prec="tf32", use_graph=use_graph))
        # the single-step product reports through the run's flag only; it must
        # still return (bounded) and leave the device usable
        h.aht(Ad, dev(H0), prec="bf16")
        torch.cuda.synchronize()
    finally:
        assert lib.test_inject(lib.INJECT_NONE) == lib.OK
    W, H, rel, _ = h.run(Ad, 10, "hals", 6, dev(W0), dev(H0), prec="tf32", use_graph=use_graph)
    assert np.abs(rel - ref["hals"]).max() <= 1e-3
    h.close()


def test_fp32_product_wait_runs_out_then_handle_recovers(lib):
    # k = 40 > 32: the FP32 products take the TMA-fed form
    A, W0, H0 = problem(1200, 900, 40, seed=77)
    ref = orc.nmf_run(A, 40, "hals", 3, W0, H0)["relres"]
    h = lib.Handle()
    Ad = dev(A)
    assert lib.test_inject(lib.INJECT_SIMT_WAIT, WAIT_MS) == lib.OK
    try:
        _expect(lib, lib.E_TIMEOUT, lambda: h.run(Ad, 40, "hals", 3, dev(W0), dev(H0)))
        _expect(lib, lib.E_TIMEOUT, lambda: h.relres(Ad, dev(W0), dev(H0)))
    finally:
        assert lib.test_inject(lib.INJECT_NONE) == lib.OK
    W, H, rel, _ = h.run(Ad, 40, "hals", 3, dev(W0), dev(H0))
    assert np.abs(rel - ref).max() <= 1e-6
    h.close()


def test_grid_barrier_wait_runs_out_then_handle_recovers(lib, small):
    A, W0, H0, _ = small
    h = lib.Handle()
    Ad = dev(A)
    ref = orc.nmf_run(A, 10, "hals", 4, W0, H0, hals_variant=1)["relres"]
    assert lib.test_inject(lib.INJECT_GRID_BARRIER, WAIT_MS) == lib.OK
    try:
        _expect(lib, lib.E_TIMEOUT, lambda: h.run(Ad, 10, "hals", 4, dev(W0), dev(H0),
                                                  hals_variant=1))
    finally:
        assert lib.test_inject(lib.INJECT_NONE) == lib.OK
    W, H, rel, info = h.run(Ad, 10, "hals", 4, dev(W0), dev(H0), hals_variant=1)
    assert info["iters_done"] == 4
    assert np.abs(rel - ref).max() <= 1e-6
    h.close()


def test_batched_product_wait_runs_out_then_handle_recovers(lib):
    ks = [8, 16, 32]
    probs = [problem(700 + 97 * i, 500 + 61 * i, k, seed=40 + i) for i, k in enumerate(ks)]
    As = [dev(A) for A, _, _ in probs]
    H0s = [dev(H0) for _, _, H0 in probs]
    h = lib.Handle()
    _, _, rel_ref, _ = h.run_batched(As, ks, 4, H0s, prec="tf32")
    assert lib.test_inject(lib.INJECT_TC_WAIT, WAIT_MS) == lib.OK
    try:
        _expect(lib, lib.E_TIMEOUT, lambda: h.run_batched(As, ks, 4, H0s, prec="tf32"))
    finally:
        assert lib.test_inject(lib.INJECT_NONE) == lib.OK
    _, _, rel, _ = h.run_batched(As, ks, 4, H0s, prec="tf32")
    np.testing.assert_array_equal(rel, rel_ref)  # deterministic: the same run again
    for i, (A, _, H0) in enumerate(probs):
        ref = orc.nmf_run(A, ks[i], "abpp", 4, np.zeros((A.shape[0], ks[i])), H0)["relres"]
        assert np.abs(rel[i] - ref).max() <= 1e-3
    h.close()


def test_allocation_failure_reports_nomem_then_handle_recovers(lib, small):
    A, W0, H0, ref = small
    h = lib.Handle()  # a fresh handle holds no workspace yet
    Ad = dev(A)
    assert lib.test_inject(lib.INJECT_NOMEM) == lib.OK
    try:
        _expect(lib, lib.E_NOMEM, lambda: h.run(Ad, 10, "abpp", 6, dev(W0), dev(H0)))
    finally:
        assert lib.test_inject(lib.INJECT_NONE) == lib.OK
    W, H, rel, _ = h.run(Ad, 10, "abpp", 6, dev(W0), dev(H0))
    assert np.abs(rel - ref["abpp"]).max() <= 1e-6
    h.close()
