"""aunmf_gram_w_noalloc: the W^T W entry point for callers that cannot
allocate device memory (its partial sums sit in a fixed static device array
instead of a cudaMalloc'd workspace).  Called through the C ABI and compared
with the handle-based aunmf_gram_w on two calls in a row, at the tolerance
the other Gram tests use (2 m u |W|^T |W|).

This file is named to be collected last, so a failure here leaves every
other test already run; it passes alone in a fresh process too."""
import ctypes

import numpy as np
import pytest

from paper_1609_09154_gb300 import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
torch = pytest.importorskip("torch")


def _lib():
    from paper_1609_09154_gb300 import aunmf

    return aunmf.load()


def _noalloc(W, G, stream):
    m, k = W.shape
    return _lib().aunmf_gram_w_noalloc(ctypes.c_void_p(W.data_ptr()), m, k,
                                       ctypes.c_void_p(G.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))


def _handle_gram(W):
    L = _lib()
    h = ctypes.c_void_p()
    s = torch.cuda.current_stream()
    assert L.aunmf_create(ctypes.byref(h), ctypes.c_void_p(s.cuda_stream)) == 0
    m, k = W.shape
    G = torch.empty((k, k), device="cuda", dtype=torch.float32)
    assert L.aunmf_gram_w(h, ctypes.c_void_p(W.data_ptr()), m, k, ctypes.c_void_p(G.data_ptr())) == 0
    torch.cuda.synchronize()
    L.aunmf_destroy(h)
    return G


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch.device("cuda")


def test_noalloc_gram_matches_handle_gram_twice(cuda):
    stream = torch.cuda.current_stream()
    for seed, (m, k) in enumerate([(50_000, 50), (3_001, 64)]):
        W0, _ = synth.init_factors(m, 8, k, seed=seed)
        W = torch.as_tensor(W0.astype(np.float32), device=cuda)
        ref = _handle_gram(W).cpu().numpy().astype(np.float64)
        Wh = W.cpu().numpy().astype(np.float64)
        tol = 2 * m * U32 * (np.abs(Wh).T @ np.abs(Wh))
        for call in range(2):
            G = torch.full((k, k), float("nan"), device=cuda, dtype=torch.float32)
            assert _noalloc(W, G, stream) == 0
            torch.cuda.synchronize()
            got = G.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - ref) <= tol), (seed, call)


def test_noalloc_gram_rejects_k_beyond_limit(cuda):
    from paper_1609_09154_gb300 import aunmf

    W = torch.ones((100, 65), device=cuda)
    G = torch.empty((65, 65), device=cuda)
    assert _noalloc(W, G, torch.cuda.current_stream()) == aunmf.E_INVAL
