"""afd_select_topk_noalloc: the top-k selection for callers that cannot call
cudaMalloc (their device memory belongs to another allocator, or a
cudaMalloc/cudaFree synchronisation is not acceptable in their loop).  Its
scratch is a file-scope device array shared by every call.  Through the C ABI
the test checks that the no-alloc selection returns exactly what the
allocating afd_select_topk returns (selection is integer work: bit-exact) on
two calls in a row with the same keys -- so state left in the shared scratch
by the first call cannot leak into the second -- including the k = 0 (cut
above every key) and k = n paths, and that a key count above the stated limit
is refused before any device work."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402

MAX_KEYS = 4096 * 4096


def _keys(n, seed):
    rng = np.random.default_rng(seed)
    keys = np.concatenate([rng.integers(-3, 4, n // 2).astype(np.float32),
                           rng.standard_normal(n - n // 2).astype(np.float32)])
    rng.shuffle(keys)
    keys[:3] = [0.0, -0.0, 0.0]
    return torch.from_numpy(keys).cuda()


@pytest.mark.parametrize("n,frac,seed", [(100003, 0.37, 1), (4097, 0.9, 2), (4096, 0.0, 3), (65537, 1.0, 4),
                                         (1000, 0.5, 5)])
def test_noalloc_select_matches_allocating_select_on_two_calls_in_a_row(n, frac, seed):
    assert torch.cuda.is_available()
    afd.lib()
    keys = _keys(n, seed)
    k = int(np.floor(frac * n + 0.5))
    ref = torch.zeros(n, dtype=torch.uint8, device="cuda")
    tau_ref = afd.afd_select_topk(keys, k, ref)
    outs, taus = [], []
    for _ in range(2):
        out = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        taus.append(afd.afd_select_topk_noalloc(keys, k, out))
        outs.append(out)
    for out, tau in zip(outs, taus):
        assert torch.equal(out, ref)
        assert int(out.sum().item()) == k
        if k == 0:
            assert np.isnan(tau) and np.isnan(tau_ref)
        else:
            assert tau == tau_ref
    assert torch.equal(outs[0], outs[1])


def test_noalloc_after_a_larger_call_leaves_no_stale_counts():
    """A small selection right after a large one reuses the shared scratch
    that the large one filled."""
    big, small = _keys(300001, 11), _keys(5000, 12)
    out_big = torch.zeros(300001, dtype=torch.uint8, device="cuda")
    afd.afd_select_topk_noalloc(big, 123456, out_big)
    ref = torch.zeros(5000, dtype=torch.uint8, device="cuda")
    tau_ref = afd.afd_select_topk(small, 2500, ref)
    out = torch.zeros(5000, dtype=torch.uint8, device="cuda")
    tau = afd.afd_select_topk_noalloc(small, 2500, out)
    assert torch.equal(out, ref) and tau == tau_ref


def test_noalloc_refuses_more_keys_than_its_scratch_holds():
    """The over-limit count goes to the C entry point directly (the Python
    wrapper always passes the tensors' own length); the small buffers are never
    touched because the count is refused first."""
    keys = torch.zeros(16, dtype=torch.float32, device="cuda")
    kept = torch.zeros(16, dtype=torch.uint8, device="cuda")
    tau = ctypes.c_float()
    rc = afd.lib().afd_select_topk_noalloc(ctypes.c_void_p(keys.data_ptr()), MAX_KEYS + 1, 1,
                                           ctypes.c_void_p(kept.data_ptr()), ctypes.byref(tau),
                                           afd.current_stream())
    assert rc == afd.AFD_ERR_INVALID_ARG
    assert "16777216" in afd.afd_last_error()
    assert int(kept.sum().item()) == 0


def test_noalloc_wrapper_refuses_host_arrays_and_short_outputs():
    keys = _keys(100, 13)
    with pytest.raises(TypeError):
        afd.afd_select_topk_noalloc(keys.cpu(), 10, torch.zeros(100, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ValueError):
        afd.afd_select_topk_noalloc(keys, 10, torch.zeros(99, dtype=torch.uint8, device="cuda"))
