"""afd_select_topk_noalloc: the top-k selection for callers that cannot call
cudaMalloc (their device memory belongs to another allocator, or a
cudaMalloc/cudaFree synchronisation is not acceptable in their loop).  Its
scratch is a file-scope device array; the test checks, through the C ABI, that
two calls in a row return exactly what the allocating afd_select_topk returns
(selection is integer work: bit-exact), and that a key count above the stated
limit is refused before any device work."""
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


def test_noalloc_select_matches_allocating_select_on_two_calls_in_a_row():
    assert torch.cuda.is_available()
    afd.lib()
    for n, frac, seed in ((100003, 0.37, 1), (4097, 0.9, 2)):
        keys = _keys(n, seed)
        k = int(np.floor(frac * n + 0.5))
        ref = torch.zeros(n, dtype=torch.uint8, device="cuda")
        tau_ref = afd.afd_select_topk(keys, k, ref)
        out = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        tau = afd.afd_select_topk_noalloc(keys, k, out)
        assert torch.equal(out, ref)
        assert tau == tau_ref
        assert int(out.sum().item()) == k


def test_noalloc_refuses_more_keys_than_its_scratch_holds():
    keys = torch.zeros(16, dtype=torch.float32, device="cuda")
    kept = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(afd.AFDError) as e:
        afd.afd_select_topk_noalloc(keys, 1, kept, n=MAX_KEYS + 1)
    assert e.value.code == afd.AFD_ERR_INVALID_ARG
    assert "16777216" in str(e.value)
