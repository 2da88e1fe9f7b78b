"""gs_sort_pairs_noalloc: the pair sort for callers that cannot allocate device memory
where they sort (a plugin whose buffers belong to a host application, a real-time loop
that cannot take cudaMalloc's synchronisation). It must give exactly what gs_sort_pairs
gives with a caller-provided temporary buffer, on consecutive calls that share the
library's one scratch array. This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(lib, keys, vals, bits, err, stream):
    return lib.gs_sort_pairs_noalloc(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                     ctypes.c_int64(keys.numel()), ctypes.c_int32(bits),
                                     ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_sort_matches_gs_sort_pairs_on_consecutive_calls():
    import torch
    from paper_2509_06433_gb300 import _lib, api
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    # calls in a row with different sizes and key widths: a call must not see anything left in
    # the shared scratch by the one before. Even pass counts (48, 43 bits: 6 passes) end in the
    # caller's arrays; odd ones (40 bits: 5 passes, 24 bits: 3) end in the scratch array and are
    # copied back; the largest accepted n fills the scratch and its look-back status completely.
    cases = [(300_001, 48), (77_777, 43), (_lib.SORT_NOALLOC_MAX_PAIRS, 40), (123_457, 24),
             (_lib.SORT_NOALLOC_MAX_PAIRS, 48)]
    for call_no, (n, bits) in enumerate(cases):
        rng = np.random.default_rng(100 + call_no)
        keys = rng.integers(0, 1 << bits, n, dtype=np.uint64)
        keys[rng.integers(0, n, n // 4)] = keys[0]  # many equal keys: stability matters
        vals = np.arange(n, dtype=np.uint32)
        k_ref = torch.as_tensor(keys.view(np.int64)).cuda()
        v_ref = torch.as_tensor(vals.view(np.int32)).cuda()
        api.gs_sort_pairs(k_ref, v_ref, bits)  # existing entry point, caller-provided scratch
        k_new = torch.as_tensor(keys.view(np.int64)).cuda()
        v_new = torch.as_tensor(vals.view(np.int32)).cuda()
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert _noalloc(lib, k_new, v_new, bits, err, stream) == 0
        torch.cuda.synchronize()
        assert err.item() == 0
        assert torch.equal(k_new, k_ref), call_no
        assert torch.equal(v_new, v_ref), call_no


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2509_06433_gb300 import _lib
    lib = _lib.load()
    keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    vals = torch.zeros(4, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib.gs_sort_pairs_noalloc(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                     ctypes.c_int64(_lib.SORT_NOALLOC_MAX_PAIRS + 1), ctypes.c_int32(48),
                                     ctypes.c_void_p(err.data_ptr()), None)
    assert code == 7  # GS_ERR_SIZE_LIMIT, nothing enqueued
