"""Device-side failure detection without a GPU fault: a bounded wait that runs out sets an
error bit the host reads, and the context stays usable afterwards."""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import torch_mods

pytestmark = pytest.mark.gpu


def test_withheld_tile_makes_the_bounded_wait_report_a_timeout():
    torch, api = torch_mods()
    from paper_2509_06433_gb300 import _lib
    lib = _lib.load()
    n = 3 * 3840
    rng = np.random.default_rng(0)
    keys = torch.as_tensor(rng.integers(0, 256, n, dtype=np.uint64).view(np.int64)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    tmp = torch.empty(api.gs_sort_pairs_tmp_size(n), dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib.gs_sort_diag_withheld_tile(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                          ctypes.c_int64(n), ctypes.c_void_p(tmp.data_ptr()), tmp.numel(),
                                          ctypes.c_void_p(err.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    assert err.item() & 2  # GS_DEVERR_TIMEOUT
    # the context is still usable: an ordinary sort afterwards is exact
    k2 = rng.integers(0, 1 << 40, 50_000, dtype=np.uint64)
    kt = torch.as_tensor(k2.view(np.int64)).cuda()
    vt = torch.arange(k2.size, dtype=torch.int32, device="cuda")
    api.gs_sort_pairs(kt, vt, 40)
    order = np.argsort(k2, kind="stable")
    np.testing.assert_array_equal(kt.cpu().numpy().view(np.uint64), k2[order])
    np.testing.assert_array_equal(vt.cpu().numpy(), order.astype(np.int32))
