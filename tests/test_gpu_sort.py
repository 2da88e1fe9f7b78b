"""The onesweep radix sort primitive (gs_sort_pairs) against a stable library sort.

Keys are compared bit for bit and values too: equal keys must keep their input
order. Cases: random 64-bit keys, keys restricted to a few bits, all keys equal,
keys that differ only in the top bits, pre-sorted and reverse-sorted input, and
sizes around the 3840-key tile (empty, 1, one tile, one tile + 1, ragged)."""
import numpy as np
import pytest

from tests.gpu_common import torch_mods

pytestmark = pytest.mark.gpu


def _run(keys_u64, vals_u32, bits):
    torch, api = torch_mods()
    k = torch.as_tensor(keys_u64.view(np.int64)).cuda()
    v = torch.as_tensor(vals_u32.view(np.int32)).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    api.gs_sort_pairs(k, v, bits, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def _expect(keys, vals, bits):
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys & mask, kind="stable")
    return keys[order], vals[order]


CASES = {
    "random64": lambda rng, n: rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64),
    "few_bits": lambda rng, n: rng.integers(0, 7, n, dtype=np.uint64),
    "all_equal": lambda rng, n: np.full(n, 0xDEADBEEF12345678, np.uint64),
    "top_bits_only": lambda rng, n: rng.integers(0, 4, n, dtype=np.uint64) << np.uint64(44),
    "presorted": lambda rng, n: np.sort(rng.integers(0, 2**48, n, dtype=np.uint64)),
    "reversed": lambda rng, n: np.sort(rng.integers(0, 2**48, n, dtype=np.uint64))[::-1].copy(),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("n", [1, 3840, 3841, 100_003])
def test_sort_pairs(case, n):
    rng = np.random.default_rng(n + len(case))
    keys = CASES[case](rng, n)
    vals = np.arange(n, dtype=np.uint32)
    bits = 64 if case in ("random64", "all_equal") else 48
    gk, gv = _run(keys.copy(), vals.copy(), bits)
    ek, ev = _expect(keys, vals, bits)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(gv, ev)


@pytest.mark.parametrize("bits", [1, 8, 13, 41, 43, 48])
def test_partial_key_bits_sort_only_the_low_bits(bits):
    rng = np.random.default_rng(bits)
    n = 50_000
    keys = rng.integers(0, 2**62, n, dtype=np.uint64)
    vals = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    gk, gv = _run(keys.copy(), vals.copy(), bits)
    # stable by the low `bits` bits; higher bits ride along with their key
    mask = np.uint64((1 << bits) - 1)
    order = np.argsort(keys & mask, kind="stable")
    np.testing.assert_array_equal(gk, keys[order])
    np.testing.assert_array_equal(gv, vals[order])


def test_empty_sort_is_noop():
    torch, api = torch_mods()
    k = torch.empty(0, dtype=torch.int64, device="cuda")
    v = torch.empty(0, dtype=torch.int32, device="cuda")
    api.gs_sort_pairs(k, v, 64)
