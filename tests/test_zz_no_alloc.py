"""sgs_sort_pairs_noalloc against sgs_sort_pairs and against numpy's stable sort.

The no-allocation sort is for callers that may not obtain device memory themselves (a
host that owns every device allocation, or code where a cudaMalloc is refused or would
stall other work).  Its scratch is a fixed array inside the library, so this test checks,
through the C ABI, that calls in a row (later ones smaller, so stale contents of the shared
array would show) give exactly the sort of the entry point that takes a caller-provided
scratch buffer, and the stable order numpy computes on the low key bits; and that an
oversized request and digits wider than the array's tables are refused.
"""
import numpy as np
import pytest
import torch

from paper_2501_00342_b300 import binding as B

pytestmark = pytest.mark.gpu


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _with_scratch(keys, vals, key_bits, digit_bits):
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    nb = B.sort_temp_bytes(len(keys), key_bits, digit_bits)
    temp = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B.sort_pairs(k.data_ptr(), v.data_ptr(), len(keys), key_bits, digit_bits, temp.data_ptr(), nb, _stream())
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def _no_alloc(keys, vals, key_bits, digit_bits):
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    code = B.lib().sgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), len(keys), key_bits, digit_bits,
                                          _stream())
    assert code == B.SGS_OK, B.status_string(code)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def _numpy_stable(keys, vals, key_bits):
    low = keys & np.uint64((1 << key_bits) - 1) if key_bits < 64 else keys
    order = np.argsort(low, kind="stable")
    return keys[order], vals[order]


def _tile_depth_keys(rng, m, key_bits):
    tiles = rng.integers(0, 1 << (key_bits - 32), m).astype(np.uint64)
    depth = rng.uniform(0.2, 60.0, m).astype(np.float32).view(np.uint32).astype(np.uint64)
    keys = (tiles << np.uint64(32)) | depth
    keys[::5] = keys[7]  # ties, to exercise stability
    return keys


def test_no_alloc_sort_matches_scratch_sort_and_numpy():
    rng = np.random.default_rng(2024)
    # 49 bits in 7 passes of 7 bits (odd: the result is copied back), 44 bits in 8 passes of
    # 6, and all 64 bits in 16 passes of 4 at the largest size: every row of the array's
    # 16 x 256 histogram and offset tables is used
    cases = [(B.SORT_NOALLOC_MAX_PAIRS, 49, 8), (77_777, 44, 6), (B.SORT_NOALLOC_MAX_PAIRS, 64, 4)]
    for m, key_bits, digit_bits in cases:
        if key_bits == 64:
            keys = rng.integers(0, 2**64 - 1, size=m, dtype=np.uint64, endpoint=True)
            keys[::7] = keys[11]
        else:
            keys = _tile_depth_keys(rng, m, key_bits)
        vals = np.arange(m, dtype=np.uint32)
        got_k, got_v = _no_alloc(keys, vals, key_bits, digit_bits)
        ref_k, ref_v = _with_scratch(keys, vals, key_bits, digit_bits)
        assert (got_k == ref_k).all() and (got_v == ref_v).all()
        np_k, np_v = _numpy_stable(keys, vals, key_bits)
        assert (got_k == np_k).all() and (got_v == np_v).all()


def test_no_alloc_sort_rejects_oversized_input_and_wide_digits():
    m = B.SORT_NOALLOC_MAX_PAIRS + 1
    k = torch.zeros(m, dtype=torch.int64, device="cuda")
    v = torch.zeros(m, dtype=torch.int32, device="cuda")
    code = B.lib().sgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), m, 44, 8, _stream())
    assert code == B.SGS_ERR_INVALID
    # the array's tables hold digits of up to 8 bits; sgs_sort_pairs would take 9
    code = B.lib().sgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), 1000, 44, 9, _stream())
    assert code == B.SGS_ERR_INVALID
