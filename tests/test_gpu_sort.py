"""The onesweep radix sort on its own, against a stable sort: random, adversarial and
ragged inputs, every digit width, key widths 1..64; the 32-bit key instantiation (the
one the rasterizer runs) on tile-boundary sizes and unaligned buffers."""
import numpy as np
import pytest
import torch

from paper_2501_00342_b300 import binding as B

pytestmark = pytest.mark.gpu


def _sort_gpu(keys, vals, key_bits, digit_bits):
    m = len(keys)
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    nb = B.sort_temp_bytes(m, key_bits, digit_bits)
    temp = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B.sort_pairs(k.data_ptr(), v.data_ptr(), m, key_bits, digit_bits, temp.data_ptr(), nb,
                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def _expect(keys, vals, key_bits):
    masked = keys & np.uint64((1 << key_bits) - 1) if key_bits < 64 else keys
    order = np.argsort(masked, kind="stable")
    return keys[order], vals[order]


CASES = {
    "all_equal": lambda rng, m: np.full(m, 0x0000123400abcdef, np.uint64),
    "all_distinct": lambda rng, m: (rng.permutation(m).astype(np.uint64) * np.uint64(2654435761)) & np.uint64((1 << 44) - 1),
    "one_digit": lambda rng, m: rng.integers(0, 256, m).astype(np.uint64) << np.uint64(24),
    "tile_depth": lambda rng, m: (rng.integers(0, 3600, m).astype(np.uint64) << np.uint64(32)) |
                                 rng.uniform(0.2, 60, m).astype(np.float32).view(np.uint32).astype(np.uint64),
    "sorted": lambda rng, m: np.arange(m, dtype=np.uint64),
    "reversed": lambda rng, m: np.arange(m, 0, -1, dtype=np.uint64),
    "random64": lambda rng, m: rng.integers(0, 2**63, m, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, m, dtype=np.uint64),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("m", [1, 7, 3840, 3841, 100_003])
def test_sort_cases(case, m):
    rng = np.random.default_rng(m)
    keys = CASES[case](rng, m)
    vals = np.arange(m, dtype=np.uint32)
    kb = 64 if case == "random64" else 44
    ks, vs = _sort_gpu(keys, vals, kb, 8)
    ek, ev = _expect(keys, vals, kb)
    assert (ks == ek).all() and (vs == ev).all()


@pytest.mark.parametrize("digit", [4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("key_bits", [1, 13, 32, 44, 57])
def test_sort_digit_widths(digit, key_bits):
    rng = np.random.default_rng(digit * 100 + key_bits)
    m = 50_000
    keys = rng.integers(0, 2**63, m, dtype=np.uint64) & np.uint64((1 << key_bits) - 1)
    keys[::7] = keys[3]  # many ties
    vals = rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32)
    ks, vs = _sort_gpu(keys, vals, key_bits, digit)
    ek, ev = _expect(keys, vals, key_bits)
    assert (ks == ek).all() and (vs == ev).all()


def test_sort_large():
    rng = np.random.default_rng(1)
    m = 20_000_000
    keys = (rng.integers(0, 1 << 14, m).astype(np.uint64) << np.uint64(32)) | \
        rng.integers(0, 1 << 32, m, dtype=np.uint64)
    vals = np.arange(m, dtype=np.uint32)
    ks, vs = _sort_gpu(keys, vals, 46, 8)
    ek, ev = _expect(keys, vals, 46)
    assert (ks == ek).all() and (vs == ev).all()


def _sort32_gpu(keys, vals, key_bits, digit_bits, offset=0):
    """Sorts on the device; offset > 0 shifts both arrays by `offset` elements inside
    larger buffers (4-byte aligned only)."""
    m = len(keys)
    kb = torch.zeros(m + offset, dtype=torch.int32, device="cuda")
    vb = torch.zeros(m + offset, dtype=torch.int32, device="cuda")
    kb[offset:] = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    vb[offset:] = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    nb = B.sort_temp_bytes(m, key_bits, digit_bits)
    temp = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    B.sort_pairs32(kb[offset:].data_ptr(), vb[offset:].data_ptr(), m, key_bits, digit_bits, temp.data_ptr(), nb,
                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return kb[offset:].cpu().numpy().view(np.uint32), vb[offset:].cpu().numpy().view(np.uint32)


def _expect32(keys, vals, key_bits):
    masked = keys & np.uint32((1 << key_bits) - 1) if key_bits < 32 else keys
    order = np.argsort(masked, kind="stable")
    return keys[order], vals[order]


@pytest.mark.parametrize("m", [1, 31, 4095, 4096, 4097, 8192, 12289, 100_003, (1 << 20) + 3])
@pytest.mark.parametrize("offset", [0, 1])
def test_sort32_sizes(m, offset):
    rng = np.random.default_rng(m + offset)
    keys = rng.integers(0, 1 << 17, m).astype(np.uint32)
    keys[::5] = keys[min(1, m - 1)]  # ties
    vals = np.arange(m, dtype=np.uint32)
    ks, vs = _sort32_gpu(keys, vals, 17, 9, offset)
    ek, ev = _expect32(keys, vals, 17)
    assert (ks == ek).all() and (vs == ev).all()


@pytest.mark.parametrize("digit", [4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("key_bits", [1, 9, 17, 31, 32])
def test_sort32_digit_widths(digit, key_bits):
    rng = np.random.default_rng(1000 + digit * 100 + key_bits)
    m = 70_001
    keys = rng.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    ks, vs = _sort32_gpu(keys, vals, key_bits, digit)
    ek, ev = _expect32(keys, vals, key_bits)
    assert (ks == ek).all() and (vs == ev).all()


def test_sort32_large_depth_keys():
    rng = np.random.default_rng(3)
    m = 30_000_000
    keys = rng.uniform(0.2, 60.0, m).astype(np.float32).view(np.uint32)
    vals = np.arange(m, dtype=np.uint32)
    ks, vs = _sort32_gpu(keys, vals, 32, 8)
    ek, ev = _expect32(keys, vals, 32)
    assert (ks == ek).all() and (vs == ev).all()
