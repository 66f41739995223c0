"""Failure detection without a GPU fault: the bounded look-back wait that the scan and the
radix sort use gives up on a slot that is never published, reports SGS_ERR_TIMEOUT, and
leaves the context usable."""
import time

import numpy as np
import pytest
import torch

from paper_2501_00342_b300 import binding as B
from paper_2501_00342_b300 import inputs as I
from paper_2501_00342_b300.render import GaussianModel, Rasterizer

pytestmark = pytest.mark.gpu

AGG, INC = B.LOOKBACK_AGGREGATE, B.LOOKBACK_INCLUSIVE


def _lookback(slots):
    host = np.asarray(slots, dtype=np.uint64).view(np.int64)
    dev = torch.from_numpy(host.copy()).cuda() if len(host) else torch.empty(0, dtype=torch.int64, device="cuda")
    out_sum = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    out_status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t = time.time()
    B.selftest_lookback(dev.data_ptr() if len(host) else None, len(host), out_sum.data_ptr(),
                        out_status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return int(out_sum.item()), int(out_status.item()), time.time() - t


def test_published_chain_sums_without_waiting():
    # walk back from the last slot: 4 (aggregate), 3 (aggregate), then 5 (inclusive) stops
    s, st, _ = _lookback([INC | 5, AGG | 3, AGG | 4])
    assert (s, st) == (12, B.SGS_OK)
    # an inclusive prefix in the middle ends the walk before the unpublished first slot
    s, st, _ = _lookback([0, INC | 100, AGG | 1])
    assert (s, st) == (101, B.SGS_OK)
    assert _lookback([])[:2] == (0, B.SGS_OK)
    # chains longer than one read window (slots are read several at a time)
    s, st, _ = _lookback([INC | 5] + [AGG | k for k in range(1, 11)])
    assert (s, st) == (60, B.SGS_OK)
    s, st, _ = _lookback([AGG | 2] * 9)  # back to slot 0, which counts as an aggregate
    assert (s, st) == (18, B.SGS_OK)


def test_unpublished_slot_times_out_and_context_survives():
    sc, cams = I.workload(0)
    model = GaussianModel.from_scene(sc)
    before = Rasterizer(model, cams).forward(model).clone()
    # slot 0 is never published: the wait polls it until its limit, then reports
    s, st, secs = _lookback([0, AGG | 7, AGG | 2])
    assert st == B.SGS_ERR_TIMEOUT and s == 9
    assert secs < 60.0
    # an unpublished slot past the first read window: the aggregates after it are summed once
    s, st, secs = _lookback([AGG | 100, 0] + [AGG | 1] * 6)
    assert st == B.SGS_ERR_TIMEOUT and s == 6
    assert secs < 60.0
    # the context is still usable and gives the same image
    after = Rasterizer(model, cams).forward(model)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
