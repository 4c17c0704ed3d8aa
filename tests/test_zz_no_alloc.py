"""lbm_bin_bubbles_noalloc: binning for callers that cannot allocate device memory.

Callers inside a CUDA graph capture, or whose runtime owns all device memory,
cannot let the library call cudaMalloc.  The no-alloc entry point bins with
scratch compiled into the library; here its output, written into buffers the
test allocates up front, must equal the binning that lbm_step produced
(lbm_get_bins) for the same bubble centres, on two calls in a row.  The file
sorts last so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_1710_07073_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


def _noalloc_bins(torch, dims, walls, pos, half_width, offsets, items, status):
    n = half_width.size
    d_pos = torch.tensor(pos.reshape(-1), dtype=torch.float64, device="cuda")
    d_hw = torch.tensor(half_width, dtype=torch.float64, device="cuda")
    d_act = torch.ones(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    lbm.lbm_bin_bubbles_noalloc(dims[0], dims[1], dims[2], walls, n, d_pos.data_ptr(),
                                d_hw.data_ptr(), d_act.data_ptr(), offsets.data_ptr(),
                                items.data_ptr(), items.numel(), status.data_ptr(),
                                stream.cuda_stream)
    stream.synchronize()
    off = offsets.cpu().numpy()
    return off, items.cpu().numpy()[:off[-1]], int(status.cpu().item())


@pytest.mark.parametrize("walls", [lbm.LBM_WALL_ALL, lbm.LBM_WALL_ZM | lbm.LBM_WALL_ZP])
def test_noalloc_binning_equals_step_binning(walls):
    import torch
    assert torch.cuda.is_available()
    dims = workloads.SWARM_CROP
    count = workloads.swarm_count_for_crop(workloads.SWARM_FULL, 100_000, dims)
    pos, vel, diam = workloads.swarm(dims, count, seed=21)
    col = lbm.Column(dims, 1.7, walls)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    half_width = lbm.lbm_default_params().width_factor * diam

    # Output buffers are allocated once, before the calls.
    ntiles = -(-dims[0] // 32) * -(-dims[1] // 4) * -(-dims[2] // 4)
    offsets = torch.empty(ntiles + 1, dtype=torch.int32, device="cuda")
    items = torch.empty(count * 72, dtype=torch.int32, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")

    for steps in (2, 5):                 # two calls in a row, different centres
        lbm.lbm_step(col.ctx, steps)
        ref = lbm.lbm_get_bins(col.ctx)
        assert ref["tile"] == (32, 4, 4)
        centres = lbm.lbm_get_bubbles(col.ctx)["pos"]
        off, its, st = _noalloc_bins(torch, dims, walls, centres, half_width, offsets, items,
                                     status)
        assert st == 0
        assert np.array_equal(off, ref["offsets"])
        assert np.array_equal(its, ref["items"])


def test_noalloc_rejects_more_tiles_than_its_scratch():
    # 2048 x 2048 x 64 needs 524,288 tiles, beyond LBM_NOALLOC_MAX_TILES.
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_bin_bubbles_noalloc(2048, 2048, 64, lbm.LBM_WALL_ALL, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.code == lbm.LBM_ERR_ARG


def test_noalloc_skips_and_flags_invalid_bubbles():
    # Caller input never passes lbm_set_bubbles' checks, so the kernel checks
    # it: an oversized or non-finite half-width and a non-finite or out-of-box
    # centre are skipped and set status bit 2; the valid bubbles are binned
    # exactly as the oracle's brute-force binning (Algorithm 1 step 2) does.
    import torch
    from oracle import binning as obin
    dims = (64, 32, 48)
    walls = lbm.LBM_WALL_ALL
    pos = np.array([[10.3, 12.1, 20.7], [40.5, 8.25, 30.0], [60.9, 30.2, 3.1],   # valid
                    [20.0, 16.0, 24.0],                                           # n too large
                    [np.nan, 16.0, 24.0],                                         # NaN centre
                    [20.0, 33.5, 24.0],                                           # outside in y
                    [20.0, 16.0, 24.0]])                                          # n = inf
    hw = np.array([2.25, 3.0, 4.5, 9.5, 2.0, 2.0, np.inf])
    valid = np.array([1, 1, 1, 0, 0, 0, 0], dtype=bool)
    ntiles = -(-dims[0] // 32) * -(-dims[1] // 4) * -(-dims[2] // 4)
    offsets = torch.empty(ntiles + 1, dtype=torch.int32, device="cuda")
    items = torch.empty(4096, dtype=torch.int32, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    off, its, st = _noalloc_bins(torch, dims, walls, pos, hw, offsets, items, status)
    assert st == lbm.LBM_NOALLOC_STATUS_SKIPPED
    ref_off, ref_items = obin.tile_lists([p for p in pos], list(hw), valid, dims, walls, (32, 4, 4))
    assert np.array_equal(off, np.array(ref_off))
    assert np.array_equal(its, np.array(ref_items))
