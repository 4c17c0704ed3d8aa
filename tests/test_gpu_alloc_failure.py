"""Allocation failure through the caller's allocator (lbm_set_allocator).

A framework that owns device memory hands the library an allocator; when that
allocator runs out, every entry point must return LBM_ERR_ALLOC with a message,
keep nothing it allocated in the failed call, and leave the context (or batch)
usable and destroyable.  The failure is made on the host: the allocator below
returns NULL on its k-th call, for every k a successful run makes.  No GPU
fault is involved.
"""
import numpy as np
import pytest

from paper_1710_07073_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


class CountingAllocator:
    """Torch-backed allocator that fails on call number ``fail_at`` (1-based)."""

    def __init__(self, torch, fail_at=None):
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.errors = []
        self.alloc = lbm.ALLOC_FN(self._alloc)
        self.free = lbm.FREE_FN(self._free)

    def _alloc(self, nbytes, _user):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes))
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, nbytes, _user):
        if self.live.get(ptr) != int(nbytes):
            self.errors.append((ptr, nbytes))
            return
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)


DIMS = (16, 16, 32)


def _run_from(phases, start):
    """Run phases[start:], each a callable; returns (index of a phase that raised
    LbmError or None, the error)."""
    for i in range(start, len(phases)):
        try:
            phases[i]()
        except lbm.LbmError as e:
            return i, e
    return None, None


def _column_phases(ctx, many, out):
    """set_fields, set_bubbles, step, read back: each a separate call."""
    rho, u = workloads.random_fields(DIMS, seed=11, amp=1e-4, rho_amp=1e-4)
    if many:
        pos, vel, diam = workloads.swarm(DIMS, 120, seed=5)
    else:
        pos, vel, diam = workloads.single_bubble(DIMS)

    def fields():
        out["u"] = lbm.lbm_get_fields(ctx)[1]

    def totals():
        out["tot"] = lbm.lbm_get_totals(ctx)

    def bubbles():
        out["pos"] = lbm.lbm_get_bubbles(ctx)["pos"]

    return [lambda: lbm.lbm_set_fields(ctx, rho.reshape(-1), u.reshape(-1)),
            lambda: lbm.lbm_set_bubbles(ctx, pos.reshape(-1), vel.reshape(-1), diam),
            lambda: lbm.lbm_step(ctx, 3), fields, totals, bubbles]


def _fresh(torch, fail_at):
    alloc = CountingAllocator(torch, fail_at)
    ctx = lbm.lbm_create(*DIMS, 1.6, lbm.LBM_WALL_ALL)
    lbm.lbm_set_allocator(ctx, alloc.alloc, alloc.free)
    return ctx, alloc


def _check_every_failure(torch, fresh, phases_of, last_error, destroy):
    """Make allocation k fail for every k of a clean run: the failing call
    returns LBM_ERR_ALLOC with a message and keeps nothing; retrying it (and
    running the rest) gives the bits of the clean run; destroy frees all."""
    h, alloc = fresh(torch, None)
    ref = {}
    assert _run_from(phases_of(h, ref), 0) == (None, None)
    ncalls = alloc.calls
    destroy(h)
    assert alloc.live == {} and not alloc.errors
    assert ncalls >= 10
    for k in range(1, ncalls + 1):
        h, alloc = fresh(torch, k)
        out = {}
        phases = phases_of(h, out)
        i, err = _run_from(phases, 0)
        assert err is not None and err.code == lbm.LBM_ERR_ALLOC, (k, i, str(err))
        assert last_error(h), k
        alloc.fail_at = None
        assert _run_from(phases, i) == (None, None), k
        assert ref.keys() == out.keys()
        for key in ref:
            assert np.array_equal(ref[key], out[key]), (k, i, key)
        destroy(h)
        assert alloc.live == {}, (k, len(alloc.live))
        assert not alloc.errors, k


@pytest.mark.parametrize("many", [False, True], ids=["few_bubbles", "many_bubbles"])
def test_column_alloc_failure_every_call(many):
    import torch
    assert torch.cuda.is_available()
    _check_every_failure(torch, _fresh, lambda h, out: _column_phases(h, many, out),
                         lbm.lbm_last_error, lbm.lbm_destroy)


def test_step_as_first_device_call_reports_alloc():
    import torch
    for k in range(1, 8):
        ctx, alloc = _fresh(torch, k)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(ctx, 1)
        assert e.value.code == lbm.LBM_ERR_ALLOC
        assert "device state" in lbm.lbm_last_error(ctx)
        alloc.fail_at = None
        lbm.lbm_step(ctx, 2)
        lbm.lbm_destroy(ctx)
        assert alloc.live == {} and not alloc.errors


BATCH_COLS = workloads.batch_columns(3, seed=3)


def _batch_phases(b, out):
    cols = BATCH_COLS
    pos = np.concatenate([c[2] for c in cols])
    vel = np.concatenate([c[3] for c in cols])
    diam = np.concatenate([c[4] for c in cols])

    def fields():
        out["u"] = lbm.lbm_batch_get_fields(b, 1, int(np.prod(cols[1][0])))[1]

    def bubbles():
        out["pos"] = lbm.lbm_batch_get_bubbles(b)["pos"]

    return [lambda: lbm.lbm_batch_set_bubbles(b, [1, 1, 1], pos.reshape(-1), vel.reshape(-1),
                                              diam),
            lambda: lbm.lbm_batch_step(b, 4), fields, bubbles]


def _fresh_batch(torch, fail_at):
    alloc = CountingAllocator(torch, fail_at)
    b = lbm.lbm_batch_create([c[0] for c in BATCH_COLS], [c[1] for c in BATCH_COLS])
    lbm.lbm_batch_set_allocator(b, alloc.alloc, alloc.free)
    return b, alloc


def test_batch_alloc_failure_every_call():
    import torch
    _check_every_failure(torch, _fresh_batch, _batch_phases, lbm.lbm_batch_last_error,
                         lbm.lbm_batch_destroy)
