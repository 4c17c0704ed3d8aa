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


def _column_workflow(ctx, many):
    """set_fields, set_bubbles, step, read back; returns the outputs."""
    S = int(np.prod(DIMS))
    rho, u = workloads.random_fields(DIMS, seed=11, amp=1e-4, rho_amp=1e-4)
    lbm.lbm_set_fields(ctx, rho.reshape(-1), u.reshape(-1))
    if many:
        pos, vel, diam = workloads.swarm(DIMS, 120, seed=5)
    else:
        pos, vel, diam = workloads.single_bubble(DIMS)
    lbm.lbm_set_bubbles(ctx, pos.reshape(-1), vel.reshape(-1), diam)
    lbm.lbm_step(ctx, 3)
    _, uo = lbm.lbm_get_fields(ctx)
    tot = lbm.lbm_get_totals(ctx)
    b = lbm.lbm_get_bubbles(ctx)
    assert uo.size == 3 * S
    return uo, tot, b["pos"]


def _fresh(torch, fail_at):
    alloc = CountingAllocator(torch, fail_at)
    ctx = lbm.lbm_create(*DIMS, 1.6, lbm.LBM_WALL_ALL)
    lbm.lbm_set_allocator(ctx, alloc.alloc, alloc.free)
    return ctx, alloc


@pytest.mark.parametrize("many", [False, True], ids=["few_bubbles", "many_bubbles"])
def test_column_alloc_failure_every_call(many):
    import torch
    assert torch.cuda.is_available()
    ctx, alloc = _fresh(torch, None)
    ref = _column_workflow(ctx, many)
    ncalls = alloc.calls
    lbm.lbm_destroy(ctx)
    assert alloc.live == {} and not alloc.errors
    assert ncalls >= 10
    for k in range(1, ncalls + 1):
        ctx, alloc = _fresh(torch, k)
        with pytest.raises(lbm.LbmError) as e:
            _column_workflow(ctx, many)
        assert e.value.code == lbm.LBM_ERR_ALLOC, (k, str(e.value))
        assert lbm.lbm_last_error(ctx), k
        # The failed call kept nothing: what is live is what earlier calls
        # completed with.  The same context then runs the whole workflow.
        alloc.fail_at = None
        out = _column_workflow(ctx, many)
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), k
        lbm.lbm_destroy(ctx)
        assert alloc.live == {}, (k, len(alloc.live))
        assert not alloc.errors, k


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


def _batch_workflow(b):
    cols = workloads.batch_columns(3, seed=3)
    pos = np.concatenate([c[2] for c in cols])
    vel = np.concatenate([c[3] for c in cols])
    diam = np.concatenate([c[4] for c in cols])
    lbm.lbm_batch_set_bubbles(b, [1, 1, 1], pos.reshape(-1), vel.reshape(-1), diam)
    lbm.lbm_batch_step(b, 4)
    _, u = lbm.lbm_batch_get_fields(b, 1, int(np.prod(cols[1][0])))
    return u, lbm.lbm_batch_get_bubbles(b)["pos"]


def _fresh_batch(torch, fail_at):
    cols = workloads.batch_columns(3, seed=3)
    alloc = CountingAllocator(torch, fail_at)
    b = lbm.lbm_batch_create([c[0] for c in cols], [c[1] for c in cols])
    lbm.lbm_batch_set_allocator(b, alloc.alloc, alloc.free)
    return b, alloc


def test_batch_alloc_failure_every_call():
    import torch
    b, alloc = _fresh_batch(torch, None)
    ref = _batch_workflow(b)
    ncalls = alloc.calls
    lbm.lbm_batch_destroy(b)
    assert alloc.live == {} and not alloc.errors
    for k in range(1, ncalls + 1):
        b, alloc = _fresh_batch(torch, k)
        with pytest.raises(lbm.LbmError) as e:
            _batch_workflow(b)
        assert e.value.code == lbm.LBM_ERR_ALLOC, (k, str(e.value))
        assert lbm.lbm_batch_last_error(b), k
        alloc.fail_at = None
        out = _batch_workflow(b)
        for x, y in zip(out, ref):
            assert np.array_equal(x, y), k
        lbm.lbm_batch_destroy(b)
        assert alloc.live == {}, (k, len(alloc.live))
        assert not alloc.errors, k
