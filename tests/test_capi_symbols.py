"""The C-ABI library builds, loads and exports every entry point lbm.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_boundary():
    names = _declared()
    for required in ("lbm_create", "lbm_set_bubbles", "lbm_step", "lbm_get_fields",
                     "lbm_get_bubbles", "lbm_destroy", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu(libpath):
    # Calls that touch no device memory work on a machine without a GPU.
    from paper_1710_07073_gb300 import lbm
    c, w = lbm.lbm_velocity_set()
    assert c.shape == (19, 3) and abs(w.sum() - 1.0) < 1e-15
    assert sorted(map(tuple, c.tolist())) == sorted(
        {(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)
         if abs(a) + abs(b) + abs(d) <= 2})
    p = lbm.lbm_default_params()
    assert p.substeps == 10 and p.width_factor == 1.5 and p.c_added_mass == 0.5
    h = lbm.lbm_create(37, 9, 11, 1.6, lbm.LBM_WALL_ALL)
    assert lbm.lbm_sites(h) == 37 * 9 * 11
    assert lbm.lbm_bytes_per_site(h) == 152
    lbm.lbm_destroy(h)
    h = lbm.lbm_create_storage(8, 8, 8, 1.6, 0, lbm.LBM_STORE_F16, 256.0)
    assert lbm.lbm_bytes_per_site(h) == 76
    lbm.lbm_destroy(h)


@pytest.mark.parametrize("args", [
    (0, 8, 8, 1.6, 0x3F), (8, 8, 8, 0.0, 0x3F), (8, 8, 8, 2.0, 0x3F),
    (8, 8, 8, 1.6, 0x01), (8, 8, 8, 1.6, 0x40), (8, 8, 8, 1.6, 0x0F | 0x40),
    (8, 8, 8, 1.6, 0x80 | 0x3F), (2048, 2048, 1024, 1.6, 0x3F)])
def test_create_rejects_bad_arguments(libpath, args):
    from paper_1710_07073_gb300 import lbm
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(*args)
    assert e.value.code == lbm.LBM_ERR_ARG


def test_bubble_arguments_checked_before_device_use(libpath):
    from paper_1710_07073_gb300 import lbm
    h = lbm.lbm_create(16, 16, 16, 1.6, lbm.LBM_WALL_ALL)
    try:
        for pos, d in (([20.0, 8, 8], 2.0), ([8, 8, 8], 0.0), ([8, 8, 8], 7.0), ([8, -1, 8], 1.0)):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_set_bubbles(h, pos, [0, 0, 0], [d])
            assert e.value.code == lbm.LBM_ERR_ARG
            assert lbm.lbm_last_error(h)
    finally:
        lbm.lbm_destroy(h)
    h = lbm.lbm_create(16, 16, 8, 1.6, lbm.LBM_WALL_XM | lbm.LBM_WALL_XP | lbm.LBM_WALL_YM
                       | lbm.LBM_WALL_YP)
    try:
        # On a periodic axis of length 8 a window of half-width 3.75 wraps onto itself.
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_bubbles(h, [8, 8, 4], [0, 0, 0], [2.5])
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("walls", [0x7F, 0x30 | 0x40, 0x33 | 0x40])
def test_create_accepts_free_slip_top_with_bounded_z(libpath, walls):
    # The free-slip top (0x40) is valid whenever the z faces are bounded.
    from paper_1710_07073_gb300 import lbm
    h = lbm.lbm_create(8, 8, 8, 1.6, walls)
    lbm.lbm_destroy(h)


def test_params_forces_bits_checked(libpath):
    # lbm_params.forces takes LBM_FORCE_LIFT and LBM_FORCE_STRESS only.
    from paper_1710_07073_gb300 import lbm
    h = lbm.lbm_create(16, 16, 16, 1.6, lbm.LBM_WALL_ALL)
    try:
        p = lbm.lbm_default_params()
        assert p.forces == 0
        p.forces = lbm.LBM_FORCE_LIFT | lbm.LBM_FORCE_STRESS
        lbm.lbm_set_params(h, p)
        assert lbm.lbm_get_params(h).forces == 3
        p.forces = 4
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_params(h, p)
        assert e.value.code == lbm.LBM_ERR_ARG
    finally:
        lbm.lbm_destroy(h)


def test_params_mapping_and_reaction_checked(libpath):
    # lbm_params.mapping takes LBM_MAP_CELL / LBM_MAP_POINT, .reaction
    # LBM_REACTION_DRAG_LIFT / LBM_REACTION_ALL; the point-sampled map refuses
    # windows of half-width 1/2 or less (no node need lie inside them).
    from paper_1710_07073_gb300 import lbm
    h = lbm.lbm_create(16, 16, 16, 1.6, lbm.LBM_WALL_ALL)
    try:
        p = lbm.lbm_default_params()
        assert p.mapping == lbm.LBM_MAP_CELL and p.reaction == lbm.LBM_REACTION_DRAG_LIFT
        for field, bad in (("mapping", 2), ("mapping", -1), ("reaction", 2)):
            q = lbm.lbm_default_params()
            setattr(q, field, bad)
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_set_params(h, q)
            assert e.value.code == lbm.LBM_ERR_ARG
        p.mapping = lbm.LBM_MAP_POINT
        p.reaction = lbm.LBM_REACTION_ALL
        lbm.lbm_set_params(h, p)
        got = lbm.lbm_get_params(h)
        assert got.mapping == 1 and got.reaction == 1
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_bubbles(h, [8.0, 8.0, 8.0], [0, 0, 0], [1.0 / 3.0])   # n = 1/2
        assert e.value.code == lbm.LBM_ERR_ARG
        assert "point-sampled" in lbm.lbm_last_error(h)
    finally:
        lbm.lbm_destroy(h)
