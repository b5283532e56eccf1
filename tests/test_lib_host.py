"""The C-ABI library without a GPU: it loads, exports every symbol that
include/slh.h declares, validates arguments on the host, and its host-only
regrid reproduces the oracle's box lists bit for bit."""
import os
import re

import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import regrid as oregrid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(slh.LIB_PATH):
        from paper_2404_02950_gb300 import build
        build.build()
    return slh.lib()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "slh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(slh_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = _declared_symbols()
    assert len(names) >= 19
    L = slh.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(slh.ABI_SYMBOLS) <= set(names)


def test_layout_alignment():
    boxes = [((0, 0, 0), (15, 31, 47)), ((16, 0, 0), (47, 15, 15)), ((48, 0, 0), (63, 63, 63))]
    for g in (1, 2, 3, 4):
        offs, geom, total, nvalid = slh.slh_level_layout(g, boxes)
        assert nvalid == 16 * 32 * 48 + 32 * 16 * 16 + 16 * 64 * 64
        for b, (lo, hi) in enumerate(boxes):
            pitch, pny, pnz, cs = geom[b]
            n = [hi[d] - lo[d] + 1 for d in range(3)]
            assert offs[b] % 64 == 0 and pitch % 8 == 0 and cs % 32 == 0
            assert pitch >= 4 + n[0] + g and pny == n[1] + 2 * g and pnz == n[2] + 2 * g
            assert cs >= pitch * pny * pnz
            end = offs[b] + 4 * cs
            assert end <= total
            if b + 1 < len(boxes):
                assert end <= offs[b + 1]


def _random_tags(rng, n):
    tags = np.zeros((n, n, n), dtype=np.uint8)
    for _ in range(int(rng.integers(1, 8))):
        c = rng.integers(0, n, size=3)
        L = int(rng.integers(1, 2 * n))
        ax = int(rng.integers(0, 3))
        for t in range(L):
            p = c.copy()
            p[ax] = (p[ax] + t) % n
            if rng.random() < 0.3:
                p[(ax + 1) % 3] = (p[(ax + 1) % 3] + 1) % n
            tags[tuple(p)] = 1
    return tags


@pytest.mark.parametrize("seed", range(12))
def test_regrid_matches_oracle_bit_exact(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.choice([16, 32, 48]))
    tags = _random_tags(rng, n)
    for bf, nbuf, mb in ((8, 2, 16), (4, 1, 8), (16, 4, 32), (2, 0, 4)):
        if n % (bf // 2):
            continue
        a = slh.slh_regrid_boxes(tags, bf, nbuf, mb)
        b = oregrid.regrid_boxes(tags, bf, nbuf, mb)
        assert a == b, (bf, nbuf, mb)


def test_regrid_with_parent_matches_oracle():
    rng = np.random.default_rng(7)
    n = 32
    tags = _random_tags(rng, n)
    tags[10:20, 8:24, 12:14] = 1
    parent = [((8, 8, 8), (23, 23, 15)), ((8, 8, 16), (15, 23, 23))]
    for nbuf in (0, 1, 3):
        a = slh.slh_regrid_boxes(tags, 8, nbuf, 16, parent=parent)
        b = oregrid.regrid_boxes(tags, 8, nbuf, 16, parent_boxes=parent)
        assert a == b


def test_regrid_many_boxes_capacity_retry():
    tags = np.ones((32, 32, 32), dtype=np.uint8)
    boxes = slh.slh_regrid_boxes(tags, 4, 0, 4)   # 16^3 blocks, 1 block per box
    assert len(boxes) == 16 ** 3
    assert boxes == oregrid.regrid_boxes(tags, 4, 0, 4)


@pytest.mark.parametrize("bf,mb,msg", [(3, 6, "power of two"), (8, 12, "multiple"), (0, 8, "power of two")])
def test_regrid_rejects_bad_arguments(bf, mb, msg):
    tags = np.zeros((16, 16, 16), dtype=np.uint8)
    with pytest.raises(slh.SlhError) as e:
        slh.slh_regrid_boxes(tags, bf, 0, mb)
    assert e.value.code == -1 and msg in str(e.value)


def test_regrid_rejects_misaligned_parent():
    tags = np.zeros((16, 16, 16), dtype=np.uint8)
    with pytest.raises(slh.SlhError) as e:
        slh.slh_regrid_boxes(tags, 8, 0, 16, parent=[((1, 0, 0), (8, 7, 7))])
    assert e.value.code == -1


def test_layout_rejects_bad_boxes():
    with pytest.raises(slh.SlhError):
        slh.slh_level_layout(3, [((0, 0, 0), (-1, 7, 7))])
    with pytest.raises(slh.SlhError):
        slh.slh_level_layout(0, [((0, 0, 0), (7, 7, 7))])
    with pytest.raises(slh.SlhError) as e:
        slh.slh_level_layout(3, [((0, 0, 0), (7, 7, 7))], nfields=5)
    assert e.value.code == -1 and "nfields" in str(e.value)


def test_layout_with_tensor_fields():
    """16 fields (psi, Pi, u_ij, v_ij): the same box geometry, 16 component
    strides per box instead of 4."""
    boxes = [((0, 0, 0), (15, 31, 47)), ((16, 0, 0), (47, 15, 15))]
    o4, g4, t4, n4 = slh.slh_level_layout(3, boxes, 4)
    o16, g16, t16, n16 = slh.slh_level_layout(3, boxes, 16)
    assert n4 == n16 and (g4 == g16).all()
    assert o16[0] == 0 and o16[1] >= 16 * g16[0][3] and t16 >= o16[1] + 16 * g16[1][3]
    assert t16 > 3.9 * t4


def test_create_rejects_bad_field_count():
    import ctypes
    h = ctypes.c_void_p()
    st = slh.lib().slh_create(ctypes.byref(h), 32, 0.5, 3, 8, slh.SLH_F64, 1, 5, None)
    assert st == -1 and b"nfields" in slh.lib().slh_last_error()


def test_float_reciprocal_index_split_is_exact():
    """The ghost kernel splits flat indexes t into (i, j, k) of an e0 x e1 x e2
    box with float32 reciprocals (k = trunc((t + 1/2) * fl(1/(e0 e1))), then
    j likewise from the remainder).  IEEE float32 arithmetic, as on the GPU,
    gives the exact quotients for every extent up to 34 per axis (regions,
    pieces and patches stay below 32 x 32 x 4 and 21 x 21 x 7)."""
    f32 = np.float32
    for e0 in range(1, 35):
        for e1 in range(1, 35):
            e01 = e0 * e1
            t = np.arange(e01 * 34, dtype=np.int64)
            k = ((t.astype(f32) + f32(0.5)) * (f32(1.0) / f32(e01))).astype(np.int64)
            rem = t - k * e01
            j = ((rem.astype(f32) + f32(0.5)) * (f32(1.0) / f32(e0))).astype(np.int64)
            i = rem - j * e0
            assert np.array_equal(k, t // e01) and np.array_equal(j, (t // e0) % e1) and np.array_equal(i, t % e0), (e0, e1)


@pytest.mark.parametrize("seed", range(8))
def test_local_regrid_matches_oracle(seed):
    """C++ local regrid (slh_local_regrid_boxes) vs the oracle: identical box
    lists on random three-level hierarchies and random block masks."""
    from oracle import local_regrid as olr
    from tests.test_oracle_local_regrid import _random_case
    boxes, masks, n0, bf = _random_case(seed)
    exp = olr.local_regrid(boxes, n0, bf, masks)
    got = slh.slh_local_regrid_boxes(boxes, n0, bf, masks)
    norm = lambda L: [[(tuple(int(v) for v in lo), tuple(int(v) for v in hi)) for lo, hi in lb] for lb in L]
    assert norm(got) == norm(exp)
    assert any(len(g) > len(b) for g, b in zip(got, boxes)) or not any(m.any() for m in masks)


@pytest.mark.parametrize("seed", range(3))
def test_regrid_parents_at_the_periodic_edge_match_oracle(seed):
    """Parents that touch the domain's faces (the allowed region wraps
    around), on a grid large enough that the clustering's grid passes run
    on several host threads."""
    rng = np.random.default_rng(300 + seed)
    n = 64
    tags = _random_tags(rng, n)
    parent = [((0, 0, 0), (19, 63, 31)), ((44, 0, 0), (63, 63, 31)), ((20, 8, 0), (43, 23, 15)),
              ((0, 0, 32), (63, 15, 63)), ((8, 40, 40), (55, 63, 63))]
    for bf, nbuf in ((2, 0), (2, 1), (4, 2)):
        a = slh.slh_regrid_boxes(tags, bf, nbuf, 4 * bf, parent=parent)
        b = oregrid.regrid_boxes(tags, bf, nbuf, 4 * bf, parent_boxes=parent)
        assert a == b, (bf, nbuf)
