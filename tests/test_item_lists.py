"""The occupied-item lists the library keeps for a film (host code, no GPU): for every colour, the
32-site words (packed) or 16-site chunks (int8, open boundaries) of each colour row and layer
that hold an occupied site, in (z, row, item) order.  Checked against the definition computed
here with numpy: a site (x, y, z) has colour ((x+z)&1) | (((y+z)&1)<<1) (four colours, Sec. 3),
sits in colour row y>>1 at column x>>1, and is occupied iff z < H(x, y)."""
import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W


@pytest.fixture(scope="module")
def I():
    try:
        from paper_1205_5588_gb300 import isingfilm
    except ImportError as e:          # the library is built by build(); no GPU is needed here
        pytest.skip(f"library not built: {e}")
    return isingfilm


def bits_for(n):
    b = 0
    while (1 << b) < n:
        b += 1
    return b


def expected_lists(H, L, sites):
    R, C = H.shape
    Rh, Ch = (R + 1) // 2, (C + 1) // 2
    per_row = -(-Ch // sites)
    wb, jb = bits_for(per_row), bits_for(Rh)
    out = []
    for c in range(4):
        entries = []
        for z in range(L):
            px, py = (c & 1) ^ (z & 1), ((c >> 1) & 1) ^ (z & 1)
            for j in range(Rh):
                y = 2 * j + py
                if y >= R:
                    continue
                for w in range(per_row):
                    xs = [2 * i + px for i in range(sites * w, min(sites * w + sites, Ch))]
                    if any(x < C and z < H[y, x] for x in xs):
                        entries.append((z << (jb + wb)) | (j << wb) | w)
        out.append(np.array(entries, dtype=np.uint32))
    return out, wb, jb


CASES = [
    ("fractal_ragged", lambda: W.fractal_heights(37, 77, 0.6, 0, 4, seed=1), 4),
    ("fractal_tall", lambda: W.fractal_heights(90, 33, 0.8, 1, 7, seed=2), 7),
    ("wide_rows", lambda: W.fractal_heights(6, 300, 0.7, 0, 3, seed=3), 3),
    ("one_row", lambda: np.full((1, 45), 2, dtype=np.uint8), 2),
    ("one_column", lambda: np.full((31, 1), 3, dtype=np.uint8), 3),
    ("all_vacant", lambda: np.zeros((5, 7), dtype=np.uint8), 3),
    ("sparse", lambda: np.random.Generator(np.random.PCG64(4)).integers(0, 9, size=(23, 19)).astype(np.uint8), 8),
]


@pytest.mark.parametrize("packed", [True, False])
@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_item_lists_match_the_definition(I, name, packed):
    make, L = {c[0]: (c[1], c[2]) for c in CASES}[name]
    H = make()
    got, wb, jb = I.item_lists(H, L, I.PACKED if packed else 0)
    want, wwb, wjb = expected_lists(H, L, 32 if packed else 16)
    assert (wb, jb) == (wwb, wjb)
    for c in range(4):
        assert np.array_equal(got[c], want[c]), (name, packed, c)


def test_item_lists_refused_for_periodic_int8(I):
    H = np.full((8, 8), 3, dtype=np.uint8)
    with pytest.raises(I.IsfError) as e:
        I.item_lists(H, 3, I.PERIODIC_X | I.PERIODIC_Y)
    assert e.value.code == -1


def row_weights(I, H, L):
    """Occupied words per colour row, all colours and layers (the partition's weights)."""
    lists, wb, jb = I.item_lists(H, L, I.PACKED)
    Rh = (H.shape[0] + 1) // 2
    w = np.zeros(Rh, dtype=np.int64)
    for lst in lists:
        np.add.at(w, (lst >> wb) & ((1 << jb) - 1), 1)
    return w


@pytest.mark.parametrize("shape,bands,max_rows", [((2048, 2048, 6, 3), 152, 24), ((300, 200, 5, 7), 40, 10),
                                                  ((90, 70, 4, 8), 45, 1), ((90, 70, 4, 8), 1, 45),
                                                  ((160, 90, 5, 31), 13, 100), ((33, 65, 6, 9), 7, 3)])
def test_slab_partition_properties(I, shape, bands, max_rows):
    """The row bands of the row-slab kernel: contiguous, cover every colour row, 1..max_rows rows
    each, and each cut within one row's weight of an even share of the occupied words."""
    R, C, L, seed = shape
    H = W.fractal_heights(R, C, 0.7, 1, L, seed=seed)
    part = I.slab_partition(H, L, bands, max_rows)
    Rh = (R + 1) // 2
    assert part[0] == 0 and part[-1] == Rh and len(part) == bands + 1
    sizes = np.diff(part)
    assert sizes.min() >= 1 and sizes.max() <= max_rows
    w = row_weights(I, H, L)
    pre = np.concatenate([[0], np.cumsum(w)])
    if bands * max_rows >= 2 * Rh:          # the row limit leaves room to balance
        for g in range(1, bands):
            assert abs(pre[part[g]] - pre[-1] * g / bands) <= w.max(), g


def test_slab_partition_refusals(I):
    H = W.fractal_heights(20, 30, 0.7, 1, 3, seed=5)
    for bands, max_rows in ((11, 5), (0, 5), (4, 2)):       # 10 colour rows
        with pytest.raises(I.IsfError) as e:
            I.slab_partition(H, 3, bands, max_rows)
        assert e.value.code == -1


def test_debug_exports_refuse_what_the_library_refuses():
    """The debug exports apply isf_lattice_create's checks: a film whose periodic colouring would
    conflict is refused with ISF_ERR_COLOURING, not given lists the library never builds."""
    from paper_1205_5588_gb300 import isingfilm as I
    H = np.full((5, 8), 2, dtype=np.uint8)          # periodic y with an odd number of rows
    with pytest.raises(I.IsfError) as e:
        I.item_lists(H, 2, flags=I.PERIODIC_Y)
    assert e.value.code == -4
