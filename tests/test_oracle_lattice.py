"""Oracle pins: the z = 12 film lattice (Sec. 2, item 2 of Sec. 3) and its colouring (Sec. 3).

The oracle's stencil is compared with FCC built independently in Cartesian space: site
(x, y, z) sits at x*a1 + y*a2 + z*a3 with unit vectors a1, a2 at 60 degrees in the layer and a3
over the centre of a triangle (ABC stacking); two sites are bonded iff they are at distance 1
(nearest neighbours of FCC).  Bond counts are checked against closed forms, and the colouring
against every bond of the film.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle

A1 = np.array([1.0, 0.0, 0.0])
A2 = np.array([0.5, math.sqrt(3) / 2, 0.0])
A3 = np.array([0.5, math.sqrt(3) / 6, math.sqrt(2.0 / 3.0)])


def cart(x, y, z):
    return x * A1 + y * A2 + z * A3


def cartesian_neighbours(R, C, L, flags):
    """All nearest-neighbour pairs at distance 1, with minimum images on periodic axes."""
    px, py, pz = bool(flags & 1), bool(flags & 2), bool(flags & 4)
    shifts = []
    for m in ((-1, 0, 1) if px else (0,)):
        for n in ((-1, 0, 1) if py else (0,)):
            for o in ((-1, 0, 1) if pz else (0,)):
                shifts.append(m * C * A1 + n * R * A2 + o * L * A3)
    sites = [(x, y, z) for z in range(L) for y in range(R) for x in range(C)]
    pos = {s: cart(*s) for s in sites}
    nb = {s: set() for s in sites}
    for a in sites:
        for b in sites:
            if a == b:
                continue
            d = min(np.linalg.norm(pos[b] + sh - pos[a]) for sh in shifts)
            if abs(d - 1.0) < 1e-9:
                nb[a].add(b)
    return nb


@pytest.mark.parametrize("R,C,L,flags", [(5, 6, 4, 0), (4, 6, 3, 3), (4, 4, 4, 7), (3, 5, 2, 0), (6, 4, 2, 1)])
def test_stencil_is_fcc(olib, R, C, L, flags):
    H = np.full((R, C), L, dtype=np.uint8)
    f = oracle.Film(H, L, flags=flags, lib=olib)
    ref = cartesian_neighbours(R, C, L, flags)
    for (x, y, z), want in ref.items():
        got = set(f.neighbours(x, y, z))
        assert got == want, ((x, y, z), sorted(got ^ want))
    # symmetric relation
    for a, bs in ref.items():
        for b in bs:
            assert a in ref[b]


def test_interior_site_has_6_in_plane_3_up_3_down(olib):
    H = np.full((5, 5), 3, dtype=np.uint8)
    f = oracle.Film(H, 3, lib=olib)
    nbs = f.neighbours(2, 2, 1)
    assert len(nbs) == 12
    dz = [z - 1 for (_, _, z) in nbs]
    assert dz.count(0) == 6 and dz.count(1) == 3 and dz.count(-1) == 3


@pytest.mark.parametrize("Lside,n", [(16, 3), (8, 1), (4, 2), (6, 5)])
def test_bond_count_flat_periodic(olib, Lside, n):
    """Full L x L x n film, periodic in-plane, open top/bottom: each layer has 3 L^2 in-plane
    bonds and each pair of adjacent layers 3 L^2 bonds (16x16x3 -> 3840, N = 768)."""
    f = oracle.Film(np.full((Lside, Lside), n, dtype=np.uint8), n, flags=3, lib=olib)
    info = f.info()
    assert info["n_occ"] == Lside * Lside * n
    assert info["n_bonds"] == 3 * Lside * Lside * n + 3 * Lside * Lside * (n - 1)


def test_bond_count_bulk_cube(olib):
    f = oracle.Film(np.full((4, 4), 4, dtype=np.uint8), 4, flags=7, lib=olib)
    assert f.info()["n_bonds"] == 6 * 64          # z = 12: 6 bonds per site


def test_bonds_and_sites_on_masked_film(olib):
    rng = np.random.Generator(np.random.PCG64(11))
    R, C, L = 6, 7, 4
    H = rng.integers(0, L + 1, size=(R, C)).astype(np.uint8)
    f = oracle.Film(H, L, lib=olib)
    ref = cartesian_neighbours(R, C, L, 0)
    occ = {(x, y, z) for (x, y, z) in ref if z < H[y, x]}
    bonds = sum(1 for a in occ for b in ref[a] if b in occ) // 2
    info = f.info()
    assert info["n_occ"] == len(occ) and info["n_bonds"] == bonds


@pytest.mark.parametrize("R,C,L,flags", [(6, 8, 3, 3), (5, 7, 6, 0), (4, 4, 4, 7), (16, 16, 3, 3)])
def test_colouring_has_no_equal_colour_bond(olib, R, C, L, flags):
    f = oracle.Film(np.full((R, C), L, dtype=np.uint8), L, flags=flags, lib=olib)
    assert f.check_colouring() == 0
    ref = cartesian_neighbours(R, C, L, flags) if R * C * L <= 400 else None
    col = lambda x, y, z: ((x + z) & 1) | (((y + z) & 1) << 1)
    if ref is not None:
        for a, bs in ref.items():
            for b in bs:
                assert col(*a) != col(*b)
    # each colour meets each of the other three colours exactly 4 times (interior site)
    if R >= 4 and C >= 4 and L >= 3:
        x, y, z = 2, 2, 1
        cs = [col(*b) for b in f.neighbours(x, y, z)]
        me = col(x, y, z)
        assert sorted(cs) == sorted([c for c in range(4) if c != me] * 4)


@pytest.mark.parametrize("R,C,L,flags", [(6, 7, 3, 1), (5, 8, 3, 2), (4, 4, 3, 4), (6, 2, 3, 1), (2, 6, 3, 2)])
def test_bad_periodic_extents_rejected(olib, R, C, L, flags):
    with pytest.raises(oracle.OracleError) as e:
        oracle.Film(np.full((R, C), L, dtype=np.uint8), L, flags=flags, lib=olib)
    assert e.value.code == -4


def test_bad_heights_rejected(olib):
    with pytest.raises(oracle.OracleError):
        oracle.Film(np.full((4, 4), 5, dtype=np.uint8), 4, lib=olib)


def test_occupancy_rule_and_init(olib):
    """z < H(x, y) is occupied; init up / down / random give +1 / -1 / +-1 there, 0 elsewhere."""
    H = np.array([[0, 1, 2], [3, 2, 0]], dtype=np.uint8)
    for init, vals in ((oracle.INIT_UP, {1}), (oracle.INIT_DOWN, {-1}), (oracle.INIT_RANDOM, {-1, 1})):
        f = oracle.Film(H, 3, init=init, seed=3, lib=olib)
        s = f.spins()
        for z, y, x in itertools.product(range(3), range(2), range(3)):
            if z < H[y, x]:
                assert s[z, y, x] in vals
            else:
                assert s[z, y, x] == 0


def _table1():
    import os
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_critical_concentration.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


def test_table1_rows_obey_eq2():
    """The paper's Table 1: p_c = 2 / z-bar (Eq. 2) on every row, to the printed precision; and
    the concentration is the monolayer count over a 4-layer film, up to rounding of image data."""
    for ml, zbar, tc, p, pc in _table1():
        assert round(2.0 / zbar, 2) == pytest.approx(pc, abs=0.011)
        assert p == pytest.approx(ml / 4.0, abs=0.011)


def test_mean_coordination_and_critical_concentration(olib):
    """z-bar = 2 * bonds / sites: 12 for the bulk, 12 - 6/L for a full periodic L-layer film,
    hence p_c = 2 / z-bar (Eq. 2) = 1/6 in the bulk."""
    f = oracle.Film(np.full((4, 4), 4, dtype=np.uint8), 4, flags=7, lib=olib)
    info = f.info()
    assert 2 * info["n_bonds"] / info["n_occ"] == 12.0
    for n in (1, 2, 3, 5):
        g = oracle.Film(np.full((6, 6), n, dtype=np.uint8), n, flags=3, lib=olib).info()
        assert 2 * g["n_bonds"] / g["n_occ"] == pytest.approx(12.0 - 6.0 / n)


def test_surface_image(olib):
    """Sec. 6: white where the topmost atom of the pixel is up, black where down, no-atom grey."""
    H = np.array([[0, 1, 2], [2, 0, 1]], dtype=np.uint8)
    f = oracle.Film(H, 2, init=oracle.INIT_UP, lib=olib)
    img = f.surface_image()
    assert img.tolist() == [[128, 255, 255], [255, 128, 255]]
    s = f.spins()
    s[1, 0, 2] = -1                       # the top atom of pixel (x=2, y=0) is at z = 1
    s[0, 1, 2] = -1                       # the top atom of pixel (x=2, y=1) is at z = 0
    s[0, 0, 2] = -1                       # below a surface atom: not visible
    f.set_spins(s)
    img = f.surface_image()
    assert img.tolist() == [[128, 255, 0], [255, 128, 0]]


# Pixels touch when their columns are in-plane neighbours: (x +- 1, y), (x, y +- 1),
# (x + 1, y - 1), (x - 1, y + 1); as a 3x3 structure over [dy + 1][dx + 1]:
TRIANGULAR = np.array([[0, 1, 1], [1, 1, 1], [1, 1, 0]])


@pytest.mark.parametrize("seed,shape", [(1, (9, 13)), (2, (20, 20)), (3, (1, 17)), (4, (31, 7)), (5, (12, 40))])
def test_domain_stats_equal_scipy_labelling(seed, shape):
    """The oracle's breadth-first domains equal scipy.ndimage.label with the triangular
    connectivity, colour by colour, on random open images (with no-atom pixels)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.Generator(np.random.PCG64(seed))
    img = rng.choice(np.array([0, 128, 255], dtype=np.uint8), size=shape, p=[0.45, 0.1, 0.45])
    got = oracle.domain_stats(img)
    for v, key in ((255, "white"), (0, "black")):
        lab, n = ndimage.label(img == v, structure=TRIANGULAR)
        sizes = np.bincount(lab.ravel())[1:]
        assert got[key] == n
        assert got["largest_" + key] == (int(sizes.max()) if n else 0)


def test_domain_stats_special_cases():
    """Hand-checked images: one diagonal chain touches along (1, -1) but not along (1, 1); a
    stripe across the periodic edge is one domain; a checkerboard is all separate pixels in
    the open case but joined along the triangular diagonal."""
    img = np.full((3, 3), 128, dtype=np.uint8)
    img[2, 0] = img[1, 1] = img[0, 2] = 255                 # (x, y) = (0,2), (1,1), (2,0): dx=+1, dy=-1
    assert oracle.domain_stats(img)["white"] == 1
    img = np.full((3, 3), 128, dtype=np.uint8)
    img[0, 0] = img[1, 1] = img[2, 2] = 255                 # dx=+1, dy=+1: not bonded
    assert oracle.domain_stats(img) == {"white": 3, "black": 0, "largest_white": 1, "largest_black": 0}
    img = np.zeros((4, 6), dtype=np.uint8)
    img[:, 0] = img[:, 5] = 255                             # two edge columns
    assert oracle.domain_stats(img)["white"] == 2
    assert oracle.domain_stats(img, periodic_x=True)["white"] == 1
    assert oracle.domain_stats(img, periodic_x=True)["largest_white"] == 8
    img = np.zeros((4, 4), dtype=np.uint8)
    img[0, :] = img[3, :] = 255
    assert oracle.domain_stats(img, periodic_y=True) == {"white": 1, "black": 1, "largest_white": 8,
                                                          "largest_black": 8}
    chk = (np.add.outer(np.arange(4), np.arange(4)) % 2 * 255).astype(np.uint8)
    # (x, y) and (x + 1, y - 1) share the parity of x + y: the diagonals x + y = const join up
    assert oracle.domain_stats(chk)["white"] + oracle.domain_stats(chk)["black"] == 7
