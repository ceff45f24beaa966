"""Pins of the oracle's graph construction (Sec. II.A, Fig. 2; Sec. III) against brute force,
scipy.ndimage.label and constructed masks with known structure."""
import numpy as np
import pytest
from scipy import ndimage

from tests.helpers import brute_components, kept_coords

OPP = [1, 0, 3, 2, 5, 4]
STEP = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]  # (dz, dy, dx)


def _check_graph(oracle, img, keep_largest):
    g = oracle.graph_build(img, keep_largest=keep_largest)
    pore = img == 0
    comp, ncomp = brute_components(pore)
    assert g.n_components == ncomp
    lab = -np.ones(img.size, dtype=np.int64)
    lab[np.flatnonzero(pore.ravel())] = comp
    assert np.array_equal(g.labels.ravel(), lab)
    if ncomp == 0:
        assert g.largest == -1 and g.n == 0
        return g
    sizes = np.bincount(comp, minlength=ncomp)
    largest = int(np.flatnonzero(sizes == sizes.max())[0])
    assert g.largest == largest
    kept = pore & (g.labels == largest) if keep_largest else pore
    assert np.array_equal(g.voxel_of_node, np.flatnonzero(kept.ravel()))
    # neighbour table from coordinates
    c = kept_coords(kept)
    index = {tuple(v): i for i, v in enumerate(c)}
    for i, v in enumerate(c):
        for d, s in enumerate(STEP):
            u = (v[0] + s[0], v[1] + s[1], v[2] + s[2])
            assert g.nbr[i, d] == index.get(u, -1)
    return g


def test_every_2x2x2_mask(oracle_lib):
    for bits in range(256):
        img = np.array([(bits >> k) & 1 for k in range(8)], dtype=np.uint8).reshape(2, 2, 2)
        _check_graph(oracle_lib, img, keep_largest=False)
        _check_graph(oracle_lib, img, keep_largest=True)


@pytest.mark.parametrize("shape,por,seed", [((5, 7, 6), 0.5, 1), ((1, 1, 9), 0.6, 2), ((3, 1, 4), 0.5, 3),
                                            ((4, 5, 3), 0.3, 4), ((6, 6, 6), 0.55, 5)])
def test_random_masks_brute_force(oracle_lib, shape, por, seed):
    rng = np.random.default_rng(seed)
    img = (rng.random(shape) >= por).astype(np.uint8)
    _check_graph(oracle_lib, img, keep_largest=True)
    _check_graph(oracle_lib, img, keep_largest=False)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_partition_matches_scipy_label(oracle_lib, seed):
    import synth

    img = synth.pore_mask((24, 20, 28), 0.2, seed)
    g = oracle_lib.graph_build(img, keep_largest=False)
    lab, nc = ndimage.label(img == 0, structure=ndimage.generate_binary_structure(3, 1))
    assert g.n_components == nc
    # same partition: a bijection between the two labelings on pore voxels
    m = img.ravel() == 0
    a, b = g.labels.ravel()[m], lab.ravel()[m]
    pairs = np.unique(np.stack([a, b]), axis=1)
    assert pairs.shape[1] == nc
    # ids are ordered by each component's first raster voxel
    first = np.array([np.flatnonzero(g.labels.ravel() == k)[0] for k in range(nc)])
    assert np.all(np.diff(first) > 0)
    sizes = np.bincount(a)
    gk = oracle_lib.graph_build(img, keep_largest=True)
    assert gk.n == sizes.max()
    assert gk.largest == int(np.argmax(sizes))


def test_checkerboard_all_isolated(oracle_lib):
    z, y, x = np.meshgrid(np.arange(5), np.arange(4), np.arange(6), indexing="ij")
    img = ((x + y + z) % 2).astype(np.uint8)  # pores where x+y+z is even: no two share a face
    g = oracle_lib.graph_build(img, keep_largest=False)
    assert g.n_components == int((img == 0).sum())
    assert np.all(g.nbr == -1)
    gk = oracle_lib.graph_build(img, keep_largest=True)
    assert gk.n == 1 and gk.voxel_of_node[0] == 0 and gk.largest == 0


def test_full_box_degrees(oracle_lib):
    img = np.zeros((4, 5, 6), dtype=np.uint8)
    g = oracle_lib.graph_build(img)
    assert g.n == img.size and g.n_components == 1
    assert np.array_equal(g.voxel_of_node, np.arange(img.size))
    deg = (g.nbr >= 0).sum(axis=1).reshape(img.shape)
    z, y, x = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    on_face = (x == 0).astype(int) + (x == 5) + (y == 0) + (y == 4) + (z == 0) + (z == 3)
    assert np.array_equal(deg, 6 - on_face)
    # in a full box the -x neighbour of node i is node i-1 unless x == 0
    i = np.arange(img.size)
    has = (i % 6) > 0
    assert np.array_equal(g.nbr[has, 0], i[has] - 1)


def test_slab_layers(oracle_lib):
    img = np.zeros((7, 3, 4), dtype=np.uint8)
    img[1::2] = 1  # pore layers z = 0, 2, 4, 6
    g = oracle_lib.graph_build(img, keep_largest=False)
    assert g.n_components == 4
    for k, z in enumerate((0, 2, 4, 6)):
        assert np.all(g.labels[z] == k)
    gk = oracle_lib.graph_build(img, keep_largest=True)
    assert gk.n == 12 and np.all(gk.nbr[:, 4:] == -1)  # equal sizes: the first layer is kept


def test_empty_and_solid(oracle_lib):
    g = oracle_lib.graph_build(np.ones((3, 3, 3), dtype=np.uint8))
    assert g.n == 0 and g.n_components == 0 and g.largest == -1
    assert np.all(g.labels == -1)
    g1 = oracle_lib.graph_build(np.zeros((1, 1, 1), dtype=np.uint8))
    assert g1.n == 1 and np.all(g1.nbr == -1)


def test_neighbour_symmetry(oracle_lib):
    import synth

    img = synth.pore_mask((16, 12, 20), 0.25, 7)
    g = oracle_lib.graph_build(img)
    for d in range(6):
        j = g.nbr[:, d]
        m = j >= 0
        assert np.array_equal(g.nbr[j[m], OPP[d]], np.flatnonzero(m))


def test_nonzero_solid_values(oracle_lib):
    # any nonzero value is solid (Sec. II.A tags solid as 1; other nonzero codes are treated alike)
    img = np.array([[[0, 2, 0, 255]]], dtype=np.uint8)
    g = oracle_lib.graph_build(img, keep_largest=False)
    assert g.n == 2 and g.n_components == 2


def test_block_interface_helpers(oracle_lib):
    """edge_interface / block_face_weights against a direct per-edge coordinate computation."""
    img = np.zeros((5, 6, 7), dtype=np.uint8)
    img[2, 3, 4] = 1
    g = oracle_lib.graph_build(img)
    bs = 2
    nb = oracle_lib.block_grid(img.shape, bs)
    nI = oracle_lib.interface_count(nb)
    theta = np.arange(1, nI + 1, dtype=np.float64)
    gw = oracle_lib.block_face_weights(img.shape, bs, g.voxel_of_node, g.nbr, theta)
    seen = {}
    c = kept_coords(img == 0)
    for i, v in enumerate(c):
        for d, s in enumerate(STEP):
            j = g.nbr[i, d]
            if j < 0:
                continue
            u = c[j]
            bi, bj = tuple(v // bs), tuple(u // bs)
            if bi == bj:
                assert gw[i, d] == 1.0
            else:
                key = (min(bi, bj), max(bi, bj))
                seen.setdefault(key, gw[i, d])
                assert gw[i, d] == seen[key]  # one value per block pair, symmetric
                assert gw[j, OPP[d]] == gw[i, d]
    # every interface between face-adjacent blocks that has a crossing edge got a distinct theta
    assert len(set(seen.values())) == len(seen)
    assert nI == nb[0] * nb[1] * (nb[2] - 1) + nb[0] * (nb[1] - 1) * nb[2] + (nb[0] - 1) * nb[1] * nb[2]
