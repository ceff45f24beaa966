"""GPU graph construction against the oracle: labels, node order and neighbour table bit-exact."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _compare(vga, oracle_lib, img, keep_largest=True):
    g = vga.Graph(img, keep_largest=keep_largest)
    og = oracle_lib.graph_build(img, keep_largest=keep_largest)
    assert (g.n, g.n_components, g.largest) == (og.n, og.n_components, og.largest)
    ex = g.export()
    assert np.array_equal(ex["labels"], og.labels)
    assert np.array_equal(ex["voxel_of_node"], og.voxel_of_node)
    assert np.array_equal(ex["nbr"], og.nbr)
    g.close()
    return og


def test_every_2x2x2_mask(vga, oracle_lib):
    for bits in range(256):
        img = np.array([(bits >> k) & 1 for k in range(8)], dtype=np.uint8).reshape(2, 2, 2)
        _compare(vga, oracle_lib, img, keep_largest=bool(bits & 1))


@pytest.mark.parametrize("shape,por,seed", [((37, 5, 3), 0.5, 1), ((1, 1, 1), 0.0, 2), ((1, 1, 70), 0.3, 3),
                                            ((70, 1, 1), 0.3, 4), ((3, 70, 33), 0.45, 5), ((9, 8, 65), 0.4, 6),
                                            ((5, 4, 31), 0.6, 7)])
def test_ragged_random_masks(vga, oracle_lib, shape, por, seed):
    rng = np.random.default_rng(seed)
    img = (rng.random(shape) < por).astype(np.uint8)
    _compare(vga, oracle_lib, img, True)
    _compare(vga, oracle_lib, img, False)


def test_constructed_masks(vga, oracle_lib):
    _compare(vga, oracle_lib, np.ones((4, 5, 6), dtype=np.uint8))   # no pores
    _compare(vga, oracle_lib, np.zeros((4, 5, 6), dtype=np.uint8))  # one component
    z, y, x = np.meshgrid(np.arange(6), np.arange(7), np.arange(40), indexing="ij")
    _compare(vga, oracle_lib, ((x + y + z) % 2).astype(np.uint8), False)  # all isolated
    _compare(vga, oracle_lib, ((x + y + z) % 2).astype(np.uint8), True)
    img = np.zeros((7, 3, 4), dtype=np.uint8)
    img[1::2] = 1
    _compare(vga, oracle_lib, img, True)  # equal-size tie: lowest id wins
    assert _compare(vga, oracle_lib, 255 * img, False).n_components == 4  # any nonzero is solid


@pytest.mark.parametrize("shape,por,seed", [((64, 64, 64), 0.17, 1), ((96, 80, 130), 0.2, 9)])
def test_smoothed_masks(vga, oracle_lib, shape, por, seed):
    img = synth.pore_mask(shape, por, seed)
    _compare(vga, oracle_lib, img, True)
    _compare(vga, oracle_lib, img, False)


def test_device_image_input(vga, oracle_lib):
    import torch

    img = synth.pore_mask((20, 30, 40), 0.25, 4)
    g = vga.Graph(torch.from_numpy(img).cuda(), keep_largest=True)
    og = oracle_lib.graph_build(img)
    assert g.n == og.n and np.array_equal(g.export()["nbr"], og.nbr)


def test_full_size_512(vga, oracle_lib):
    """512^3 at 17% porosity, the paper's image size (Sec. IV.A): bit-exact against the oracle."""
    img = synth.pore_mask((512, 512, 512), 0.17, 3)
    og = _compare(vga, oracle_lib, img, True)
    assert og.n > 2.0e7
