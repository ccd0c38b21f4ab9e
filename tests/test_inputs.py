"""The seeded synthetic inputs follow their stated recipe: the two-phase
inclusion composites (stop at the first disk that reaches the soft fraction),
the thresholded Gaussian foam (exact solid fraction), the uneven batch (sides
and fractions in their ranges), and determinism under a fixed seed."""
import numpy as np

from gen.images import batch_specimens, foam_volume, inclusion_image, warmstart_specimens


def test_inclusion_image_recipe():
    img = inclusion_image(64, 64, 3.0, 8.0, 0.30, 0)
    assert img.shape == (64, 64) and img.dtype == np.uint8
    assert set(np.unique(img)) <= {1, 2}
    soft = np.count_nonzero(img == 2) / img.size
    # at least the target, and over it by less than one disk of the largest radius
    assert 0.30 <= soft < 0.30 + np.pi * 8.0 ** 2 / img.size
    assert np.array_equal(img, inclusion_image(64, 64, 3.0, 8.0, 0.30, 0))  # deterministic
    assert not np.array_equal(img, inclusion_image(64, 64, 3.0, 8.0, 0.30, 1))
    big = inclusion_image(256, 192, 10.0, 60.0, 0.30, 1)  # ragged, large radii
    assert big.shape == (192, 256)
    assert 0.30 <= np.count_nonzero(big == 2) / big.size < 0.30 + np.pi * 60.0 ** 2 / big.size


def test_foam_volume_recipe():
    v = foam_volume(32, 2.0, 0.35, seed=2)
    assert v.shape == (32, 32, 32) and set(np.unique(v)) <= {0, 1}
    # thresholded at the 65th percentile of the smoothed noise
    assert abs(np.count_nonzero(v) - 0.35 * v.size) <= 1
    assert np.array_equal(v, foam_volume(32, 2.0, 0.35, seed=2))
    # smoothing makes solid voxels cluster: far more solid-solid face pairs than
    # independent voxels at the same fraction would give
    pairs = np.count_nonzero(v[1:] & v[:-1]) / (31 * 32 * 32)
    assert pairs > 0.35 ** 2 + 0.1


def test_batch_and_warmstart_specimens():
    imgs = batch_specimens(12)
    assert len(imgs) == 12
    for im in imgs:
        assert im.shape[0] == im.shape[1] and 32 <= im.shape[0] <= 512
        soft = np.count_nonzero(im == 2) / im.size
        assert 0.10 <= soft < 0.50 + np.pi * 64 / im.size
    assert len({im.shape[0] for im in imgs}) > 1  # uneven sizes
    again = batch_specimens(12)
    assert all(np.array_equal(a, b) for a, b in zip(imgs, again))
    ws = warmstart_specimens([1000, 1001], side=64)
    assert [w.shape for w in ws] == [(64, 64), (64, 64)] and not np.array_equal(ws[0], ws[1])
