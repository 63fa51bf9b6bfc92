"""Pins of the superpixel reference (oracle/slic_ref.py): on a constant
image SLIC keeps the initial grid cells; with a weak spatial term no
superpixel straddles a strong intensity edge; the dilation of one pixel is a
(2 gamma + 1)^2 square; patches tile their boxes with packed offsets."""
import numpy as np

from oracle import slic_ref


def test_constant_image_gives_the_voronoi_cells_of_the_grid():
    """One assignment on a constant image is the nearest grid centre (brute
    force over all centres, ties to the lower index)."""
    img = np.full((48, 40), 5.0, np.float32)
    lab, K = slic_ref.slic_labels(img, 8, 10.0, 1)
    nx, ny = 5, 6
    assert K == nx * ny
    cx = np.array([(i + 0.5) * 8 for j in range(ny) for i in range(nx)])
    cy = np.array([(j + 0.5) * 8 for j in range(ny) for i in range(nx)])
    yy, xx = np.meshgrid(np.arange(48), np.arange(40), indexing="ij")
    d = (xx[..., None] - cx) ** 2 + (yy[..., None] - cy) ** 2
    assert np.array_equal(lab, np.argmin(d, axis=-1))


def test_superpixels_follow_an_intensity_edge():
    img = np.zeros((40, 40), np.float32)
    img[:, 17:] = 1000.0
    lab, K = slic_ref.slic_labels(img, 10, 0.5, 10)
    for c in range(K):
        m = lab == c
        if m.any():
            assert len(np.unique(img[m])) == 1, c


def test_patch_boxes_members_and_offsets():
    rng = np.random.default_rng(3)
    stacks = [rng.uniform(0, 100, (2, 30, 36)).astype(np.float32)]
    desc, member, npix = slic_ref.patches_build_slic([(36, 30, 2)], stacks, 10, 5.0, 2, n_iter=4)
    assert desc.shape[0] > 0 and member.size == npix
    off = 0
    for r in desc:
        assert r[6] == off and r[2] >= 0 and r[3] >= 0 and r[2] + r[4] <= 36 and r[3] + r[5] <= 30
        m = member[off:off + r[4] * r[5]].reshape(r[5], r[4])
        # the box is exactly the dilated superpixel's bounding box (clipped)
        assert m[0].any() or r[3] == 0
        assert m.any(axis=0).all() and m.any(axis=1).all()
        off += r[4] * r[5]
    # dilation of a single pixel
    img = np.zeros((20, 20), np.float32)
    lab = np.full((20, 20), 1)
    lab[9, 9] = 0
    one = (lab == 0)
    box = one[9 - 3:9 + 4, 9 - 3:9 + 4]
    assert box.sum() == 1
