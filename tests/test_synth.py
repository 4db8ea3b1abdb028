"""The seeded input generators (CPU): the ground-truth convention I1(x + gt(x)) ~ I0(x) that every
end-point error in the GPU tests and the bench relies on, the stereo and RGB variants, seeding
and value ranges.  The generators use scipy's filters and interpolation; these checks warp with
scipy too, so they test the generators' geometry, not an interpolator."""
import numpy as np
import pytest
from scipy import ndimage

from paper_1603_03590_gb300 import synth


def warp_back(I1, gt):
    """I1(x + gt(x)) by linear interpolation, edge clamped."""
    h, w = I1.shape
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    return ndimage.map_coordinates(I1.astype(np.float64), [ys + gt[..., 1], xs + gt[..., 0]], order=1, mode="nearest")


def test_translation_pair_convention():
    I0, I1, gt = synth.translation_pair(3)
    assert I0.shape == I1.shape == (96, 128) and gt.shape == (96, 128, 2)
    assert I0.dtype == I1.dtype == gt.dtype == np.float32
    assert np.all(gt[..., 0] == np.float32(2.3)) and np.all(gt[..., 1] == np.float32(-1.7))
    err = np.abs(warp_back(I1, gt) - I0)[4:-4, 4:-4]  # away from the clamped border
    # two linear interpolations of a sigma-2 texture: small against the frames' own difference
    assert err.mean() < 0.1 * np.abs(I1 - I0)[4:-4, 4:-4].mean()
    assert err.max() < 0.05


@pytest.mark.parametrize("seed,horizontal", [(11, False), (12, False), (13, True)])
def test_layered_pair_ground_truth_explains_frame_1(seed, horizontal):
    """Outside occlusions and layer boundaries, frame 1 sampled along the ground truth equals
    frame 0; without the motion the typical difference is several times larger."""
    I0, I1, gt = synth.layered_pair(seed, width=256, height=128, n_ellipses=4, max_disp=8.0, horizontal=horizontal)
    assert I0.shape == I1.shape == (128, 256) and gt.shape == (128, 256, 2)
    assert 0.0 <= I0.min() and I0.max() <= 1.0 and 0.0 <= I1.min() and I1.max() <= 1.0
    inner = (slice(10, -10), slice(10, -10))
    moved = np.abs(warp_back(I1, gt) - I0)[inner]
    unmoved = np.abs(I1.astype(np.float64) - I0)[inner]
    assert (moved < 0.02).mean() > 0.85, (moved < 0.02).mean()
    # the textures are smooth, so many pixels match by chance without the motion; the typical
    # error with it is still a small fraction of the typical error without it
    assert np.median(moved) < 0.4 * np.median(unmoved)
    if horizontal:
        assert np.all(gt[..., 1] == 0.0) and np.abs(gt[..., 0]).max() > 0.5


def test_stereo_pair_refuses_rotation():
    with pytest.raises(ValueError):
        synth.layered_pair(1, width=64, height=48, n_ellipses=1, horizontal=True, rotation_deg=1.0)


def test_rgb_shares_the_grayscale_geometry():
    """The geometry is drawn before the textures, so the RGB pair of a seed has the grayscale
    pair's ground truth; its channels carry independent textures."""
    _, _, gt1 = synth.layered_pair(21, width=96, height=64, n_ellipses=3, max_disp=6.0)
    I0, I1, gt3 = synth.layered_pair(21, width=96, height=64, n_ellipses=3, max_disp=6.0, channels=3)
    assert I0.shape == I1.shape == (3, 64, 96)
    assert np.array_equal(gt1, gt3)
    assert not np.array_equal(I0[0], I0[1]) and not np.array_equal(I0[1], I0[2])
    for c in range(3):
        ok = np.abs(warp_back(I1[c], gt3) - I0[c])[6:-6, 6:-6] < 0.02
        assert ok.mean() > 0.8


def test_rotation_is_composed_on_top():
    """A pure rotation (no ellipses, background motion drawn as usual) moves the corners of the
    frame by about theta times their distance from the centre."""
    _, _, g0 = synth.layered_pair(31, width=200, height=100, n_ellipses=0, max_disp=0.0)
    _, _, g2 = synth.layered_pair(31, width=200, height=100, n_ellipses=0, max_disp=0.0, rotation_deg=2.0)
    d = g2 - g0
    r = np.hypot(99.5, 49.5)
    assert abs(np.hypot(*d[0, 0]) - np.radians(2.0) * r) < 0.05 * np.radians(2.0) * r
    assert np.hypot(*d[50, 100]) < 0.05  # the pixel next to the centre barely moves


def test_seeding_is_deterministic():
    a = synth.layered_pair(41, width=80, height=48, n_ellipses=2, max_disp=4.0)
    b = synth.layered_pair(41, width=80, height=48, n_ellipses=2, max_disp=4.0)
    c = synth.layered_pair(42, width=80, height=48, n_ellipses=2, max_disp=4.0)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])


def test_mixed_resolutions_and_workload_table():
    sizes = synth.mixed_resolutions(2000, 64)
    assert len(sizes) == 64 and set(sizes) <= set(synth.MIXED_SIZES)
    assert len(set(sizes)) == len(synth.MIXED_SIZES)  # 64 uniform draws reach every size
    assert synth.mixed_resolutions(2000, 64) == sizes
    I0, I1, gt = synth.workload_pair("stereo320x240", 0)
    assert I0.shape == (240, 320) and np.all(gt[..., 1] == 0.0)
    I0, _, gt = synth.workload_pair("translate128x96", 0)
    assert I0.shape == (96, 128)
    with pytest.raises(KeyError):
        synth.workload_pair("no such workload", 0)
