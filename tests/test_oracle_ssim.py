"""Pins of the oracle's photometric loss of Eq. 5 (L1 + SSIM) against
closed forms, invariants, an independent library computation and central
finite differences (no GPU)."""
import numpy as np
import pytest

import oracle


def _rand(shape, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=shape)


def test_window_is_a_normalised_sigma_1_5_gaussian():
    w = oracle.ssim_window()
    k = np.arange(-5, 6)
    assert w.shape == (11,)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w[::-1], rtol=0, atol=0)
    assert np.all(np.diff(w[:6]) > 0)
    # second moment of the truncated normal with sigma = 1.5 (the tails
    # beyond 3.3 sigma hold ~1e-3 of the mass)
    assert abs((k * k * w).sum() - 2.25) < 1e-2


def test_ssim_of_an_image_with_itself_is_one_and_stationary():
    x = _rand((13, 11, 3), 0)
    S, _ = oracle.ssim_map(x, x)
    assert np.abs(S - 1.0).max() < 1e-12
    loss, g = oracle.photo_loss_grad(x, x, 0.8, 0.2)
    assert abs(loss) < 1e-12
    # the maximum of SSIM: its gradient vanishes (and sign(0) = 0 for L1)
    assert np.abs(g).max() < 1e-12


def test_constant_images_closed_form_with_border_weights():
    """x = a, y = b everywhere: with s(p) the window mass inside the image
    at pixel p (product of the 1-D partial sums), mx = a s, my = b s,
    vx = a^2 s (1 - s), vy = b^2 s (1 - s), cxy = a b s (1 - s)."""
    H, W, a, b = 14, 12, 0.7, 0.3
    w = oracle.ssim_window()

    def mass(n):
        return np.array([sum(w[k + 5] for k in range(-5, 6) if 0 <= i + k < n) for i in range(n)])

    s = np.outer(mass(H), mass(W))[:, :, None]
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    exp = ((2 * a * b * s * s + C1) * (2 * a * b * s * (1 - s) + C2) /
           ((a * a * s * s + b * b * s * s + C1) * ((a * a + b * b) * s * (1 - s) + C2)))
    S, _ = oracle.ssim_map(np.full((H, W, 1), a), np.full((H, W, 1), b))
    assert np.abs(S - exp).max() < 1e-12
    # away from the border the window is whole: (2ab + C1) / (a^2 + b^2 + C1)
    assert abs(S[7, 6, 0] - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-12


def test_window_sums_match_a_library_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    x, y = _rand((17, 23, 3), 1), _rand((17, 23, 3), 2)
    w = oracle.ssim_window()
    k2 = np.outer(w, w)

    def lib(a):
        return np.stack([ndimage.correlate(a[:, :, c], k2, mode="constant", cval=0.0) for c in range(3)], 2)

    mx, my = lib(x), lib(y)
    vx, vy, cxy = lib(x * x) - mx * mx, lib(y * y) - my * my, lib(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    S_lib = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    S, _ = oracle.ssim_map(x, y)
    assert np.abs(S - S_lib).max() < 1e-12
    assert np.abs(oracle.window_sum(x) - mx).max() < 1e-14


def test_ssim_symmetric_and_at_most_one():
    x, y = _rand((9, 10, 3), 3), _rand((9, 10, 3), 4)
    S1, _ = oracle.ssim_map(x, y)
    S2, _ = oracle.ssim_map(y, x)
    assert np.abs(S1 - S2).max() < 1e-14
    assert S1.max() <= 1.0 + 1e-12


@pytest.mark.parametrize("l1w,sw", [(0.8, 0.2), (0.0, 1.0), (1.0, 0.0)])
def test_gradient_matches_central_differences(l1w, sw):
    x, y = _rand((7, 6, 3), 5), _rand((7, 6, 3), 6)
    _, g = oracle.photo_loss_grad(x, y, l1w, sw)
    h = 1e-6
    fd = np.zeros_like(x)
    for idx in np.ndindex(*x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd[idx] = (oracle.photo_loss_grad(xp, y, l1w, sw)[0] - oracle.photo_loss_grad(xm, y, l1w, sw)[0]) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max() + 1e-12


def test_loss_weights_split_l1_and_ssim():
    x, y = _rand((8, 9, 3), 7), _rand((8, 9, 3), 8)
    S, _ = oracle.ssim_map(x, y)
    l1 = np.abs(x - y).mean()
    assert abs(oracle.photo_loss_grad(x, y, 1.0, 0.0)[0] - l1) < 1e-15
    assert abs(oracle.photo_loss_grad(x, y, 0.0, 1.0)[0] - (1.0 - S.mean())) < 1e-15
    assert abs(oracle.photo_loss_grad(x, y, 0.8, 0.2)[0] - (0.8 * l1 + 0.2 * (1.0 - S.mean()))) < 1e-15
