"""Pins of the oracle's MCMC densification rules (relocation of dead
Gaussians and noise on the means; no GPU) by their defining properties:
N stacked copies composite to the source's alpha at the centre and to the
same alpha integral along a line (checked by quadrature), draws follow the
cumulative opacity, and the noise gate and covariance match closed forms."""
import numpy as np
import pytest

from oracle import mcmc


@pytest.mark.parametrize("o", [0.02, 0.3, 0.9, 0.995])
def test_one_copy_leaves_a_gaussian_unchanged(o):
    oN, sN = mcmc.relocated_opacity_scale(o, [0.1, 0.2, 0.3], 1)
    assert abs(oN - o) < 1e-15
    assert np.allclose(sN, [0.1, 0.2, 0.3], rtol=1e-14)


@pytest.mark.parametrize("o", [0.02, 0.3, 0.9, 0.995])
@pytest.mark.parametrize("N", [2, 3, 5, 8])
def test_stacked_copies_composite_like_the_source(o, N):
    s = 0.7
    oN, sN = mcmc.relocated_opacity_scale(o, [s], N, bounded=False)
    sN = float(sN[0])
    # alpha at the centre after compositing N copies front to back
    assert abs((1.0 - (1.0 - oN) ** N) - o) < 1e-12
    # integral of the composited alpha along a line through the centre
    x = np.linspace(-12 * max(s, sN), 12 * max(s, sN), 400001)
    a_N = 1.0 - (1.0 - oN * np.exp(-x * x / (2 * sN * sN))) ** N
    a_1 = o * np.exp(-x * x / (2 * s * s))
    assert abs(np.trapezoid(a_N, x) - np.trapezoid(a_1, x)) <= 1e-9 * np.trapezoid(a_1, x)
    # the copies are fainter and no wider than the source
    assert oN < o and sN <= s * (1 + 1e-12)


def test_draws_follow_the_cumulative_opacity():
    op = np.array([0.5, 0.001, 0.2, 0.3])       # Gaussian 1 is dead
    dead = op <= mcmc.DEAD_OPACITY
    total = 1.0
    # intervals: [0, .5) -> 0, [.5, .7) -> 2, [.7, 1) -> 3
    u = np.array([0.0, 0.49, 0.5, 0.69, 0.7, 0.999]) / total
    assert list(mcmc.draw_sources(op, dead, u)) == [0, 0, 2, 2, 3, 3]


def _params(n, rng):
    return dict(mean=rng.normal(size=(n, 3)), log_scale=rng.normal(-2, 0.3, (n, 3)),
                quat=rng.normal(size=(n, 4)), opacity_logit=rng.normal(0, 2, n), sh=rng.normal(size=(n, 4, 3)))


def test_relocation_moves_dead_gaussians_onto_their_sources():
    rng = np.random.default_rng(0)
    p = _params(40, rng)
    p["opacity_logit"][[3, 7, 11]] = -8.0          # dead: sigmoid(-8) = 3.4e-4
    u = rng.uniform(size=3)
    out, src = mcmc.relocate(p, u)
    o_before = mcmc.sigmoid(p["opacity_logit"])
    assert len(src) == 3 and not np.isin(src, [3, 7, 11]).any()
    counts = np.bincount(src, minlength=40)
    for d, j in zip([3, 7, 11], src):
        for k in p:
            np.testing.assert_array_equal(out[k][d], out[k][j])
    for j in np.nonzero(counts)[0]:
        N = counts[j] + 1
        oN = mcmc.sigmoid(out["opacity_logit"][j])
        assert abs((1 - (1 - oN) ** N) - o_before[j]) < 1e-12
    untouched = [i for i in range(40) if i not in (3, 7, 11) and counts[i] == 0]
    for k in p:
        np.testing.assert_array_equal(out[k][untouched], p[k][untouched])


def test_nothing_to_relocate_or_nothing_alive():
    rng = np.random.default_rng(1)
    p = _params(10, rng)
    p["opacity_logit"][:] = 1.0
    out, src = mcmc.relocate(p, [])
    assert len(src) == 0 and all(np.array_equal(out[k], p[k]) for k in p)
    p["opacity_logit"][:] = -9.0
    out, src = mcmc.relocate(p, rng.uniform(size=10))
    assert len(src) == 0 and all(np.array_equal(out[k], p[k]) for k in p)


def test_noise_is_gated_by_opacity_and_shaped_by_the_covariance():
    mean = np.zeros((3, 3))
    log_scale = np.log(np.array([[0.1, 0.2, 0.3]] * 3))
    quat = np.array([[1.0, 0, 0, 0]] * 3)           # identity rotation
    logit = np.log(np.array([1e-4, 0.005, 0.5]) / (1 - np.array([1e-4, 0.005, 0.5])))
    eta = np.tile([1.0, 1.0, 1.0], (3, 1))
    out = mcmc.noise_means(mean, log_scale, quat, logit, eta, noise_lr=2.0)
    gate = 1 / (1 + np.exp(100 * (np.array([1e-4, 0.005, 0.5]) - 0.005)))
    exp = 2.0 * gate[:, None] * np.array([0.01, 0.04, 0.09])
    assert np.abs(out - exp).max() < 1e-15
    assert abs(gate[1] - 0.5) < 1e-12 and gate[2] < 1e-20
    # a rotated Gaussian: Sigma = R diag(s^2) R^T
    q = np.array([[np.cos(0.4), 0.0, 0.0, np.sin(0.4)]])   # 0.8 rad about z
    S = mcmc.covariance(np.log([[0.1, 0.2, 0.3]]), q)[0]
    c, s_ = np.cos(0.8), np.sin(0.8)
    R = np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1]])
    assert np.abs(S - R @ np.diag([0.01, 0.04, 0.09]) @ R.T).max() < 1e-15


def test_reset_opacity_is_bounded():
    """A faint source drawn several times would give copies at or below the
    dead threshold (o = 0.012, N = 3: o_N = 0.004); an opaque one would give
    o_N = 1 and an infinite logit.  The bounds keep both inside
    [0.005, 1 - 2^-23]; the scale is the unbounded rule's."""
    oN, sN = mcmc.relocated_opacity_scale(0.012, [0.3], 3)
    oN_u, sN_u = mcmc.relocated_opacity_scale(0.012, [0.3], 3, bounded=False)
    assert oN_u < 0.005 and oN == 0.005 and np.array_equal(sN, sN_u)
    o = mcmc.sigmoid(40.0)                          # rounds to 1 in double
    oN, _ = mcmc.relocated_opacity_scale(o, [0.3], 1)
    assert oN == mcmc.MAX_OPACITY and np.isfinite(np.log(oN / (1 - oN)))


def test_growth_count_rule():
    assert mcmc.n_grow(100, 1000) == 5
    assert mcmc.n_grow(990, 1000) == 10
    assert mcmc.n_grow(1000, 1000) == 0 and mcmc.n_grow(1200, 1000) == 0
    assert mcmc.n_grow(19, 1000) == 0                 # floor(19.95) = 19


def test_growth_appends_reset_copies_of_drawn_sources():
    rng = np.random.default_rng(5)
    p = _params(30, rng)
    p["opacity_logit"][[4, 9]] = -9.0               # dead: never drawn
    u = rng.uniform(size=6)
    out, src = mcmc.grow(p, u)
    assert len(src) == 6 and all(len(out[k]) == 36 for k in out)
    assert not np.isin(src, [4, 9]).any()
    np.testing.assert_array_equal(src, mcmc.draw_sources(mcmc.sigmoid(p["opacity_logit"]),
                                                         mcmc.sigmoid(p["opacity_logit"]) <= mcmc.DEAD_OPACITY, u))
    for i, j in enumerate(src):
        for k in p:
            np.testing.assert_array_equal(out[k][30 + i], out[k][j])
    counts = np.bincount(src, minlength=30)
    o0 = mcmc.sigmoid(p["opacity_logit"])
    for j in np.nonzero(counts)[0]:
        oN = mcmc.sigmoid(out["opacity_logit"][j])
        exp = max(1 - (1 - o0[j]) ** (1.0 / (counts[j] + 1)), mcmc.DEAD_OPACITY)
        assert abs(oN - exp) < 1e-12
    for j in np.nonzero(counts == 0)[0]:
        for k in p:
            np.testing.assert_array_equal(out[k][j], p[k][j])
