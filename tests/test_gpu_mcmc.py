"""Parity of the MCMC densification kernels (gs_mcmc_relocate,
gs_mcmc_noise) with the FP64 oracle (oracle/mcmc.py) on the float32-rounded
parameters the GPU holds; the random draws are inputs on both sides."""
import numpy as np
import pytest

from oracle import mcmc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ["mean", "log_scale", "quat", "opacity_logit", "sh"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _scene(n, seed, dead_frac):
    rng = np.random.default_rng(seed)
    p = dict(mean=rng.normal(size=(n, 3)), log_scale=rng.normal(-3, 0.3, (n, 3)), quat=rng.normal(size=(n, 4)),
             opacity_logit=rng.normal(0, 2, n), sh=rng.normal(0, 0.3, (n, 16, 3)))
    dead = rng.choice(n, int(dead_frac * n), replace=False)
    p["opacity_logit"][dead] = rng.uniform(-12.0, -5.5, len(dead))      # sigmoid(-5.5) = 0.0041
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}


def _gpu(p):
    from paper_2603_04847_gb300 import Gaussians
    return Gaussians.from_numpy(p)


def _host(g):
    return {k: t.detach().cpu().numpy().astype(np.float64) for k, t in zip(KEYS, g.tensors())}


def _relocate(p, u):
    from paper_2603_04847_gb300.core import gs_mcmc_relocate
    g = _gpu(p)
    src = torch.full((len(p["opacity_logit"]),), -7, dtype=torch.int32, device="cuda")
    nd = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs_mcmc_relocate(g, torch.as_tensor(u, dtype=torch.float64, device="cuda"), src, nd)
    torch.cuda.synchronize()
    return _host(g), src.cpu().numpy(), int(nd.item())


def test_relocation_matches_the_oracle():
    p = _scene(5000, 0, 0.08)
    dead = mcmc.sigmoid(p["opacity_logit"]) <= mcmc.DEAD_OPACITY
    u = np.random.default_rng(1).uniform(size=int(dead.sum()))
    exp, src_e = mcmc.relocate(p, u)
    got, src, nd = _relocate(p, u)
    assert nd == dead.sum() > 350
    assert (src[~dead] == -1).all()
    np.testing.assert_array_equal(src[dead], src_e)
    for k in KEYS:
        assert np.abs(got[k] - exp[k]).max() <= 1e-5 * max(1.0, np.abs(exp[k]).max()), k
    # the sources drawn more than once were reset: the stack composites to
    # the old alpha at the centre
    counts = np.bincount(src_e, minlength=5000)
    j = int(np.argmax(counts))
    assert counts[j] >= 1
    oN = mcmc.sigmoid(got["opacity_logit"][j])
    assert abs((1 - (1 - oN) ** (counts[j] + 1)) - mcmc.sigmoid(p["opacity_logit"][j])) < 1e-5


def test_relocation_with_no_dead_gaussian_changes_nothing():
    p = _scene(1000, 2, 0.0)
    p["opacity_logit"] = np.maximum(p["opacity_logit"], -3.0)      # none below 0.005
    got, src, nd = _relocate(p, np.zeros(1))
    assert nd == 0 and (src == -1).all()
    for k in KEYS:
        np.testing.assert_array_equal(got[k], p[k])


def test_noise_matches_the_oracle():
    from paper_2603_04847_gb300.core import gs_mcmc_noise
    p = _scene(3000, 3, 0.3)
    eta = np.asarray(np.random.default_rng(4).normal(size=(3000, 3)), np.float32).astype(np.float64)
    exp = mcmc.noise_means(p["mean"], p["log_scale"], p["quat"], p["opacity_logit"], eta, 1.0)
    g = _gpu(p)
    gs_mcmc_noise(g, torch.as_tensor(eta, dtype=torch.float32, device="cuda"), 1.0)
    torch.cuda.synchronize()
    got = _host(g)["mean"]
    assert np.abs(got - exp).max() <= 1e-6
    moved = np.abs(exp - p["mean"]).max(axis=1) > 1e-4
    assert moved.sum() > 500 and (~moved).sum() > 500   # the gate separates dead from opaque


def _grow(p, n, u):
    from paper_2603_04847_gb300.core import gs_mcmc_grow
    n_add = len(u)
    big = {k: np.concatenate([v, np.zeros((n_add,) + v.shape[1:])], 0) for k, v in p.items()}
    g = _gpu(big)
    src = torch.full((n_add,), -7, dtype=torch.int32, device="cuda")
    gs_mcmc_grow(g, n, torch.as_tensor(u, dtype=torch.float64, device="cuda"), src)
    torch.cuda.synchronize()
    return _host(g), src.cpu().numpy()


def test_growth_matches_the_oracle():
    """The growth step (5 % more Gaussians, below the cap): draws bit-exact,
    sources reset, new rows copies of them."""
    p = _scene(5000, 6, 0.08)
    n_add = mcmc.n_grow(5000, 6000)
    assert n_add == 250
    u = np.random.default_rng(7).uniform(size=n_add)
    exp, src_e = mcmc.grow(p, u)
    got, src = _grow(p, 5000, u)
    np.testing.assert_array_equal(src, src_e)
    for k in KEYS:
        assert np.abs(got[k] - exp[k]).max() <= 1e-5 * max(1.0, np.abs(exp[k]).max()), k
    for i, j in enumerate(src):
        for k in KEYS:
            np.testing.assert_array_equal(got[k][5000 + i], got[k][j])


def test_draws_never_land_on_dead_gaussians_at_block_edges():
    """Dead Gaussians at the first slot of every 256-item scan block and at
    the end, uniforms at 0 and just below 1: every relocation and growth
    draw lands on a live Gaussian, the one the oracle draws."""
    p = _scene(4096, 8, 0.0)
    p["opacity_logit"] = np.maximum(p["opacity_logit"], -3.0)
    dead_idx = np.r_[np.arange(0, 4096, 256), 4095]
    p["opacity_logit"][dead_idx] = -9.0
    p = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}
    u = np.array([0.0, 0.5, 1.0 - 2.0 ** -53, 1.0 - 2.0 ** -40, 0.999999, 1e-300] + [0.25] * 11)
    dead = mcmc.sigmoid(p["opacity_logit"]) <= mcmc.DEAD_OPACITY
    assert dead.sum() == len(u)
    exp, src_e = mcmc.relocate(p, u)
    got, src, nd = _relocate(p, u)
    assert nd == len(u)
    assert not dead[src[dead]].any()
    np.testing.assert_array_equal(src[dead], src_e)
    gexp, gsrc_e = mcmc.grow(p, u)
    ggot, gsrc = _grow(p, 4096, u)
    assert not dead[gsrc].any()
    np.testing.assert_array_equal(gsrc, gsrc_e)


def test_reset_opacity_bounds_on_the_gpu():
    """A faint source drawn three times (o = 0.012: the unbounded o_N is
    0.004, below the dead threshold) and an opaque one (logit 40, o rounds
    to 1) drawn once: the reset opacities are 0.005 and 1 - 2^-23, finite
    logits, as the oracle's."""
    n = 8
    p = dict(mean=np.zeros((n, 3)), log_scale=np.full((n, 3), -2.0), quat=np.tile([1.0, 0, 0, 0], (n, 1)),
             opacity_logit=np.full(n, -9.0), sh=np.zeros((n, 16, 3)))
    p["opacity_logit"][0] = np.log(0.012 / 0.988)
    p = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}
    u = np.array([0.1, 0.5, 0.9, 0.2, 0.7, 0.3, 0.6])       # all 7 dead draw the only live one
    exp, src_e = mcmc.relocate(p, u[:3])
    got, src, _ = _relocate(p, u[:3])
    np.testing.assert_array_equal(src[1:4], [0, 0, 0])
    assert mcmc.sigmoid(got["opacity_logit"][0]) == pytest.approx(mcmc.DEAD_OPACITY, rel=1e-5)
    assert np.abs(got["opacity_logit"] - exp["opacity_logit"]).max() < 1e-4
    q = {k: v.copy() for k, v in p.items()}
    q["opacity_logit"][0] = 40.0
    exp, _ = mcmc.grow(q, u[:1])
    got, gsrc = _grow(q, n, u[:1])
    assert gsrc[0] == 0 and np.isfinite(got["opacity_logit"]).all()
    assert got["opacity_logit"][0] == pytest.approx(exp["opacity_logit"][0], rel=1e-5)


def test_moments_of_written_rows_restart_from_zero():
    from paper_2603_04847_gb300.core import gs_mcmc_reset_moments
    n_rows = 1000
    m = [torch.ones((n_rows, 3), device="cuda"), torch.ones((n_rows, 48), device="cuda")]
    v = [torch.ones_like(t) for t in m]
    src = torch.tensor([-1, 5, -1, 999, 5], dtype=torch.int32, device="cuda")
    gs_mcmc_reset_moments(n_rows, src, 990, list(zip(m, v)))
    torch.cuda.synchronize()
    zero = {991, 993, 994, 5, 999}
    for t in m + v:
        a = t.cpu().numpy()
        rows = {int(i) for i in np.nonzero((a == 0).all(1))[0]}
        assert rows == zero and (a[sorted(set(range(n_rows)) - zero)] == 1).all()
