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
