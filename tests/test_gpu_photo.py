"""Parity of gs_photo_loss (Eq. 5 with its SSIM term) with the FP64 oracle
on batches of views of uneven, ragged sizes, and the joint step that uses it
(eager, graph-captured and one-view-per-launch)."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(37, 29), (16, 16), (1, 1), (50, 23), (64, 48), (17, 33)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _views(sizes):
    wh = np.array(sizes, dtype=np.int64)
    V = len(sizes)
    K = np.array([[100.0, 100.0, w / 2.0, h / 2.0] for w, h in sizes])
    Rt = np.zeros((V, 12))
    Rt[:, [0, 4, 8]] = 1.0
    return wh, K, Rt


def _run(sizes, views, image, target, l1w, sw, tile):
    from paper_2603_04847_gb300 import Batch, Cameras
    from paper_2603_04847_gb300.core import gs_photo_loss, photo_loss_workspace_bytes
    wh, K, Rt = _views(sizes)
    cams = Cameras.from_numpy(wh, K, Rt)
    batch = Batch(cams, views, tile=tile)
    img = torch.as_tensor(image, dtype=torch.float32, device="cuda")
    tgt = torch.as_tensor(target, dtype=torch.float32, device="cuda")
    v = torch.full_like(img, np.nan)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(photo_loss_workspace_bytes(batch), dtype=torch.uint8, device="cuda")
    gs_photo_loss(cams, batch, img, tgt, l1w, sw, loss, v, ws)
    torch.cuda.synchronize()
    return float(loss.item()), v.cpu().numpy()


def _oracle(sizes, views, image, target, l1w, sw):
    loss, grads, o = 0.0, [], 0
    for vi in views:
        W, H = sizes[vi]
        n = W * H
        x = image[o:o + n].astype(np.float64).reshape(H, W, 3)
        y = target[o:o + n].astype(np.float64).reshape(H, W, 3)
        l, g = oracle.photo_loss_grad(x, y, l1w, sw)
        loss += l
        grads.append(g.reshape(n, 3))
        o += n
    return loss, np.concatenate(grads)


def _images(sizes, views, seed, smooth=False):
    rng = np.random.default_rng(seed)
    P = sum(sizes[v][0] * sizes[v][1] for v in views)
    if not smooth:
        return (rng.uniform(0, 1, (P, 3)).astype(np.float32), rng.uniform(0, 1, (P, 3)).astype(np.float32))
    # slowly varying images with small local variance (the FP32 local
    # variance E[x^2] - E[x]^2 then cancels most of its digits)
    t = np.linspace(0.2, 0.8, P)[:, None]
    return ((t + rng.normal(0, 0.02, (P, 3))).astype(np.float32),
            (t + 0.05 + rng.normal(0, 0.02, (P, 3))).astype(np.float32))


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("l1w,sw", [(0.8, 0.2), (0.0, 1.0), (1.0, 0.0)])
def test_photo_loss_matches_oracle_on_uneven_views(tile, l1w, sw):
    views = [0, 1, 2, 3, 4, 5, 3]
    x, y = _images(SIZES, views, 0)
    loss, v = _run(SIZES, views, x, y, l1w, sw, tile)
    ref_loss, ref_v = _oracle(SIZES, views, x, y, l1w, sw)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    assert np.isfinite(v).all()
    assert rel_linf(v, ref_v) <= 1e-4


def test_photo_loss_smooth_images():
    """Small local variance (4e-4 against means of 0.2-0.8): the FP32
    variance E[x^2] - E[x]^2 loses ~3 digits, which leaves each pixel's SSIM
    with an error of ~1e-4 of (vx + vy + C2); the bars here are 1e-4 on the
    loss and 1e-3 on the gradient (the loss's error was 2.4e-5 on a GB300)."""
    views = [4, 0]
    x, y = _images(SIZES, views, 1, smooth=True)
    loss, v = _run(SIZES, views, x, y, 0.8, 0.2, 16)
    ref_loss, ref_v = _oracle(SIZES, views, x, y, 0.8, 0.2)
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    assert rel_linf(v, ref_v) <= 1e-3


def test_photo_loss_identical_images_have_zero_loss_and_gradient():
    views = [0, 3]
    x, _ = _images(SIZES, views, 2)
    loss, v = _run(SIZES, views, x, x.copy(), 0.8, 0.2, 16)
    assert abs(loss) < 1e-6
    assert np.abs(v).max() < 1e-7


def test_photo_loss_argument_errors():
    from paper_2603_04847_gb300 import Batch, Cameras, GsError
    from paper_2603_04847_gb300.core import gs_photo_loss, photo_loss_workspace_bytes
    wh, K, Rt = _views(SIZES[:2])
    cams = Cameras.from_numpy(wh, K, Rt)
    batch = Batch(cams, [0, 1], tile=16)
    P = batch.n_pixels
    img = torch.zeros((P, 3), dtype=torch.float32, device="cuda")
    ws = torch.empty(photo_loss_workspace_bytes(batch), dtype=torch.uint8, device="cuda")
    with pytest.raises(GsError):
        gs_photo_loss(cams, batch, img, img, 0.8, -0.2, None, img.clone(), ws)
    with pytest.raises(GsError):
        gs_photo_loss(cams, batch, img, img, 0.8, 0.2, None, img.clone(), ws[:16])


def _joint(mode, lam=0.2, seed=0):
    from paper_2603_04847_gb300 import Cameras, Gaussians, Hyper, JointStep
    w = synth.make_workload("batched", n_gaussians=3000, n_views=5, width=(80, 160), height=(64, 120),
                            n_tracks=200, seed=seed)
    wh, K, Rt = w["wh"], w["K"], w["Rt"]
    cams = Cameras.from_numpy(wh, K, Rt)
    g = Gaussians.from_numpy(w["scene"])
    tr = w["tracks"]
    rng = np.random.default_rng(1)
    xy = rng.uniform(10, 60, (len(tr["obs_point"]), 2))
    P = (wh[:, 0] * wh[:, 1]).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(P)])
    targets = torch.as_tensor(rng.uniform(0, 1, (int(off[-1]), 3)), dtype=torch.float32, device="cuda")
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    js = JointStep(g, cams, dev(tr["X"], torch.float32), dev(tr["obs_point"], torch.int32),
                   dev(xy, torch.float32), dev(tr["view_obs_offset"], torch.int64), targets, off,
                   [4, 1, 3], Hyper(lambda_ba=0.1, lr_pose=1e-3, eps=1e-6, lambda_ssim=lam), mode=mode)
    js.ensure_capacity()
    return js, wh


def test_joint_step_photometric_term_with_ssim():
    """One step with lambda_SSIM = 0.2: its photometric loss and the dL/dimage
    it feeds to the compositing backward equal the oracle's Eq. 5 of the
    step's own rendered images."""
    js, wh = _joint("batched")
    js.step()
    torch.cuda.synchronize()
    r = js.renderers[0]
    img = r.image.cpu().numpy()
    tgt = js.target_batch.cpu().numpy()
    sizes = [tuple(int(a) for a in s) for s in wh]
    ref_loss, ref_v = _oracle(sizes, [4, 1, 3], img, tgt, 0.8, 0.2)
    assert abs(float(js.loss[0].item()) - ref_loss) <= 1e-5 * ref_loss
    assert rel_linf(r.v_image.cpu().numpy(), ref_v) <= 1e-4
    assert js.status_flags() == 0


def test_joint_step_with_ssim_graph_and_plain_match_eager():
    def state(js):
        return [t.detach().cpu().numpy().copy() for t in js.g.tensors() + [js.X, js.xi, js.Rt]]

    eager, _ = _joint("batched")
    for _ in range(2):
        eager.step()
    graphed, _ = _joint("batched")
    graphed.capture(warmup=0)
    for _ in range(2):
        graphed.run()
    plain, _ = _joint("plain")
    for _ in range(2):
        plain.step()
    torch.cuda.synchronize()
    for x, y, z in zip(state(eager), state(graphed), state(plain)):
        np.testing.assert_allclose(y, x, rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(z, x, rtol=1e-4, atol=1e-6)
