"""Batches laid out on the device (gs_batch_layout): buffers sized for any
views of the scene, offsets recomputed from the device copy of the view ids,
so one captured step serves batches of uneven views (Algorithm 1, "Sample
image indices", with views of different resolutions)."""
import numpy as np
import pytest

import synth
from _gpu import gpu_backward

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _scene(n=4000, views=6, seed=0):
    return synth.make_workload("batched", n_gaussians=n, n_views=views, width=(60, 170), height=(40, 130),
                               n_tracks=50, seed=seed)


def _render(w, batch, cams, g, r=None):
    from paper_2603_04847_gb300 import Renderer
    if r is None:
        r = Renderer(g.n, cams, batch)
    r.ensure_capacity(g)
    r.forward(g)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("tile", [16, 32])
def test_device_layout_matches_a_host_laid_out_batch(tile):
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians
    w = _scene()
    cams = Cameras.from_numpy(w["wh"], w["K"], w["Rt"])
    g = Gaussians.from_numpy(w["scene"])
    dyn = Batch(cams, [0, 1, 2], tile=tile, capacity=Batch.capacity_for(cams, 3, tile))
    r = None
    rng = np.random.default_rng(3)
    for views in ([5, 0, 3], [1, 4, 2], [3, 3, 5], [0, 1, 2]):
        dyn.set_views(cams, views)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dyn.px_offset.cpu().numpy(), dyn.px_offset_host)
        np.testing.assert_array_equal(dyn.tile_offset.cpu().numpy(), dyn.tile_offset_host)
        r = _render(w, dyn, cams, g, r)
        ref = _render(w, Batch(cams, views, tile=tile), cams, g)
        P = dyn.pixels
        assert P == ref.batch.n_pixels and P <= dyn.n_pixels
        np.testing.assert_array_equal(r.image[:P].cpu().numpy(), ref.image.cpu().numpy())
        np.testing.assert_array_equal(r.T_final[:P].cpu().numpy(), ref.T_final.cpu().numpy())
        np.testing.assert_array_equal(r.n_contrib[:P].cpu().numpy(), ref.n_contrib.cpu().numpy())
        n = ref.n_instances()
        assert r.n_instances() == n
        np.testing.assert_array_equal(r.tl.vals[:n].cpu().numpy(), ref.tl.vals[:n].cpu().numpy())
        nt = ref.batch.n_tiles
        np.testing.assert_array_equal(r.tl.ranges[:2 * nt].cpu().numpy(), ref.tl.ranges.cpu().numpy())
        assert not r.tl.ranges[2 * nt:].cpu().numpy().any()
        v = rng.normal(0, 1, (P, 3))
        vd = np.zeros((dyn.n_pixels, 3))
        vd[:P] = v
        got, exp = gpu_backward(r, g, v_image=vd), gpu_backward(ref, g, v_image=v)
        for k in ("mean", "log_scale", "quat", "opacity_logit", "sh", "tangent"):
            np.testing.assert_allclose(got[k], exp[k], rtol=1e-4, atol=1e-6 * max(np.abs(exp[k]).max(), 1e-30))
        assert int(r.status.item()) == 0


def test_layout_past_capacity_empties_the_remaining_slots():
    """Views whose pixels exceed the batch's capacity, swapped in on the
    device behind the host's back: the first slot that does not fit and all
    after it get no pixels and no tiles, GS_FLAG_CAPACITY is raised, and the
    slots that fit render as a batch of just those views."""
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, Renderer
    from paper_2603_04847_gb300._lib import GS_FLAG_CAPACITY
    w = _scene()
    # three 64x48 views and a 200x150 one that does not fit beside them
    w["wh"][:3] = (64, 48)
    w["wh"][3] = (200, 150)
    w["K"][:, 2:] = w["wh"] / 2.0
    w["K"][:, :2] = 0.9 * w["wh"][:, :1]
    cams = Cameras.from_numpy(w["wh"], w["K"], w["Rt"])
    g = Gaussians.from_numpy(w["scene"])
    P = (w["wh"][:, 0] * w["wh"][:, 1]).astype(np.int64)
    small, big = [0, 1, 2], 3
    dyn = Batch(cams, small, capacity=Batch.capacity_for(cams, 3, views=small))
    assert P[0] + P[big] > dyn.n_pixels
    r = Renderer(g.n, cams, dyn)
    views = [small[0], big, small[1]]
    dyn.views.copy_(torch.tensor(views, dtype=torch.int32))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dyn.layout(cams, status)
    torch.cuda.synchronize()
    assert int(status.item()) & GS_FLAG_CAPACITY
    px = dyn.px_offset.cpu().numpy()
    to = dyn.tile_offset.cpu().numpy()
    assert px[1] == P[small[0]] and px[2] == px[1] and px[3] == px[1]
    assert to[2] == to[1] and to[3] == to[1]
    r.ensure_capacity(g)
    r.forward(g)
    torch.cuda.synchronize()
    ref = _render(w, Batch(cams, [small[0]]), cams, g)
    n = int(P[small[0]])
    np.testing.assert_array_equal(r.image[:n].cpu().numpy(), ref.image.cpu().numpy())
    assert r.n_instances() == ref.n_instances()
    assert int(r.status.item()) == GS_FLAG_CAPACITY   # the forward's own layout flags it again


def _joint(dynamic, views, mode="batched"):
    from paper_2603_04847_gb300 import Cameras, Gaussians, Hyper, JointStep
    w = _scene(n=3000, views=7, seed=2)
    wh, K, Rt = w["wh"], w["K"], w["Rt"]
    cams = Cameras.from_numpy(wh, K, Rt)
    g = Gaussians.from_numpy(w["scene"])
    tr = w["tracks"]
    rng = np.random.default_rng(1)
    xy = rng.uniform(10, 60, (len(tr["obs_point"]), 2))
    off = np.concatenate([[0], np.cumsum((wh[:, 0] * wh[:, 1]).astype(np.int64))])
    targets = torch.as_tensor(rng.uniform(0, 1, (int(off[-1]), 3)), dtype=torch.float32, device="cuda")
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    js = JointStep(g, cams, dev(tr["X"], torch.float32), dev(tr["obs_point"], torch.int32),
                   dev(xy, torch.float32), dev(tr["view_obs_offset"], torch.int64), targets, off,
                   views, Hyper(lambda_ba=0.1, lr_pose=1e-3, eps=1e-6), mode=mode, dynamic_batch=dynamic)
    return js


def _state(js):
    return [t.detach().cpu().numpy().copy() for t in js.g.tensors() + [js.X, js.xi, js.Rt]]


PLAN = [[4, 1, 3], [0, 6, 2], [5, 5, 1], [2, 3, 0]]


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_one_captured_step_over_batches_of_uneven_views(mode):
    """A step captured once and replayed with only the device copy of the
    view ids changed (views of other sizes each time) follows the same
    trajectory as eager steps on batches laid out on the host."""
    ref = _joint(False, PLAN[0], mode)
    for views in PLAN:
        ref.next_batch(views)
        ref.ensure_capacity()
        ref.step()
    torch.cuda.synchronize()
    js = _joint(True, PLAN[0], mode)
    for views in PLAN:                   # size the instance lists for every batch
        js.next_batch(views)
        js.ensure_capacity()
    js.next_batch(PLAN[0])
    js.capture(warmup=0)
    pinned = torch.zeros(3, dtype=torch.int32).pin_memory()
    for views in PLAN:
        pinned.copy_(torch.tensor(views, dtype=torch.int32))
        js.batch.views.copy_(pinned, non_blocking=True)
        if mode != "batched":
            for b, sb in enumerate(js.slot_batches):
                sb.views.copy_(pinned[b:b + 1], non_blocking=True)
        js.run()
        torch.cuda.synchronize()
    for x, y in zip(_state(ref), _state(js)):
        np.testing.assert_allclose(y, x, rtol=1e-4, atol=1e-6)
    assert js.status_flags() == 0 and ref.status_flags() == 0
