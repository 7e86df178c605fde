"""Edge cases of the CUDA path: empty and fully culled scenes, ragged image
sizes, capacity overflow, non-finite parameters, argument errors, and the
CUDA-graph replay of the joint step against eager launches."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, gpu_backward, gpu_forward, knife_mask, oracle_cam, oracle_scene, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _cam_arrays(W, H, f=220.0):
    Rt = np.zeros((1, 12))
    Rt[0, [0, 4, 8]] = 1.0
    return np.array([[W, H]]), np.array([[f, f, W / 2, H / 2]]), Rt


def test_empty_scene_renders_background():
    wh, K, Rt = _cam_arrays(40, 30)
    sc = dict(mean=np.zeros((0, 3)), log_scale=np.zeros((0, 3)), quat=np.zeros((0, 4)),
              opacity_logit=np.zeros(0), sh=np.zeros((0, 1, 3)))
    r, *_ = gpu_forward(sc, wh, K, Rt, [0], bg=(0.1, 0.2, 0.3))
    img = r.image.cpu().numpy()
    bg32 = np.array([0.1, 0.2, 0.3], dtype=np.float32)
    np.testing.assert_array_equal(img, np.tile(bg32, (1200, 1)))
    assert (r.T_final.cpu().numpy() == 1.0).all() and (r.n_contrib.cpu().numpy() == 0).all()
    assert r.n_instances() == 0


def test_all_culled_scene():
    wh, K, Rt = _cam_arrays(48, 32)
    n = 50
    rng = np.random.default_rng(0)
    sc = dict(mean=np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(-5, -1, n)], 1),
              log_scale=np.full((n, 3), -2.0), quat=rng.normal(size=(n, 4)), opacity_logit=np.zeros(n),
              sh=np.zeros((n, 1, 3)))
    r, *_ = gpu_forward(sc, wh, K, Rt, [0])
    assert r.n_instances() == 0
    assert (r.image.cpu().numpy() == 0).all()


@pytest.mark.parametrize("W,H", [(250, 190), (17, 33), (1, 1), (16, 16)])
def test_ragged_sizes_match_oracle(W, H):
    w = synth.make_workload("tiny", n_gaussians=500)
    sc = w["scene"]
    wh, K, Rt = _cam_arrays(W, H)
    r, *_ = gpu_forward(sc, wh, K, Rt, [0])
    ref = oracle.render(oracle_scene(sc), oracle_cam(wh, K, Rt, 0), knife_eps=1e-4)
    img = r.image.cpu().numpy().reshape(H, W, 3)
    ok = ~knife_mask(ref)
    if ok.any() and np.abs(ref["image"][ok]).max() > 0:
        assert rel_linf(img[ok], ref["image"][ok]) <= 1e-4
    else:
        assert np.abs(img[ok]).max() <= 1e-6


def test_capacity_overflow_sets_flag_and_is_recoverable():
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, Renderer, _lib
    w = synth.make_workload("tiny", n_gaussians=800)
    g = Gaussians.from_numpy(w["scene"])
    cams = Cameras.from_numpy(w["wh"], w["K"], w["Rt"])
    r = Renderer(g.n, cams, Batch(cams, [0]), capacity=64)
    r.forward(g)
    torch.cuda.synchronize()
    assert int(r.status.item()) & _lib.GS_FLAG_CAPACITY
    need = r.n_instances()
    assert need > 64
    assert r.ensure_capacity(g)
    r.forward(g)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0 and r.tl.capacity >= need
    ref, *_ = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], [0])
    np.testing.assert_array_equal(r.image.cpu().numpy(), ref.image.cpu().numpy())


def test_nonfinite_gaussian_is_flagged_and_culled():
    from paper_2603_04847_gb300 import _lib
    w = synth.make_workload("tiny", n_gaussians=300)
    sc = {k: v.copy() for k, v in w["scene"].items()}
    sc["mean"][5, 0] = np.nan
    sc["sh"][9, 0, 1] = np.inf
    r, *_ = gpu_forward(sc, w["wh"], w["K"], w["Rt"], [0])
    assert int(r.status.item()) & _lib.GS_FLAG_NONFINITE
    nt = r.proj.n_tiles.cpu().numpy()
    assert nt[5] == 0 and nt[9] == 0
    keep = np.ones(300, bool)
    keep[[5, 9]] = False
    sc2 = {k: v[keep] for k, v in w["scene"].items()}
    r2, *_ = gpu_forward(sc2, w["wh"], w["K"], w["Rt"], [0])
    np.testing.assert_array_equal(r.image.cpu().numpy(), r2.image.cpu().numpy())


def test_argument_errors_are_reported():
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, GsError, Projected, gs_project
    from paper_2603_04847_gb300.core import new_status
    w = synth.make_workload("tiny", n_gaussians=10)
    g = Gaussians.from_numpy(w["scene"])
    cams = Cameras.from_numpy(w["wh"], w["K"], w["Rt"])
    b = Batch(cams, [0])
    b.tile = 8
    with pytest.raises(GsError, match="UNSUPPORTED"):
        gs_project(g, cams, b, Projected(g.n, 1), new_status())
    cams_bad = Cameras.from_numpy(w["wh"], w["K"], w["Rt"], near=-1.0)
    with pytest.raises(GsError, match="GS_ERR_ARG"):
        gs_project(g, cams_bad, Batch(cams, [0]), Projected(g.n, 1), new_status())
    g.quat = torch.empty(g.n * 4 + 1, device="cuda")[1:].view(g.n, 4)  # misaligned
    with pytest.raises(GsError, match="aligned"):
        gs_project(g, cams, Batch(cams, [0]), Projected(g.n, 1), new_status())


def _joint(mode, seed=0):
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
                   [4, 1, 3], Hyper(lambda_ba=0.1, lr_pose=1e-3, eps=1e-6), mode=mode)
    js.ensure_capacity()
    return js


def _state(js):
    return [t.detach().cpu().numpy().copy() for t in js.g.tensors() + [js.X, js.xi, js.Rt]]


def test_graph_replay_matches_eager_and_plain():
    eager = _joint("batched")
    for _ in range(3):
        eager.step()
    torch.cuda.synchronize()
    graphed = _joint("batched")
    graphed.capture(warmup=0)   # capturing does not run the step
    for _ in range(3):
        graphed.run()
    torch.cuda.synchronize()
    plain = _joint("plain")
    for _ in range(3):
        plain.step()
    torch.cuda.synchronize()
    a, b, c = _state(eager), _state(graphed), _state(plain)
    for x, y, z in zip(a, b, c):
        np.testing.assert_allclose(y, x, rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(z, x, rtol=1e-4, atol=1e-6)
    assert eager.status_flags() == 0
    assert int(eager.step_no.item()) == 3 and int(graphed.step_no.item()) == 3


def test_records_cleared_by_the_projection_backward():
    """The joint step leaves the backward's screen-space records zero
    behind its projection backward (gs_project_bwd_clearing), so it skips
    the clearing pass: three graph replays equal three steps that zero the
    records explicitly before each backward, and the records are zero
    after every step."""
    cleared = _joint("batched")
    cleared.capture(warmup=0)
    for _ in range(3):
        cleared.run()
        torch.cuda.synchronize()
        for r in cleared.renderers:
            assert not r.ws_bwd[:r.batch.B * r.n * 48].any()
    zeroed = _joint("batched")
    for _ in range(3):
        for r in zeroed.renderers:
            r.zero_records()
        zeroed.step()
    torch.cuda.synchronize()
    for x, y in zip(_state(cleared), _state(zeroed)):
        np.testing.assert_allclose(x, y, rtol=1e-4, atol=1e-6)
    assert cleared.status_flags() == 0


def test_project_bwd_clearing_equals_project_bwd():
    from paper_2603_04847_gb300 import Gaussians
    from paper_2603_04847_gb300.core import gs_project_bwd
    w = synth.make_workload("batched", n_gaussians=2000, n_views=3, width=(60, 90), height=(40, 70), n_tracks=10)
    r, g, cams, batch = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], [0, 1, 2])
    rng = np.random.default_rng(4)
    vimg = torch.as_tensor(rng.normal(size=(batch.pixels, 3)), dtype=torch.float32, device="cuda")
    from paper_2603_04847_gb300.core import gs_raster_bwd
    gs_raster_bwd(g, cams, batch, r.proj, r.tl, r.bg, r.image, r.T_final, r.n_contrib, vimg, None, 1.0, None,
                  r.ws_bwd)
    rec = r.ws_bwd[:batch.B * g.n * 48].clone()
    outs = []
    for clear in (False, True):
        r.ws_bwd[:batch.B * g.n * 48].copy_(rec)
        dg = Gaussians.zeros_like(g)
        tan = torch.zeros((cams.V, 6), dtype=torch.float64, device="cuda")
        gs_project_bwd(g, cams, batch, r.proj, dg, tan, r.ws_bwd, clear_records=clear)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in dg.tensors()] + [tan.cpu().numpy()])
        if clear:
            assert not r.ws_bwd[:batch.B * g.n * 48].any()
        else:
            assert torch.equal(r.ws_bwd[:batch.B * g.n * 48], rec)
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_target_stream_matches_device_resident_targets():
    """Streaming each step's targets from pinned host memory one step ahead
    (TargetStream: two alternating device copies filled on a copy stream)
    gives the same training trajectory as targets resident on the device,
    with the view batch changing every step."""
    from paper_2603_04847_gb300.step import TargetStream
    plan = [[4, 1, 3], [0, 2, 4], [1, 0, 2], [3, 4, 0]]
    ref = _joint("batched")
    for views in plan:
        ref.next_batch(views)
        ref.ensure_capacity()
        ref.step()
    torch.cuda.synchronize()
    js = _joint("batched")
    host = js.targets.cpu().pin_memory()
    ts = TargetStream(js, host, js.target_px_offset)
    ts.put(plan[0])
    for i, views in enumerate(plan):
        ts.begin()
        js.next_batch(views)
        js.ensure_capacity()
        js.step()
        ts.end()
        if i + 1 < len(plan):
            ts.put(plan[i + 1])
    torch.cuda.synchronize()
    for x, y in zip(_state(ref), _state(js)):
        np.testing.assert_allclose(y, x, rtol=1e-4, atol=1e-6)
    assert js.status_flags() == 0


def test_tile_sizes_give_identical_images_and_gradients():
    """16- and 32-pixel tiles composite the same splats in the same order at
    every pixel (a splat missing from a pixel's 16-tile list cannot reach
    it), so images and transmittance are bit-identical and gradients agree
    to rounding of the order of the per-tile atomic sums."""
    w = synth.make_workload("batched", n_gaussians=8000, n_views=3, width=(150, 260), height=(100, 190), n_tracks=10)
    outs = []
    for tile in (16, 32):
        r, g, *_ = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], [2, 0, 1], tile=tile)
        rng = np.random.default_rng(9)
        v = rng.normal(0, 1, (r.batch.n_pixels, 3))
        got = gpu_backward(r, g, v_image=v)
        outs.append((r.image.cpu().numpy(), r.T_final.cpu().numpy(), got))
    (i16, t16, g16), (i32, t32, g32) = outs
    np.testing.assert_array_equal(i32, i16)
    np.testing.assert_array_equal(t32, t16)
    for k in ("mean", "log_scale", "quat", "opacity_logit", "sh", "tangent"):
        np.testing.assert_allclose(g32[k], g16[k], rtol=1e-4, atol=1e-6 * np.abs(g16[k]).max())


def test_every_tuning_candidate_gives_the_same_image_and_lists():
    """The autotuner's candidates change only how work is split: images,
    per-pixel state and sorted lists are bit-identical under all of them."""
    from paper_2603_04847_gb300.autotune import CANDIDATES
    from paper_2603_04847_gb300.core import gs_get_tuning, gs_set_tuning
    w = synth.make_workload("batched", n_gaussians=6000, n_views=3, width=(150, 260), height=(100, 190), n_tracks=10)
    saved = gs_get_tuning()
    ref = None
    try:
        for rf, rb, sb in CANDIDATES:
            gs_set_tuning(rf, rb, sb)
            r, *_ = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], [0, 1, 2])
            n = r.n_instances()
            out = [r.image.cpu().numpy(), r.T_final.cpu().numpy(), r.n_contrib.cpu().numpy(),
                   r.tl.vals.cpu().numpy()[:n], r.tl.ranges.cpu().numpy()]
            if ref is None:
                ref = out
            else:
                for a, b in zip(out, ref):
                    np.testing.assert_array_equal(a, b)
    finally:
        gs_set_tuning(saved["render_fwd_batch"], saved["render_bwd_batch"], saved["sort_blocks_per_sm"])


def test_adam_groups_match_oracle():
    from paper_2603_04847_gb300.core import gs_adam_update_groups
    rng = np.random.default_rng(6)
    sizes = [1, 7, 4096, 4097, 20003, 3]
    lrs = [1e-3, 5e-3, 2e-2, 1e-4, 3e-3, 1.0]
    host = [[f32(rng.normal(size=n)) for _ in range(4)] for n in sizes]
    for h in host:
        h[3] = np.abs(h[3])
    dev = [[torch.tensor(a, dtype=torch.float32, device="cuda") for a in h] for h in host]
    # an unaligned view exercises the scalar path
    base = torch.zeros(20004 + 1, dtype=torch.float32, device="cuda")
    dev[4][0] = base[1:20004]
    dev[4][0].copy_(torch.tensor(host[4][0], device="cuda"))
    step = torch.tensor([4], dtype=torch.int32, device="cuda")
    gs_adam_update_groups([(d[0], d[1], d[2], d[3], lr) for d, lr in zip(dev, lrs)], 0.9, 0.999, 1e-15, step)
    torch.cuda.synchronize()
    for h, d, lr in zip(host, dev, lrs):
        p, g, m, v = (a.copy() for a in h)
        oracle.adam(p, g, m, v, lr, 0.9, 0.999, 1e-15, 4)
        np.testing.assert_allclose(d[0].cpu().numpy(), p, rtol=1e-5, atol=3e-7 * max(1.0, lr * 1e3))
        np.testing.assert_allclose(d[2].cpu().numpy(), m, rtol=1e-5, atol=3e-7)


def test_sort_wait_that_runs_out_flags_a_stall_and_ends():
    """The radix passes' bounded wait: with the test hook in which no
    predecessor block is ever seen to publish its digit counts
    (sort_spin_limit = -4), every wait of a multi-tile pass gives up after 4
    polls.  GS_FLAG_SORT_STALL is raised, the launches end (the stream
    synchronises), the sort stops -- no instances, every tile list empty,
    the image is the background -- and with the default bound back the same
    buffers render the scene again, identical to a fresh renderer."""
    from paper_2603_04847_gb300.core import gs_get_tuning, gs_set_tuning
    from paper_2603_04847_gb300._lib import GS_FLAG_SORT_STALL
    w = synth.make_workload("tiny", n_gaussians=20000)   # 20000 records: five 4096-item radix tiles
    wh, K, Rt = _cam_arrays(256, 192)
    r, g, *_ = gpu_forward(w["scene"], wh, K, Rt, [0])
    ref_img = r.image.cpu().numpy().copy()
    assert r.n_instances() > 0 and int(r.status.item()) == 0
    saved = gs_get_tuning()
    try:
        gs_set_tuning(saved["render_fwd_batch"], saved["render_bwd_batch"], saved["sort_blocks_per_sm"], -4)
        r.status.zero_()
        r.forward(g)
        torch.cuda.synchronize()
        assert int(r.status.item()) & GS_FLAG_SORT_STALL
        assert r.n_instances() == 0
        assert not r.tl.ranges.cpu().numpy().any()
        assert (r.image.cpu().numpy() == 0).all()
    finally:
        gs_set_tuning(saved["render_fwd_batch"], saved["render_bwd_batch"], saved["sort_blocks_per_sm"], 0)
    r.status.zero_()
    r.forward(g)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    np.testing.assert_array_equal(r.image.cpu().numpy(), ref_img)
