"""The deterministic compositing backward (gs_raster_bwd_det,
Renderer(deterministic=True)): every (record, tile) instance writes its
sums into a slot of its own and the per-record sums are formed in a fixed
order, so its results do not depend on the order in which tiles run.

- Two runs give bit-identical gradients of every Gaussian parameter, the
  pose tangent and the fused L1 loss, on the thin-streak scene (where the
  atomic backward's run-to-run spread is largest), for both tile sizes and
  with both an explicit dL/dimage and the fused L1.
- Against the oracle it meets the parity bars of the default backward.
- At the 8-view 1237x822, 200k-Gaussian size it is bit-identical across
  runs and equals the atomic backward to FP32 summation rounding.
- When the tile lists do not hold every instance (capacity overflow) the
  gradients are zero and the overflow is flagged, like the atomic path's
  empty-gradient behaviour for missing instances.
- The deterministic track term (track_reproj_fwd_bwd_det, a launch per
  slot) is bit-identical across runs and equals the default term to FP32
  summation rounding.  The whole deterministic joint step is checked in
  test_gpu_joint_step.py."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, gpu_backward, gpu_forward, knife_mask, oracle_cam, oracle_scene, pose_rel_err, rel_linf
from test_gpu_parity import GRAD_TOL, thin_splats, tiny

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _run(sc, wh, K, Rt, views, tile, fused, deterministic=True, seed=11):
    r, g, cams, batch = gpu_forward(sc, wh, K, Rt, views, tile=tile, deterministic=deterministic)
    rng = np.random.default_rng(seed)
    if fused:
        tgt = f32(rng.uniform(0, 1, size=(batch.n_pixels, 3)))
        out = gpu_backward(r, g, target=tgt, l1_weight=0.7)
    else:
        out = gpu_backward(r, g, v_image=f32(rng.normal(size=(batch.n_pixels, 3))))
    return r, batch, out


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("tile", [16, 32])
def test_two_runs_are_bit_identical(tile, fused):
    w, sc, wh, K, Rt = thin_splats()
    a = _run(sc, wh, K, Rt, [0], tile, fused)[2]
    b = _run(sc, wh, K, Rt, [0], tile, fused)[2]
    for k in KEYS + ("tangent",):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["loss"] == b["loss"]
    assert np.abs(a["mean"]).max() > 0


def test_matches_the_oracle():
    w, sc, wh, K, Rt = tiny()
    r, batch, _ = _run(sc, wh, K, Rt, [0], 16, False)
    cam = oracle_cam(wh, K, Rt, 0)
    osc = oracle_scene(sc)
    ref = oracle.render(osc, cam, knife_eps=1e-4)
    ok = ~knife_mask(ref)
    rng = np.random.default_rng(4)
    wv = f32(rng.normal(size=(192, 256, 3)))
    wv[~ok] = 0.0
    from paper_2603_04847_gb300 import Gaussians
    g = Gaussians.from_numpy(sc)
    got = gpu_backward(r, g, v_image=wv.reshape(-1, 3))
    exp = oracle.render_bwd(osc, cam, wv)
    for k in KEYS:
        assert rel_linf(got[k], exp[k]) <= GRAD_TOL, (k, rel_linf(got[k], exp[k]))
    assert pose_rel_err(got["tangent"][0], exp["tangent"], exp["tangent_abs"]) <= GRAD_TOL


def test_full_size_bit_identical_and_equal_to_the_atomic_backward():
    w = synth.make_workload("mid")
    views = list(range(8))
    det0 = _run(w["scene"], w["wh"], w["K"], w["Rt"], views, 16, True)
    assert det0[0].n_instances() > 1_000_000
    det1 = _run(w["scene"], w["wh"], w["K"], w["Rt"], views, 16, True)[2]
    atom = _run(w["scene"], w["wh"], w["K"], w["Rt"], views, 16, True, deterministic=False)[2]
    d0 = det0[2]
    for k in KEYS + ("tangent",):
        np.testing.assert_array_equal(d0[k], det1[k], err_msg=k)
        assert rel_linf(d0[k], atom[k]) <= 1e-4, (k, rel_linf(d0[k], atom[k]))
    assert d0["loss"] == det1["loss"]
    assert d0["loss"] == pytest.approx(atom["loss"], rel=1e-12)


def test_overflow_gives_zero_gradients_and_a_flag():
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, Renderer, _lib
    w = synth.make_workload("tiny", n_gaussians=800)
    g = Gaussians.from_numpy(w["scene"])
    cams = Cameras.from_numpy(w["wh"], w["K"], w["Rt"])
    r = Renderer(g.n, cams, Batch(cams, [0]), capacity=64, deterministic=True)
    r.forward(g)
    torch.cuda.synchronize()
    assert int(r.status.item()) & _lib.GS_FLAG_CAPACITY
    assert r.n_instances() > 64
    out = gpu_backward(r, g, v_image=f32(np.ones((r.batch.n_pixels, 3))))
    for k in KEYS + ("tangent",):
        assert not np.any(out[k]), k
    # grown, it renders and differentiates like a fresh renderer
    assert r.ensure_capacity(g)
    r.forward(g)
    a = gpu_backward(r, g, v_image=f32(np.ones((r.batch.n_pixels, 3))))
    ref, g2, *_ = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], [0], deterministic=True)
    b = gpu_backward(ref, g2, v_image=f32(np.ones((ref.batch.n_pixels, 3))))
    for k in KEYS + ("tangent",):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_track_term_bit_identical_and_equal_to_the_atomic_term():
    from paper_2603_04847_gb300 import Batch, Cameras
    from paper_2603_04847_gb300.core import track_reproj_fwd_bwd, track_workspace_bytes
    w = synth.make_workload("mid", n_tracks=20000)
    tr = w["tracks"]
    cams = Cameras.from_numpy(w["wh"], w["K"], w["Rt"])
    batch = Batch(cams, [3, 0, 5, 7, 1, 3])          # a repeated view too
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    rng = np.random.default_rng(0)
    X = dev(tr["X"] + rng.normal(0, 0.01, tr["X"].shape), torch.float32)
    op = dev(tr["obs_point"], torch.int32)
    xy = dev(rng.uniform(0, 800, (len(tr["obs_point"]), 2)), torch.float32)
    voff = dev(tr["view_obs_offset"], torch.int64)
    ws = torch.empty(track_workspace_bytes(batch), dtype=torch.uint8, device="cuda")
    res = []
    for det in (True, True, False):
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        gX = torch.zeros_like(X)
        gt = torch.zeros((cams.V, 6), dtype=torch.float64, device="cuda")
        nm = torch.zeros(1, dtype=torch.int32, device="cuda")
        track_reproj_fwd_bwd(X, op, xy, voff, cams, batch, 1.0, 0.5, loss, gX, gt, nm, ws, deterministic=det)
        torch.cuda.synchronize()
        res.append((loss.item(), gX.cpu().numpy(), gt.cpu().numpy(), int(nm.item())))
    (l0, g0, t0, m0), (l1, g1, t1, m1), (la, ga, ta, ma) = res
    assert l0 == l1 and m0 == m1 == ma
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(t0, t1)
    # the default term runs all slots in one launch, so its per-thread
    # float sums group the observations differently
    assert abs(l0 - la) <= 1e-6 * abs(la)
    assert rel_linf(g0, ga) <= 1e-6
    assert rel_linf(t0, ta) <= 1e-5
    assert np.abs(g0).max() > 0 and np.abs(t0).max() > 0
