"""The path at the edges of its supported range, against the FP64 oracle.

- Depths spanning a factor of ~160 (float codes of the visible depths
  span more than 2^24, so the depth sort runs its fourth 8-bit pass):
  tile lists in (tile, depth, index) order, image and gradients.
- A batch of GS_MAX_BATCH (64) uneven views in one launch per stage, one
  view repeated: every view's image and the summed gradients.
- Tile ids of 17 and 18 bits (tile passes of 9 + 8 and 9 + 9 bits): the
  tile lists equal a lexicographic sort of the projection's own (tile,
  depth key, record) triples, and the ranges their counts."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, gpu_backward, gpu_forward, knife_mask, oracle_cam, oracle_scene, pose_rel_err, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KNIFE_EPS = 1e-4
GRAD_TOL = 1e-3
IMG_TOL = 1e-4
P = oracle.P


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _wide_depth_scene(n=1500, seed=21):
    """Gaussians in front of an identity camera (f = 220, 256x192) with
    log-uniform depths in [0.5, 80] and screen sizes of a few pixels at
    every depth."""
    rng = np.random.default_rng(seed)
    z = np.exp(rng.uniform(np.log(0.5), np.log(80.0), n))
    x = z * rng.uniform(-0.6, 0.6, n)
    y = z * rng.uniform(-0.45, 0.45, n)
    s = z[:, None] * 0.012 * np.exp(rng.uniform(-0.7, 0.7, (n, 3)))
    sh = np.zeros((n, 4, 3))
    sh[:, 0] = rng.uniform(-1.0, 1.0, (n, 3))
    sh[:, 1:] = rng.normal(0.0, 0.2, (n, 3, 3))
    return dict(mean=np.stack([x, y, z], 1), log_scale=np.log(s), quat=rng.normal(size=(n, 4)),
                opacity_logit=rng.normal(0.0, 1.5, n), sh=sh)


def _identity_cam(W=256, H=192, f=220.0):
    Rt = np.zeros((1, 12))
    Rt[0, [0, 4, 8]] = 1.0
    return np.array([[W, H]], dtype=np.int32), np.array([[f, f, W / 2, H / 2]]), Rt


def _knife(proj, eps=2e-4):
    """Records whose tile rectangle or visibility sits within rounding of a
    decision boundary (either answer is valid there)."""
    b = proj[:, [P["bound_x0"], P["bound_y0"], P["bound_x1"], P["bound_y1"]]]
    b = b + np.array([-1.0, -1.0, 1.0, 1.0]) * oracle.RECT_MARGIN
    return (np.abs(b - np.round(b)) < eps).any(1) | (np.abs(proj[:, P["opacity"]] - 1 / 255) < 1e-6)


@pytest.mark.parametrize("tile", [16, 32])
def test_depths_spanning_more_than_24_bits_of_float_codes(tile):
    sc = _wide_depth_scene()
    wh, K, Rt = _identity_cam()
    W, H = 256, 192
    cam = oracle_cam(wh, K, Rt, 0)
    osc = oracle_scene(sc)
    proj = oracle.project(osc, cam)
    vis = proj[:, P["visible"]] > 0
    codes = np.float32(proj[vis, P["depth"]]).view(np.uint32).astype(np.int64)
    assert codes.max() - codes.min() >= 1 << 24, "the scene must need the fourth depth pass"
    r, g, cams, batch = gpu_forward(sc, wh, K, Rt, [0], tile=tile)

    # tile lists: (tile, depth, index) order away from knife edges
    knife = _knife(proj)
    assert knife.sum() <= max(5, g.n // 100), knife.sum()
    t_o, d_o, g_o = oracle.tile_lists(proj, W, H, tile)
    keep = ~knife[g_o]
    n_inst = r.n_instances()
    vals = r.tl.vals.cpu().numpy()[:n_inst].astype(np.int64)
    ktile = r.tl.tiles.cpu().numpy()[:n_inst].astype(np.int64)
    kk = ~knife[vals]
    np.testing.assert_array_equal(ktile[kk], t_o[keep])
    kv, ov = vals[kk], g_o[keep]
    # FP32 depths within rounding of each other may come in either order
    for i in np.nonzero(kv != ov)[0]:
        d1, d2 = proj[kv[i], P["depth"]], proj[ov[i], P["depth"]]
        assert abs(d1 - d2) <= 1e-6 * d1, (i, kv[i], ov[i], d1, d2)

    # image and gradients of a random cotangent
    ref = oracle.render(osc, cam, knife_eps=KNIFE_EPS)
    ok = ~knife_mask(ref)
    img = r.image.cpu().numpy().reshape(H, W, 3)
    assert rel_linf(img[ok], ref["image"][ok]) <= IMG_TOL
    rng = np.random.default_rng(5)
    wv = f32(rng.normal(size=(H, W, 3)))
    wv[~ok] = 0.0
    got = gpu_backward(r, g, v_image=wv.reshape(-1, 3))
    exp = oracle.render_bwd(osc, cam, wv)
    for name in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        assert rel_linf(got[name], exp[name]) <= GRAD_TOL, name
    assert pose_rel_err(got["tangent"][0], exp["tangent"], exp["tangent_abs"]) <= GRAD_TOL


def test_a_batch_of_the_maximum_number_of_views():
    from paper_2603_04847_gb300 import _lib
    B = _lib.GS_MAX_BATCH
    w = synth.make_workload("batched", n_gaussians=2000, n_views=B - 1, width=(20, 48), height=(16, 40),
                            n_tracks=10, seed=17)
    sc, wh, K, Rt = w["scene"], w["wh"], w["K"], w["Rt"]
    views = list(range(B - 1))[::-1] + [5]   # every view, the last slot repeats view 5
    assert len(views) == B
    r, g, cams, batch = gpu_forward(sc, wh, K, Rt, views)
    osc = oracle_scene(sc)
    img = r.image.cpu().numpy()
    rng = np.random.default_rng(8)
    vfull = np.zeros_like(img, dtype=np.float64)
    exp = {k: 0.0 for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")}
    tan = np.zeros((len(wh), 6))
    tab = np.zeros((len(wh), 6))
    for b, v in enumerate(views):
        cam = oracle_cam(wh, K, Rt, v)
        ref = oracle.render(osc, cam, knife_eps=KNIFE_EPS)
        Wb, Hb = int(wh[v][0]), int(wh[v][1])
        a = int(batch.px_offset_host[b])
        ok = ~knife_mask(ref)
        ib = img[a:a + Wb * Hb].reshape(Hb, Wb, 3)
        if ok.any():
            assert rel_linf(ib[ok], ref["image"][ok]) <= IMG_TOL, (b, v)
        wv = f32(rng.normal(size=(Hb, Wb, 3)))
        wv[~ok] = 0.0
        vfull[a:a + Wb * Hb] = wv.reshape(-1, 3)
        e = oracle.render_bwd(osc, cam, wv)
        for k in exp:
            exp[k] = exp[k] + e[k]
        tan[v] += e["tangent"]
        tab[v] += e["tangent_abs"]
    got = gpu_backward(r, g, v_image=vfull)
    for k in exp:
        assert rel_linf(got[k], exp[k]) <= GRAD_TOL, k
    for v in range(len(wh)):
        assert pose_rel_err(got["tangent"][v], tan[v], tab[v]) <= GRAD_TOL, v


def _expected_lists(r, batch, N):
    """(tile, record) of every instance, sorted by (global tile, depth key,
    record), from the projection's rectangles and depth keys (numpy)."""
    rect = r.proj.rect.cpu().numpy()[:batch.B * N].astype(np.int64) & 0xFFFF
    ntl = r.proj.n_tiles.cpu().numpy()[:batch.B * N].astype(np.int64)
    key = r.proj.depth_key.cpu().numpy()[:batch.B * N].view(np.uint32).astype(np.int64)
    rec = np.nonzero(ntl > 0)[0]
    x0, y0, x1 = rect[rec, 0], rect[rec, 1], rect[rec, 2]
    w = x1 - x0 + 1
    cnt = ntl[rec]
    np.testing.assert_array_equal(cnt, w * (rect[rec, 3] - y0 + 1))
    rep = np.repeat(np.arange(len(rec)), cnt)
    local = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    b = rec[rep] // N
    tiles_x = (batch.W.astype(np.int64) + batch.tile - 1) // batch.tile
    tile = (batch.tile_offset_host[b] + (y0[rep] + local // w[rep]) * tiles_x[b]
            + x0[rep] + local % w[rep])
    order = np.lexsort((rec[rep], key[rec[rep]], tile))
    return tile[order], rec[rep][order]


@pytest.mark.parametrize("n_views,bits", [(9, 17), (17, 18)])
def test_tile_ids_of_17_and_18_bits(n_views, bits):
    w = synth.make_workload("batched", n_gaussians=30000, n_views=n_views, width=(1900, 1920),
                            height=(1060, 1080), n_tracks=10, seed=4)
    sc, wh, K, Rt = w["scene"], w["wh"], w["K"], w["Rt"]
    r, g, cams, batch = gpu_forward(sc, wh, K, Rt, list(range(n_views)))
    assert int(np.ceil(np.log2(batch.n_tiles))) == bits
    t_exp, v_exp = _expected_lists(r, batch, g.n)
    n_inst = r.n_instances()
    assert n_inst == len(t_exp) and n_inst > 20 * 4096
    np.testing.assert_array_equal(r.tl.tiles.cpu().numpy()[:n_inst].astype(np.int64), t_exp)
    np.testing.assert_array_equal(r.tl.vals.cpu().numpy()[:n_inst].astype(np.int64), v_exp)
    ranges = r.tl.ranges.cpu().numpy()[:2 * batch.n_tiles].reshape(-1, 2).astype(np.int64)
    counts = np.bincount(t_exp, minlength=batch.n_tiles)
    np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], counts)
    nz = counts > 0
    np.testing.assert_array_equal(ranges[nz, 0], (np.cumsum(counts) - counts)[nz])
