"""The allocation-free track term (track_reproj_fwd_bwd_static), for callers
that cannot allocate device memory when they run it, must give what the
workspace entry point (track_reproj_fwd_bwd) gives.  Checked through the C
ABI on two calls in a row with different batches, so the second call runs on
the library's scratch array as the first left it.  Collected last on
purpose: a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build, _lib
    build.build()
    return _lib.load()


def _problem(seed, views):
    rng = np.random.default_rng(seed)
    V = 6
    wh, K, Rt = synth.cameras_sphere(rng, V, (320, 480), (240, 360))
    n_points = 3000
    X = rng.uniform(-1, 1, (n_points, 3))
    obs_point = np.repeat(np.arange(n_points), 3)
    obs_view = np.concatenate([rng.choice(V, 3, replace=False) for _ in range(n_points)])
    order = np.argsort(obs_view, kind="stable")
    obs_point, obs_view = obs_point[order], obs_view[order]
    xy = rng.uniform(0, 1, (len(obs_point), 2)) * wh[obs_view]
    off = np.zeros(V + 1, dtype=np.int64)
    np.add.at(off, obs_view + 1, 1)
    off = np.cumsum(off)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    from paper_2603_04847_gb300 import Batch, Cameras
    cams = Cameras.from_numpy(wh, K, Rt)
    return dict(cams=cams, batch=Batch(cams, views), X=dev(X, torch.float32), op=dev(obs_point, torch.int32),
                xy=dev(xy, torch.float32), off=dev(off, torch.int64), V=V)


def _run(lib, p, static):
    from paper_2603_04847_gb300 import _lib
    from paper_2603_04847_gb300.core import track_workspace_bytes
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    gX = torch.zeros_like(p["X"])
    gt = torch.zeros((p["V"], 6), dtype=torch.float64, device="cuda")
    nm = torch.zeros(1, dtype=torch.int32, device="cuda")
    cc, bc = p["cams"].c(), p["batch"].c()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    common = (ptr(p["X"]), p["X"].shape[0], ptr(p["op"]), ptr(p["xy"]), ptr(p["off"]), ctypes.byref(cc),
              ctypes.byref(bc), 1.0, 0.1, ptr(loss), ptr(gX), ptr(gt), ptr(nm))
    if static:
        rc = lib.track_reproj_fwd_bwd_static(*common, stream)
    else:
        ws = torch.empty(track_workspace_bytes(p["batch"]), dtype=torch.uint8, device="cuda")
        rc = lib.track_reproj_fwd_bwd(*common, ptr(ws), ws.numel(), stream)
    assert rc == _lib.GS_OK, lib.gs_last_error()
    torch.cuda.synchronize()
    return loss.item(), gX.cpu().numpy(), gt.cpu().numpy(), int(nm.item())


def _rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def test_static_scratch_matches_workspace_entry_point(lib):
    for seed, views in [(0, [0, 3, 5]), (1, [5, 1, 2, 4, 0])]:
        p = _problem(seed, views)
        ref = _run(lib, p, static=False)
        got = _run(lib, p, static=True)
        assert got[0] == pytest.approx(ref[0], rel=1e-5)
        assert _rel(got[1], ref[1]) <= GRAD_TOL
        for v in views:
            for part in (slice(0, 3), slice(3, 6)):
                assert _rel(got[2][v, part], ref[2][v, part]) <= GRAD_TOL
        assert not got[2][[v for v in range(p["V"]) if v not in views]].any()
        assert got[3] == ref[3]
