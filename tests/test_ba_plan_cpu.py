"""The host-side plan of the bundle adjustment's elimination by camera pairs
(sfm_ba_pair_lists, host code in libgs, no GPU needed) against a direct
enumeration: every ordered pair (a, b) of one point's observations with
cam(b) <= cam(a), grouped by camera pair in order, within a pair in order
of the point and of a's and b's list positions; chunks of at most `chunk`
incidences per pair.  Entries of out-of-range observations or cameras are
left out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def plan_fn():
    from paper_2603_04847_gb300 import build
    build.build()
    from paper_2603_04847_gb300.core import sfm_ba_pair_lists
    return sfm_ba_pair_lists


def _enumerate(V, P, oc, off, ids, chunk):
    by_pair = {}
    for k in range(P):
        lst = [int(o) for o in ids[off[k]:off[k + 1]] if 0 <= o < len(oc) and 0 <= oc[o] < V]
        for a in lst:
            for b in lst:
                if oc[b] <= oc[a]:
                    by_pair.setdefault((int(oc[a]), int(oc[b])), []).append((k, a, b))
    inc, cams, pchunks, cstart = [], [], [0], []
    for key in sorted(by_pair):
        lst = by_pair[key]
        cams.append(key)
        for c in range(0, len(lst), chunk):
            cstart.append(len(inc) + c)
        inc += lst
        pchunks.append(len(cstart))
    cstart.append(len(inc))
    return (np.array(inc, np.int32).reshape(-1, 3), np.array(cams, np.int32).reshape(-1, 2),
            np.array(pchunks, np.int32), np.array(cstart, np.int64))


@pytest.mark.parametrize("chunk", [1, 3, 128])
def test_plan_equals_a_direct_enumeration(plan_fn, chunk):
    rng = np.random.default_rng(chunk)
    V, P, M = 7, 40, 260
    op = rng.integers(0, P + 3, M).astype(np.int32)       # some points out of range
    oc = rng.integers(0, V, M).astype(np.int32)
    oc[rng.random(M) < 0.03] = V + 1                      # some cameras out of range
    ok = op < P
    ids = np.nonzero(ok)[0]
    ids = ids[np.argsort(op[ids], kind="stable")].astype(np.int32)
    ids = np.concatenate([ids, [M + 5]]).astype(np.int32)  # an entry past the observations
    cnt = np.bincount(op[ok], minlength=P)
    cnt[P - 1] += 1
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    got = plan_fn(V, P, oc, off, ids, chunk=chunk)
    inc, cams, pchunks, cstart = _enumerate(V, P, oc, off, ids, chunk)
    np.testing.assert_array_equal(got["inc"], inc)
    np.testing.assert_array_equal(got["pair_cams"], cams)
    np.testing.assert_array_equal(got["pair_chunks"], pchunks)
    np.testing.assert_array_equal(got["chunk_start"], cstart)


def test_empty_problem(plan_fn):
    got = plan_fn(3, 2, np.zeros(0, np.int32), np.zeros(3, np.int64), np.zeros(0, np.int32))
    assert got["inc"].shape == (0, 3) and got["pair_cams"].shape == (0, 2)
    np.testing.assert_array_equal(got["pair_chunks"], [0])
    np.testing.assert_array_equal(got["chunk_start"], [0])


def test_bad_arguments_are_reported(plan_fn):
    from paper_2603_04847_gb300._lib import GsError
    with pytest.raises(GsError):
        plan_fn(3, 1, np.zeros(2, np.int32), np.array([0, 2], np.int64), np.array([0, 1], np.int32), chunk=0)
    with pytest.raises(GsError):
        plan_fn(-1, 1, np.zeros(2, np.int32), np.array([0, 2], np.int64), np.array([0, 1], np.int32))
