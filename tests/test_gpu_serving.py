"""The serving runtime (svt_server): requests admitted while others run on the
device give, each one, the same tracks as the request run alone through a
context, and the oracle's tracks."""
import numpy as np
import pytest

from paper_1312_0917_gb300 import binding as B, synth
from gpu_util import assert_same_tracks, run_gpu

pytestmark = pytest.mark.gpu


def requests(seed, n, max_events=256):
    sizes = synth.request_sizes(seed, n, max_events)
    return [synth.make_batch("scaled", seed=1000 * seed + i, n_events=int(k)).words
            for i, k in enumerate(sizes)]


def serve_all(srv, reqs):
    """Submit every request (blocking only while all slots are busy) and
    collect the results; -> {request index: (result, tracks)}."""
    ids = {}
    out = {}
    for i, w in enumerate(reqs):
        ids[srv.submit(w)] = i
        while True:   # collect what has completed meanwhile
            r = srv.wait(0)
            if r is None:
                break
            out[ids[r["request_id"]]] = (r, srv.take(r["request_id"], r["n_tracks"]))
    while len(out) < len(reqs):
        r = srv.wait(10_000_000)
        assert r is not None, "a request did not complete"
        out[ids[r["request_id"]]] = (r, srv.take(r["request_id"], r["n_tracks"]))
    return out


@pytest.fixture(scope="module")
def alone_ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = B.Context(0, max_words=1 << 21, max_events=4096, max_roads=1 << 17)
    yield c
    c.close()


@pytest.mark.parametrize("mode", [B.PERSISTENT, B.PLAIN], ids=["persistent", "plain"])
def test_results_in_the_mix_equal_alone_and_oracle(alone_ctx, orc, consts, cuts, mode):
    reqs = requests(1 if mode == B.PERSISTENT else 2, 24)
    srv = B.Server(consts, cuts["scaled"], mode=mode, n_slots=4)
    try:
        assert srv.config()["n_slots"] == 4
        got = serve_all(srv, reqs)
    finally:
        srv.close()
    alone_ctx.load_constants(consts, cuts["scaled"])
    for i, w in enumerate(reqs):
        r, tracks = got[i]
        assert r["status"] == B.OK
        st, alone, stats = run_gpu(alone_ctx, w, B.PERSISTENT)
        assert st == B.OK
        assert tracks.tobytes() == alone.tobytes(), "request %d differs from its run alone" % i
        assert r["n_events"] == stats["n_events"] and r["n_combinations"] == stats["n_combinations"]
        rc, want = orc.run(w, consts, cuts["scaled"])
        assert rc == 0
        assert_same_tracks(tracks, want)
        assert r["latency_ns"] > 0


def test_a_bad_request_does_not_disturb_the_others(orc, consts, cuts):
    reqs = requests(3, 8, 64)
    bad = reqs[3].copy()
    bad[5] |= np.uint32(1 << 20)            # a reserved payload bit: SVT_E_BADWORD
    reqs[3] = bad
    srv = B.Server(consts, cuts["scaled"], n_slots=2)
    try:
        got = serve_all(srv, reqs)
        assert srv.submit(np.zeros(0, np.uint32)) > 0   # an empty request is valid
        r = srv.wait(10_000_000)
        assert r["status"] == B.OK and r["n_tracks"] == 0
    finally:
        srv.close()
    rc, _, _, pos = orc.unpack(bad)
    assert got[3][0]["status"] == rc == B.E_BADWORD
    for i, w in enumerate(reqs):
        if i != 3:
            rc, want = orc.run(w, consts, cuts["scaled"])
            assert got[i][0]["status"] == B.OK
            assert_same_tracks(got[i][1], want)


def test_admission_limits(consts, cuts):
    srv = B.Server(consts, cuts["scaled"], n_slots=1, max_words=4096)
    try:
        with pytest.raises(B.SvtError) as e:
            srv.submit(np.zeros(5000, np.uint32))
        assert e.value.code == B.E_CAPACITY
        w = synth.make_batch("scaled", seed=5, n_events=3).words
        rid = srv.submit(w)
        r = srv.wait(10_000_000)
        assert r["request_id"] == rid and r["status"] == B.OK
        with pytest.raises(B.SvtError) as e:   # a second take of the same result
            srv.take(rid, r["n_tracks"])
            srv.take(rid, r["n_tracks"])
        assert e.value.code == B.E_STATE
    finally:
        srv.close()


@pytest.mark.parametrize("limits", [dict(max_words=8192), dict(max_events=7), dict(max_roads=300)],
                         ids=["words", "events", "roads"])
def test_a_request_larger_than_a_slot_is_split_at_event_boundaries(alone_ctx, orc, consts, cuts, limits):
    """A request with more words, events or roads than a slot holds runs in
    chunks on whichever slots free up; its one result equals the whole
    request run alone (and the oracle), next to ordinary requests."""
    big = synth.make_batch("scaled", seed=77, n_events=60).words      # about 60 k words
    small = requests(4, 6, 5)
    srv = B.Server(consts, cuts["scaled"], n_slots=2, **limits)
    try:
        got = serve_all(srv, small[:3] + [big] + small[3:])
    finally:
        srv.close()
    alone_ctx.load_constants(consts, cuts["scaled"])
    for i, w in enumerate(small[:3] + [big] + small[3:]):
        r, tracks = got[i]
        assert r["status"] == B.OK
        st, alone, stats = run_gpu(alone_ctx, w, B.PERSISTENT)
        assert st == B.OK and tracks.tobytes() == alone.tobytes(), i
        assert r["n_events"] == stats["n_events"] and r["n_combinations"] == stats["n_combinations"]
    rc, want = orc.run(big, consts, cuts["scaled"])
    assert rc == 0 and got[3][0]["n_events"] == 60
    assert_same_tracks(got[3][1], want)


def test_a_split_request_reports_the_first_failing_chunk(consts, cuts):
    """Status of a split request: the first chunk (in stream order) that
    failed; no tracks then.  An event larger than a slot is refused."""
    big = synth.make_batch("scaled", seed=78, n_events=40).words
    bad = big.copy()
    bad[len(bad) * 3 // 4] |= np.uint32(1 << 20)    # a reserved payload bit in a late chunk
    trunc = big[:-5]                                # the last event loses its end
    srv = B.Server(consts, cuts["scaled"], n_slots=2, max_words=4096)
    try:
        got = serve_all(srv, [bad, trunc, big])
    finally:
        srv.close()
    assert got[0][0]["status"] == B.E_BADWORD and got[0][0]["n_tracks"] == 0
    assert got[1][0]["status"] == B.E_TRUNCATED and got[1][0]["n_tracks"] == 0
    assert got[2][0]["status"] == B.OK and got[2][0]["n_events"] == 40
    one_event = int(np.diff(synth.make_batch("scaled", seed=78, n_events=2).event_offsets).max())
    srv = B.Server(consts, cuts["scaled"], n_slots=1, max_words=one_event - 1)
    try:
        with pytest.raises(B.SvtError) as e:
            srv.submit(big)
        assert e.value.code == B.E_CAPACITY
    finally:
        srv.close()
