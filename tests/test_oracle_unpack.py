"""Pins of the oracle's unpack stage (Sec. II-A, first function).

The generator's own record of what it encoded is the reference for round
trips; hand-written streams pin the grammar, the limits and the status codes.
"""
import numpy as np
import pytest

from paper_1312_0917_gb300 import synth

EE, EP = 1 << 31, 1 << 30


def hdr(wedge=0, barrel=0, excl=0):
    return (7 << 27) | wedge | (barrel << 4) | (excl << 7)


def cw(v):
    return (5 << 27) | (v & 0xFFFF)


def pw(v):
    return (6 << 27) | (v & 0xFFFF)


def hit(layer, c):
    return (layer << 27) | c


def road(hits, wedge=0, barrel=0, excl=0, curv=0, phi=0, last_of_event=False):
    w = [hdr(wedge, barrel, excl), cw(curv), pw(phi)] + [hit(l, c) for l, c in hits]
    w[-1] |= EP | (EE if last_of_event else 0)
    return w


def check_roundtrip(orc, b):
    rc, roads, ne, _ = orc.unpack(b.words)
    assert rc == 0 and ne == b.n_events and len(roads) == len(b.roads)
    t = b.roads
    for a, g in [("event", "event"), ("road", "road"), ("wedge", "wedge"),
                 ("barrel", "barrel"), ("excl", "excl"), ("curv", "curv"),
                 ("phi", "phi"), ("n", "n"), ("coord", "coords")]:
        assert np.array_equal(roads[a].astype(np.int64), t[g]), a


@pytest.mark.parametrize("name,n_events", [("small", None), ("scaled", 40),
                                           ("uneven", 300), ("stress", 3)])
def test_roundtrip_generator(orc, name, n_events):
    check_roundtrip(orc, synth.make_batch(name, seed=3, n_events=n_events))


def test_roundtrip_shared_hits(orc):
    cfg = synth.Config("sh", 30, ("fixed", 12), ("uniform", 1, 3), shared_hits=0.7)
    check_roundtrip(orc, synth.make_batch(cfg, seed=5))


def test_hand_stream_fields(orc):
    words = (road([(2, 7), (0, 4095), (2, 9), (4, 0)], wedge=11, barrel=5, excl=3,
                  curv=-32768, phi=32767)
             + road([(1, 1), (0, 2), (3, 3)], wedge=4, barrel=2, excl=0, curv=-1,
                    phi=5, last_of_event=True)
             + road([], wedge=1, barrel=1, excl=4, curv=2, phi=-2, last_of_event=True))
    rc, roads, ne, _ = orc.unpack(words)
    assert rc == 0 and ne == 2 and len(roads) == 3
    r0, r1, r2 = roads
    assert (r0["event"], r0["road"], r0["wedge"], r0["barrel"], r0["excl"]) == (0, 0, 11, 5, 3)
    assert (r0["curv"], r0["phi"]) == (-32768, 32767)
    assert list(r0["n"]) == [1, 0, 2, 0, 1]
    assert r0["coord"][0][0] == 4095 and list(r0["coord"][2][:2]) == [7, 9]
    assert r0["coord"][4][0] == 0
    assert (r1["event"], r1["road"], r1["curv"], r1["phi"]) == (0, 1, -1, 5)
    assert list(r1["n"]) == [1, 1, 0, 1, 0]
    assert (r2["event"], r2["road"], list(r2["n"])) == (1, 0, [0, 0, 0, 0, 0])


def test_hit_order_across_layers_is_irrelevant(orc):
    a = road([(0, 1), (1, 2), (0, 3), (2, 4)], last_of_event=True)
    b = road([(2, 4), (0, 1), (1, 2), (0, 3)], last_of_event=True)
    ra, rb = orc.unpack(a)[1], orc.unpack(b)[1]
    assert ra.tobytes() == rb.tobytes()


def test_empty_stream(orc):
    rc, roads, ne, _ = orc.unpack(np.zeros(0, np.uint32))
    assert rc == 0 and ne == 0 and len(roads) == 0


BAD, TRUNC, LIMIT = -2, -3, -4


def status(orc, words):
    rc, _, _, pos = orc.unpack(np.array(words, dtype=np.uint32))
    return rc, pos


def test_truncated(orc):
    w = road([(0, 1)], last_of_event=True)
    assert status(orc, w[:-1]) == (TRUNC, 3)               # cut mid-road
    w2 = road([(0, 1)]) + road([(0, 2)])                  # no EE at all
    assert status(orc, w2) == (TRUNC, len(w2))


def test_badword_cases(orc):
    good = road([(0, 1), (1, 2)], last_of_event=True)
    # a hit where the header belongs
    assert status(orc, [hit(0, 1)] + good) == (BAD, 0)
    # header field out of range: wedge 12, barrel 6, excluded layer 5
    for h in (hdr(12, 0, 0), hdr(0, 6, 0), hdr(0, 0, 5)):
        assert status(orc, [h] + good[1:]) == (BAD, 0)
    # reserved payload bits
    assert status(orc, good[:3] + [hit(0, 1) | (1 << 12)] + good[4:]) == (BAD, 3)
    assert status(orc, [good[0], cw(1) | (1 << 16)] + good[2:]) == (BAD, 1)
    assert status(orc, [hdr() | (1 << 10)] + good[1:]) == (BAD, 0)
    # EE without EP
    assert status(orc, good[:-1] + [good[-1] & ~EP]) == (BAD, len(good) - 1)
    # curvature and phi swapped
    assert status(orc, [good[0], good[2], good[1]] + good[3:]) == (BAD, 1)
    # road closed before its phi word
    assert status(orc, [hdr(), cw(0) | EP | EE]) == (BAD, 1)
    assert status(orc, [hdr() | EP | EE]) == (BAD, 0)
    # a header word in the hit section
    assert status(orc, good[:3] + [hdr()] + good[3:]) == (BAD, 3)


def test_limits(orc):
    nine = road([(2, i) for i in range(9)], last_of_event=True)
    assert status(orc, nine) == (LIMIT, 3 + 8)
    eight = road([(2, i) for i in range(8)], last_of_event=True)
    assert status(orc, eight) == (0, 0)
    ev = []
    for r in range(257):
        ev += road([(0, r)], last_of_event=(r == 256))
    assert status(orc, ev) == (LIMIT, 256 * 4)
    ok = []
    for r in range(256):
        ok += road([(0, r)], last_of_event=(r == 255))
    assert status(orc, ok)[0] == 0


def test_earliest_fault_wins_and_badword_before_limit(orc):
    ev = []
    for r in range(257):
        ev += road([(0, r)], last_of_event=(r == 256))
    bad_hdr = list(ev)
    bad_hdr[256 * 4] = hdr(12)                            # 257th header also malformed
    assert status(orc, bad_hdr) == (BAD, 256 * 4)
    early = list(ev)
    early[5] = hit(0, 1) | (1 << 20)                      # an earlier fault
    assert status(orc, early) == (BAD, 5)
