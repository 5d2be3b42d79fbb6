"""Pins of the oracle's hit-warrior (and the chain end to end).

The rule: among one event's passing combinations, t is dropped iff some u
with a lower key (chi2, road, comb) shares >= 3 hits (equal coordinate on the
same layer).  The references here are hand derivations (hand_cases.py) and a
numpy brute force over all pairs, applied to the oracle's passing list.
"""
import numpy as np
import pytest

from paper_1312_0917_gb300 import synth
import hand_cases


def brute_force_survivors(passing):
    """Pairwise rule over all pairs of each event (numpy, blocked)."""
    keep = np.ones(len(passing), dtype=bool)
    ev = passing["event"]
    bounds = np.concatenate([[0], np.nonzero(np.diff(ev))[0] + 1, [len(ev)]])
    for a, b in zip(bounds[:-1], bounds[1:]):
        p = passing[a:b]
        order = np.lexsort((p["comb"], p["road"], p["chi2"]))
        rank = np.empty(len(p), dtype=np.int64)
        rank[order] = np.arange(len(p))                # rank of the key
        co = p["coord"].astype(np.int32)
        for i0 in range(0, len(p), 256):
            blk = co[i0:i0 + 256]
            shared = (blk[:, None, :] == co[None, :, :]).sum(axis=2)
            lower = rank[None, :] < rank[i0:i0 + 256, None]
            keep[a + i0:a + i0 + len(blk)] = ~((shared >= 3) & lower).any(axis=1)
    return passing[keep]


def same_tracks(a, b):
    fields = ("event", "road", "comb", "p", "chi2", "coord")
    return len(a) == len(b) and all(np.array_equal(a[f], b[f]) for f in fields)


@pytest.mark.parametrize("name,events,cut,expected", hand_cases.CASES,
                         ids=[c[0] for c in hand_cases.CASES])
@pytest.mark.parametrize("mode", [0, 1])
def test_hand_cases(orc, name, events, cut, expected, mode):
    words = hand_cases.case_words(events)
    rc, out = orc.run(words, hand_cases.consts(), cut, warrior=mode)
    assert rc == 0
    got = [(int(t["event"]), int(t["road"]), int(t["comb"])) for t in out]
    assert got == expected


def shared_cfg(n_events=40):
    return synth.Config("shared", n_events, ("fixed", 10), ("uniform", 1, 3),
                        shared_hits=0.6)


@pytest.mark.parametrize("cfg,seed", [("small", 0), ("small", 4), (shared_cfg(), 1),
                                      (shared_cfg(), 2)])
def test_matches_brute_force(orc, consts, cfg, seed):
    b = synth.make_batch(cfg, seed=seed)
    rc, allfits = orc.fit_all(b.words, consts)
    cut = int(np.sort(allfits["chi2"])[(9 * len(allfits) + 9) // 10 - 1])
    rc, passing = orc.run(b.words, consts, cut, warrior=-1)
    want = brute_force_survivors(passing)
    for mode in (0, 1):
        rc, got = orc.run(b.words, consts, cut, warrior=mode)
        assert rc == 0 and same_tracks(got, want), mode
    if isinstance(cfg, synth.Config):
        # cross-road kills happened: some survivor of a road-local brute force
        # is dropped by another road of its event
        local = []
        for (e, r) in {(int(x["event"]), int(x["road"])) for x in passing}:
            sel = passing[(passing["event"] == e) & (passing["road"] == r)]
            local.append(brute_force_survivors(sel))
        assert sum(len(x) for x in local) > len(want)


def test_scaled_events_match_brute_force(orc, consts, cuts):
    b = synth.make_batch("scaled", seed=0, n_events=3)
    rc, passing = orc.run(b.words, consts, cuts["scaled"], warrior=-1)
    want = brute_force_survivors(passing)
    rc, got = orc.run(b.words, consts, cuts["scaled"], warrior=1)
    assert same_tracks(got, want)


def test_invariant_under_hit_word_order(orc, consts, cuts):
    """Reordering hit words across layers (same order within each layer)
    leaves the output unchanged."""
    b = synth.make_batch("small", seed=9)
    rc, ref = orc.run(b.words, consts, cuts["small"])
    w = b.words.copy()
    typ = (w >> 27) & 7
    ep = (w >> 30) & 1
    out = []
    start = 0
    for end in np.nonzero(ep)[0]:
        rw = w[start:end + 1].copy()
        flags = rw[-1] & np.uint32(0xC0000000)
        rw[-1] &= np.uint32(0x3FFFFFFF)
        hits = rw[3:]
        order = np.argsort(-(typ[start + 3:end + 1].astype(np.int64)), kind="stable")
        rw[3:] = hits[order]
        rw[-1] |= flags
        out.append(rw)
        start = end + 1
    w2 = np.concatenate(out)
    assert not np.array_equal(w2, b.words)
    rc, got = orc.run(w2, consts, cuts["small"])
    assert same_tracks(got, ref)


def test_survivor_invariants(orc, consts, cuts):
    """survivors subset of passing subset of fits; no survivor has a lower-key
    partner sharing >= 3 hits among the survivors either."""
    b = synth.make_batch("small", seed=0)
    rc, fits = orc.fit_all(b.words, consts, cuts["small"])
    rc, passing = orc.run(b.words, consts, cuts["small"], warrior=-1)
    rc, surv = orc.run(b.words, consts, cuts["small"], warrior=1)
    key = lambda a: set(zip(a["event"].tolist(), a["road"].tolist(), a["comb"].tolist()))
    assert key(surv) <= key(passing) <= key(fits)
    assert len(brute_force_survivors(surv)) == len(surv)
