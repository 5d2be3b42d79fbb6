"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work: bit-exact, every field of every surviving track, the status
codes and the counters.  Both execution modes are checked.
"""
import numpy as np
import pytest

from paper_1312_0917_gb300 import binding as B, synth
import hand_cases
from gpu_util import assert_same_tracks, oracle_parallel, run_gpu, torch_words
from test_oracle_warrior import shared_cfg

pytestmark = pytest.mark.gpu
MODES = [B.PERSISTENT, B.PLAIN]
MODE_IDS = ["persistent", "plain"]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    __graft_entry__.build()
    c = B.Context(0, max_combinations=1 << 27)
    yield c
    c.close()


def oracle_tracks(orc, words, consts, cut):
    rc, out = orc.run(words, consts, cut)
    assert rc == 0
    return out


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("case", hand_cases.CASES, ids=[c[0] for c in hand_cases.CASES])
def test_hand_cases(ctx, orc, case, mode):
    name, events, cut, expected = case
    words = hand_cases.case_words(events)
    ctx.load_constants(hand_cases.consts(), cut)
    st, got, _ = run_gpu(ctx, words, mode)
    assert st == B.OK
    assert [(int(t["event"]), int(t["road"]), int(t["comb"])) for t in got] == expected
    assert_same_tracks(got, oracle_tracks(orc, words, hand_cases.consts(), cut))


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_config(ctx, orc, consts, cuts, mode, seed):
    b = synth.make_batch("small", seed=seed)
    ctx.load_constants(consts, cuts["small"])
    st, got, stats = run_gpu(ctx, b.words, mode)
    assert st == B.OK
    want = oracle_tracks(orc, b.words, consts, cuts["small"])
    assert_same_tracks(got, want)
    rc, passing = orc.run(b.words, consts, cuts["small"], warrior=-1)
    assert stats["n_events"] == b.n_events and stats["n_roads"] == len(b.roads)
    assert stats["n_combinations"] == b.n_fits
    assert stats["n_passing"] == len(passing)
    assert stats["n_tracks"] == len(want)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_shared_hits_cross_road(ctx, orc, consts, mode, seed):
    """Roads of one event copy hits from each other: exercises the cross-road
    part of the hit-warrior."""
    b = synth.make_batch(shared_cfg(60), seed=seed)
    rc, chi = orc.chi2_all(b.words, consts)
    cut = int(np.sort(chi)[(9 * len(chi) + 9) // 10 - 1])
    ctx.load_constants(consts, cut)
    st, got, _ = run_gpu(ctx, b.words, mode)
    assert st == B.OK
    assert_same_tracks(got, oracle_tracks(orc, b.words, consts, cut))


@pytest.mark.parametrize("mode,max_ctas", [(B.PERSISTENT, 0), (B.PERSISTENT, 4), (B.PERSISTENT, 5),
                                           (B.PLAIN, 0)], ids=["persistent", "persistent-4", "persistent-5",
                                                               "plain"])
def test_event_sizes_around_the_warp_limit_of_the_flag_stage(ctx, orc, consts, mode, max_ctas):
    """The cross-road flag stage takes a batch of few events per CTA a CTA
    per event; with more events (here: a grid of 4 or 5 CTAs), events of at
    most 64 roads one warp each and larger ones a CTA each.  Events of 1, 2,
    63, 64, 65, 128 and 256 roads, interleaved, whose roads copy hits from
    each other, equal the oracle, and cross-road groups are published."""
    parts = []
    for i, r in enumerate((64, 65, 1, 63, 256, 64, 128, 65, 2, 63)):
        cfg = synth.Config("mix%d" % r, 3, ("fixed", r), ("uniform", 1, 3), shared_hits=0.6)
        parts.append(synth.make_batch(cfg, seed=40 + i).words)
    words = np.concatenate(parts)
    rc, chi = orc.chi2_all(words, consts)
    cut = int(np.sort(chi)[(9 * len(chi) + 9) // 10 - 1])
    ctx.load_constants(consts, cut)
    ctx.set_launch(max_ctas=max_ctas)
    try:
        st, got, stats = run_gpu(ctx, words, mode)
    finally:
        ctx.set_launch()
    assert st == B.OK and stats["n_groups"] > 0
    assert_same_tracks(got, oracle_tracks(orc, words, consts, cut))


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_duplicate_coordinates_and_empty_layers(ctx, orc, consts, mode):
    """Coordinates drawn from a tiny range: equal values inside a layer and
    across roads everywhere; hits 0..3 per layer (empty layers)."""
    cfg = synth.Config("dups", 40, ("fixed", 12), ("uniform", 0, 4))
    b = synth.make_batch(cfg, seed=5)
    w = b.words.copy()
    hit = ((w >> 27) & 7) <= 4
    w[hit] = (w[hit] & np.uint32(0xFFFFF000)) | (w[hit] & np.uint32(0x3))
    rc, chi = orc.chi2_all(w, consts)
    cut = int(np.sort(chi)[(9 * len(chi) + 9) // 10 - 1])
    ctx.load_constants(consts, cut)
    st, got, _ = run_gpu(ctx, w, mode)
    assert st == B.OK
    assert_same_tracks(got, oracle_tracks(orc, w, consts, cut))


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_scaled_full_batch(ctx, consts, cuts, mode):
    """The 3000-event x 64-road batch, every track checked."""
    b = synth.make_batch("scaled", seed=0)
    ctx.load_constants(consts, cuts["scaled"])
    st, got, stats = run_gpu(ctx, b.words, mode)
    assert st == B.OK and stats["n_combinations"] == b.n_fits
    assert_same_tracks(got, oracle_parallel(b, consts, cuts["scaled"]))


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_uneven_full_batch(ctx, consts, cuts, mode):
    b = synth.make_batch("uneven", seed=0)
    ctx.load_constants(consts, cuts["uneven"])
    st, got, stats = run_gpu(ctx, b.words, mode)
    assert st == B.OK and stats["n_combinations"] == b.n_fits
    assert_same_tracks(got, oracle_parallel(b, consts, cuts["uneven"]))


_STRESS = {}


def stress_oracle(orc, consts, cuts):
    """The stress batch and its oracle tracks (the oracle's event-parallel
    driver on every host core; computed once per session)."""
    if "want" not in _STRESS:
        b = synth.make_batch("stress", seed=0)
        rc, want, times = orc.run_mt(b.words, consts, cuts["stress"])
        assert rc == 0 and times["threads"] >= 1
        _STRESS.update(batch=b, want=want)
    return _STRESS["batch"], _STRESS["want"]


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_stress_every_event_against_the_oracle(orc, consts, cuts, mode):
    """200 events x 128 roads x 8^5 combinations (838,860,800 fits): the whole
    batch on the GPU, every track of every event against the oracle."""
    import __graft_entry__
    __graft_entry__.build()
    b, want = stress_oracle(orc, consts, cuts)
    c = B.Context(0, max_combinations=b.n_fits if mode == B.PLAIN else 1 << 10)
    try:
        c.load_constants(consts, cuts["stress"])
        st, got, stats = run_gpu(c, b.words, mode)
    finally:
        c.close()
    assert st == B.OK
    assert stats["n_combinations"] == b.n_fits == 200 * 128 * 8 ** 5
    assert_same_tracks(got, want)
    assert len(np.unique(got["event"])) == 200


_FULL = {}


@pytest.mark.parametrize("name", ["stress", "scaled", "uneven"])
def test_every_batch_in_the_benchmarks_launch_configuration(orc, consts, cuts, name):
    """The benchmark's timed configuration of each batch: autotuned on the
    batch, then replayed from a CUDA graph; every track of every event
    against the oracle.  On the stress batch also each block size's build at
    its occupancy maximum."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    if name == "stress":
        b, want = stress_oracle(orc, consts, cuts)
    else:
        if name not in _FULL:
            b = synth.make_batch(name, seed=0)
            _FULL[name] = (b, oracle_parallel(b, consts, cuts[name]))
        b, want = _FULL[name]
    c = B.Context(0, max_combinations=1 << 10)
    try:
        c.load_constants(consts, cuts[name])
        d = torch_words(b.words)
        assert c.unpack(d, len(b.words)) == B.OK
        c.autotune(reps=1)
        c.use_graph(True)
        for _ in range(2):
            st, got, _ = run_gpu(c, b.words, B.PERSISTENT, d_words=d)
            assert st == B.OK
            assert_same_tracks(got, want)
        c.use_graph(False)
        if name == "stress":
            for block in (128, 256, 512):
                c.set_launch(block=block)
                st, other, _ = run_gpu(c, b.words, B.PERSISTENT, d_words=d)
                assert st == B.OK and other.tobytes() == got.tobytes(), block
    finally:
        c.close()


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_unpack_roads(ctx, orc, consts, cuts, mode):
    b = synth.make_batch("uneven", seed=4, n_events=400)
    ctx.load_constants(consts, cuts["uneven"])
    d = torch_words(b.words)
    assert ctx.unpack(d, len(b.words)) == B.OK
    if mode == B.PERSISTENT:
        B.check(ctx.fit_events(mode), "fit")
    st, roads = ctx.get_roads()
    assert st == B.OK
    rc, want, ne, _ = orc.unpack(b.words)
    assert len(roads) == len(want)
    for f in ("event", "road", "wedge", "barrel", "excl", "curv", "phi", "n"):
        assert np.array_equal(roads[f].astype(np.int64), want[f].astype(np.int64)), f
    assert np.array_equal(roads["coord"], want["coord"])


def malformed_streams():
    from test_oracle_unpack import road, hdr, hit, cw, EE, EP
    good = road([(0, 1), (1, 2)], last_of_event=True)
    ev257 = []
    for r in range(257):
        ev257 += road([(0, r)], last_of_event=(r == 256))
    big = list(synth.make_batch("small", seed=1).words)
    cases = {
        "empty": [],
        "truncated_mid_road": good[:-1],
        "no_ee": road([(0, 1)]) + road([(0, 2)]),
        "hit_first": [hit(0, 1)] + good,
        "bad_wedge": [hdr(12)] + good[1:],
        "reserved_hit_bits": good[:3] + [hit(0, 1) | (1 << 12)] + good[4:],
        "ee_without_ep": good[:-1] + [good[-1] & ~EP],
        "swapped_xft": [good[0], good[2], good[1]] + good[3:],
        "short_road": [hdr(), cw(0) | EP | EE],
        "nine_hits": road([(2, i) for i in range(9)], last_of_event=True),
        "257_roads": ev257,
        "bad_257th_header": ev257[:256 * 4] + [hdr(12)] + ev257[256 * 4 + 1:],
        "late_fault_after_good_events": big[:-5] + [big[-5] | (1 << 20)] + big[-4:],
        "limit_then_bad": road([(2, i) for i in range(9)]) + [hit(0, 1) | (1 << 13)] + good,
        "trailing_road_after_ee": good + road([(1, 1)]),
        # roads of 256 words or more (only malformed ones can be that long)
        # take the decoder's per-layer counting path
        "long_road_limit": road([(2, i % 4096) for i in range(300)], last_of_event=True),
        "long_road_among_short": road([(0, 1)]) + road([(1, i % 4096) for i in range(300)]) +
                                 road([(0, 2)], last_of_event=True),
        "long_road_bad_after_limit": (lambda r: r[:200] + [r[200] | (1 << 13)] + r[201:])(
            road([(3, i % 4096) for i in range(300)], last_of_event=True)),
        "long_road_bad_before_limit": (lambda r: r[:5] + [r[5] | (1 << 13)] + r[6:])(
            road([(3, i % 4096) for i in range(300)], last_of_event=True)),
    }
    return cases


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("name", list(malformed_streams()))
def test_status_codes_match_oracle(ctx, orc, consts, mode, name):
    words = np.array(malformed_streams()[name], dtype=np.uint32)
    ctx.load_constants(consts, 1 << 40)
    rc, _, _, pos = orc.unpack(words)
    st, got, stats = run_gpu(ctx, words, mode)
    assert st == rc, (st, rc)
    if rc != 0:
        assert len(got) == 0 and stats["status"] == rc and stats["error_word"] == pos
    else:
        rc2, want = orc.run(words, consts, 1 << 40)
        assert_same_tracks(got, want)


def test_back_to_back_batches_and_modes(ctx, orc, consts, cuts):
    """State is reset between batches: alternate configs and modes."""
    ctx.load_constants(consts, cuts["small"])
    for seed, mode in [(7, B.PERSISTENT), (8, B.PLAIN), (7, B.PERSISTENT), (9, B.PERSISTENT)]:
        b = synth.make_batch(shared_cfg(30), seed=seed)
        st, got, _ = run_gpu(ctx, b.words, mode)
        assert st == B.OK
        assert_same_tracks(got, oracle_tracks(orc, b.words, consts, cuts["small"]))


def launch_grid(ctx):
    """Every configuration the autotuner measures (block size, CTAs per SM up
    to that size's occupancy maximum, small_n4, roads per queue claim)."""
    out = []
    for block in (128, 256, 512):
        ctx.set_launch(block=block)
        for bps in range(1, ctx.get_launch()["blocks_per_sm"] + 1):
            for small in (64, 128, 256):
                for run in (4, 8, 16):
                    out.append(dict(block=block, blocks_per_sm=bps, small_n4=small, run_roads=run, max_ctas=0))
    ctx.set_launch()
    return out


def test_launch_settings_are_bit_equal(ctx, orc, consts, cuts):
    """Every launch configuration of the autotuner's grid, and a few outside
    it, give the same bytes as the default on an uneven batch (which equals
    the oracle)."""
    b = synth.make_batch("uneven", seed=2, n_events=1500)
    ctx.load_constants(consts, cuts["uneven"])
    ctx.set_launch()
    st, ref, _ = run_gpu(ctx, b.words, B.PERSISTENT)
    assert st == B.OK
    assert_same_tracks(ref, oracle_tracks(orc, b.words, consts, cuts["uneven"]))
    grid = launch_grid(ctx)
    assert {g["block"] for g in grid} == {128, 256, 512} and len(grid) >= 3 * 3 * 3 * 3
    extra = [dict(block=256, blocks_per_sm=0, small_n4=16, run_roads=4),
             dict(block=512, blocks_per_sm=0, small_n4=1, run_roads=16)]
    for cfg in grid + extra:
        ctx.set_launch(**cfg)
        st2, got, _ = run_gpu(ctx, b.words, B.PERSISTENT)
        assert st2 == B.OK and ref.tobytes() == got.tobytes(), cfg
    ctx.set_launch()


def test_launch_settings_are_checked(ctx):
    for bad in (dict(block=64), dict(block=384), dict(run_roads=3), dict(run_roads=32),
                dict(small_n4=257), dict(blocks_per_sm=-1), dict(max_ctas=-1)):
        with pytest.raises(B.SvtError) as e:
            ctx.set_launch(**bad)
        assert e.value.code == B.E_INVAL
    ctx.set_launch(block=512)
    got = ctx.get_launch()
    assert got["block"] == 512 and got["blocks_per_sm"] >= 1 and got["small_n4"] == 256 and got["run_roads"] == 8
    ctx.set_launch()


def test_graph_launch(ctx, consts, cuts):
    import torch
    b = synth.make_batch("scaled", seed=3, n_events=300)
    ctx.load_constants(consts, cuts["scaled"])
    s = torch.cuda.Stream()
    d = torch_words(b.words)
    st, ref, _ = run_gpu(ctx, b.words, B.PERSISTENT, stream=s, d_words=d)
    ctx.use_graph(True)
    try:
        for _ in range(3):
            st2, got, _ = run_gpu(ctx, b.words, B.PERSISTENT, stream=s, d_words=d)
            assert st2 == B.OK and got.tobytes() == ref.tobytes()
        st3, got3, _ = run_gpu(ctx, b.words, B.PLAIN, stream=s, d_words=d)
        assert st3 == B.OK and got3.tobytes() == ref.tobytes()
    finally:
        ctx.use_graph(False)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_words_and_tracks_in_page_locked_host_memory(ctx, orc, consts, cuts, mode):
    """The kernels read words from page-locked host memory in place and the
    output stage writes the tracks into a page-locked host buffer: the same
    tracks as device buffers (and the oracle), with and without a graph; a
    host buffer too small for the tracks is a capacity error."""
    import torch
    b = synth.make_batch("scaled", seed=21, n_events=200)
    ctx.load_constants(consts, cuts["scaled"])
    st, ref, _ = run_gpu(ctx, b.words, mode)
    assert st == B.OK
    assert_same_tracks(ref, oracle_tracks(orc, b.words, consts, cuts["scaled"]))
    h_words = torch.from_numpy(b.words.view(np.int32)).pin_memory()
    h_out = torch.zeros(len(ref) * 40 + 4000, dtype=torch.uint8).pin_memory()
    cap = h_out.numel() // 40
    try:
        ctx.set_track_output(h_out, cap)
        for graph in (False, True, True):
            ctx.use_graph(graph and mode == B.PERSISTENT)
            assert ctx.unpack(h_words, len(b.words)) == B.OK
            B.check(ctx.fit_events(mode), "svt_fit_events")
            st, n = ctx.get_tracks(out=h_out, cap=cap)
            assert st == B.OK and n == len(ref)
            assert h_out.numpy()[:n * 40].tobytes() == ref.tobytes()
        ctx.use_graph(False)
        st, other = ctx.get_tracks()   # a copy out of the host buffer
        assert st == B.OK and other.tobytes() == ref.tobytes()
        ctx.set_track_output(h_out, len(ref) - 1)
        assert ctx.unpack(h_words, len(b.words)) == B.OK
        B.check(ctx.fit_events(mode), "svt_fit_events")
        st, n = ctx.get_tracks(out=h_out, cap=cap)
        assert st == B.E_CAPACITY
    finally:
        ctx.use_graph(False)
        ctx.set_track_output(None)
    st, got, _ = run_gpu(ctx, b.words, mode)
    assert st == B.OK and got.tobytes() == ref.tobytes()


def test_pageable_host_memory_is_refused(ctx, consts, cuts):
    b = synth.make_batch("small", seed=1)
    ctx.load_constants(consts, cuts["small"])
    words = np.ascontiguousarray(b.words)
    assert ctx.unpack(words, len(words)) == B.E_INVAL
    out = np.zeros(100, dtype=B.TRACK_DTYPE)
    with pytest.raises(B.SvtError) as e:
        ctx.set_track_output(out, len(out))
    assert e.value.code == B.E_INVAL


def test_capacity_errors(consts, cuts):
    import __graft_entry__
    __graft_entry__.build()
    b = synth.make_batch("small", seed=0)
    c = B.Context(0, max_tracks=16, max_words=1 << 14, max_events=1 << 8, max_roads=1 << 12,
                  hash_slots=1 << 10, max_combinations=1 << 14)
    c.load_constants(consts, cuts["small"])
    st, got, _ = run_gpu(c, b.words, B.PERSISTENT)
    assert st == B.E_CAPACITY and len(got) == 0
    big = synth.make_batch("small", seed=0, n_events=300)
    d = torch_words(big.words)
    assert c.unpack(d, len(big.words)) == B.E_CAPACITY          # > max_words
    c.close()


def test_word_limit_of_contexts_and_servers(consts, cuts):
    """A batch holds fewer than 2^31 words: larger limits are refused at
    creation (SVT_E_INVAL) for contexts and servers alike."""
    with pytest.raises(B.SvtError) as e:
        B.Context(0, max_words=1 << 31)
    assert e.value.code == B.E_INVAL
    with pytest.raises(B.SvtError) as e:
        B.Server(consts, cuts["small"], n_slots=1, max_words=1 << 31)
    assert e.value.code == B.E_INVAL
    c = B.Context(0, max_words=(1 << 20) + 1)   # a limit below 2^31 is accepted
    c.close()


def test_timeout_is_reported_and_context_survives(consts, cuts, orc):
    """A CTA that never arrives at the first grid barrier: the others' bounded
    waits run out (1 ms), the batch ends with SVT_E_TIMEOUT, and the next
    batch on the same context is correct."""
    import __graft_entry__
    __graft_entry__.build()
    b = synth.make_batch("small", seed=0)
    c = B.Context(0)
    c.load_constants(consts, cuts["small"])
    c.debug_wait(1000, True)
    st, got, _ = run_gpu(c, b.words, B.PERSISTENT)
    assert st == B.E_TIMEOUT and len(got) == 0
    c.debug_wait(0, False)
    st, got, _ = run_gpu(c, b.words, B.PERSISTENT)
    assert st == B.OK
    assert_same_tracks(got, oracle_tracks(orc, b.words, consts, cuts["small"]))
    c.close()


def test_graph_replay_after_a_timeout_that_left_the_group_table_dirty(consts, orc):
    """A batch whose barrier wait runs out after the fit stage leaves group
    minima in the cross-road table.  With graph replay on, the cached graph
    of the next batches must not skip the clearing: two replays after the
    timeout equal the oracle and publish every group anew (a stale table
    would already hold them, and none would be counted)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    b = synth.make_batch(shared_cfg(60), seed=2)
    rc, chi = orc.chi2_all(b.words, consts)
    cut = int(np.sort(chi)[(9 * len(chi) + 9) // 10 - 1])
    want = oracle_tracks(orc, b.words, consts, cut)
    c = B.Context(0)
    c.load_constants(consts, cut)
    s = torch.cuda.Stream()
    d = torch_words(b.words)
    try:
        c.debug_wait(100000, 0)   # 100 ms waits, held by the graph
        c.use_graph(True)
        st, got, stats = run_gpu(c, b.words, B.PERSISTENT, stream=s, d_words=d)
        assert st == B.OK
        assert_same_tracks(got, want)
        groups = stats["n_groups"]
        assert groups > 0
        c.debug_wait(100000, 2)   # block 0 leaves after the fit stage, once
        st, got, _ = run_gpu(c, b.words, B.PERSISTENT, stream=s, d_words=d)
        assert st == B.E_TIMEOUT and len(got) == 0
        for _ in range(2):
            st, got, stats = run_gpu(c, b.words, B.PERSISTENT, stream=s, d_words=d)
            assert st == B.OK and stats["n_groups"] == groups
            assert_same_tracks(got, want)
    finally:
        c.close()


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_group_table_overflow_is_a_capacity_error(consts, orc, mode):
    """A batch with more cross-road groups than 3/4 of a small group table:
    SVT_E_CAPACITY and no tracks; the table is left empty, so the next batch
    on the context is correct."""
    import __graft_entry__
    __graft_entry__.build()
    b = synth.make_batch(shared_cfg(60), seed=3)
    rc, chi = orc.chi2_all(b.words, consts)
    cut = int(np.sort(chi)[(9 * len(chi) + 9) // 10 - 1])
    big = B.Context(0, max_combinations=1 << 20)
    big.load_constants(consts, cut)
    st, _, stats = run_gpu(big, b.words, mode)
    big.close()
    assert st == B.OK and stats["n_groups"] > 48
    c = B.Context(0, hash_slots=1 << 6, max_combinations=1 << 20)
    try:
        c.load_constants(consts, cut)
        st, got, _ = run_gpu(c, b.words, mode)
        assert st == B.E_CAPACITY and len(got) == 0
        small = synth.make_batch("small", seed=0)
        c.load_constants(consts, cut)
        st, got, stats = run_gpu(c, small.words, mode)
        assert st == B.OK and stats["n_groups"] <= 48
        assert_same_tracks(got, oracle_tracks(orc, small.words, consts, cut))
    finally:
        c.close()


def test_constant_bounds_rejected():
    import __graft_entry__
    __graft_entry__.build()
    c = B.Context(0, max_words=1 << 12)
    z = hand_cases.consts()
    z["C"][5, 0, :] = 32767              # could overflow the exact 32-bit sum
    with pytest.raises(B.SvtError) as e:
        c.load_constants(z, 1)
    assert e.value.code == B.E_INVAL
    c.close()


def test_autotune_keeps_the_fastest_and_the_tracks(ctx, orc, consts, cuts):
    b = synth.make_batch("uneven", seed=3, n_events=300)
    ctx.load_constants(consts, cuts["uneven"])
    d = torch_words(b.words)
    assert ctx.unpack(d, len(b.words)) == B.OK
    grid = launch_grid(ctx)
    pts = ctx.autotune(reps=3)
    assert [p[0] for p in pts] == grid
    assert all(p[1] > 0 for p in pts)
    assert ctx.get_launch() == min(pts, key=lambda p: p[1])[0]   # the fastest is kept
    st, got, _ = run_gpu(ctx, b.words, B.PERSISTENT, d_words=d)
    assert st == B.OK
    assert_same_tracks(got, oracle_tracks(orc, b.words, consts, cuts["uneven"]))
    ctx.set_launch()


def test_two_contexts_taking_batches_in_turn(ctx, consts, cuts):
    """The end-to-end pattern of the benchmark: two contexts on two streams,
    batch i + 1 copied in and launched before batch i's tracks are read back
    (their cooperative kernels queue behind each other).  Every batch equals
    the same batch run alone."""
    import torch
    batches = [synth.make_batch("scaled", seed=s, n_events=400) for s in (11, 12, 13, 14, 15)]
    ctx.load_constants(consts, cuts["scaled"])
    ctx.use_graph(False)
    ref = []
    for b in batches:
        st, t, _ = run_gpu(ctx, b.words, B.PERSISTENT)
        assert st == B.OK
        ref.append(t.tobytes())
    ctxs = [ctx, B.Context(0)]
    ctxs[1].load_constants(consts, cuts["scaled"])
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    h = [torch.from_numpy(b.words.view(np.int32)).pin_memory() for b in batches]
    n_max = max(len(b.words) for b in batches)
    d = [torch.empty(n_max, dtype=torch.int32, device="cuda") for _ in range(2)]
    try:
        for graph in (False, True):
            for c in ctxs:
                c.use_graph(graph)

            def submit(i):
                k = i % 2
                with torch.cuda.stream(streams[k]):
                    d[k][:h[i].numel()].copy_(h[i], non_blocking=True)
                assert ctxs[k].unpack(d[k], h[i].numel(), streams[k]) == B.OK
                B.check(ctxs[k].fit_events(B.PERSISTENT, streams[k]), "svt_fit_events")

            submit(0)
            for i in range(len(batches)):
                if i + 1 < len(batches):
                    submit(i + 1)
                st, t = ctxs[i % 2].get_tracks(stream=streams[i % 2])
                assert st == B.OK and t.tobytes() == ref[i], (graph, i)
    finally:
        ctx.use_graph(False)
        ctxs[1].close()


def test_integer_peak_is_measured():
    """svt_measure_int_peak: positive rates of the order of the device's
    multiply-add lanes x clock (152 SMs x 64 lanes x ~2 GHz ~ 2e13)."""
    import __graft_entry__
    __graft_entry__.build()
    peak = B.measure_int_peak(0)
    assert 1e12 < peak["imad"] < 1e14 and 1e12 < peak["iadd"] < 1e14
    assert peak["mixed"] >= 0.9 * peak["imad"]
