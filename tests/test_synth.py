"""The seeded input generator: published splitmix64 values, determinism, shapes."""
import numpy as np

from paper_1312_0917_gb300 import synth


def test_splitmix64_published_sequence():
    # splitmix64 seeded with 0: output i is mix((i + 1) * golden); the first
    # three are the widely quoted reference values of the generator
    # (Steele, Lea, Flood 2014).
    g = np.array([0x9E3779B97F4A7C15 * (i + 1) % (1 << 64) for i in range(3)],
                 dtype=np.uint64)
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in synth._mix(g)] == ref


def test_deterministic_and_seeded():
    a = synth.make_batch("small", seed=0)
    b = synth.make_batch("small", seed=0)
    c = synth.make_batch("small", seed=1)
    assert np.array_equal(a.words, b.words)
    assert not np.array_equal(a.words[:100], c.words[:100])


def test_uniform_int_range_and_spread():
    v = synth.uniform_int(0, 99, np.arange(200000), -3, 4)
    assert v.min() == -3 and v.max() == 4
    counts = np.bincount(v + 3)
    assert counts.min() > 0.95 * 25000 and counts.max() < 1.05 * 25000


def test_config_shapes():
    b = synth.make_batch("small")
    assert b.n_events == 100 and len(b.roads) == 800
    assert b.roads["n"].min() == 1 and b.roads["n"].max() == 2
    s = synth.make_batch("stress", n_events=2)
    assert len(s.roads) == 256 and (s.roads["n"] == 8).all()
    assert s.n_fits == 256 * 8 ** 5
    u = synth.make_batch("uneven", n_events=3000)
    rpe = np.bincount(u.roads["event"])
    assert rpe.min() >= 1 and rpe.max() <= 256
    assert 28 < rpe.mean() < 36                       # geometric, mean 32
    n = u.roads["n"].reshape(-1)
    assert n.max() <= 8 and abs((n == 1).mean() - 0.5) < 0.01


def test_words_well_formed():
    b = synth.make_batch("scaled", n_events=50)
    w = b.words
    ee = (w >> 31) & 1
    ep = (w >> 30) & 1
    assert ee.sum() == 50 and ep.sum() == len(b.roads)
    assert (ep[ee == 1] == 1).all() and ee[-1] == 1
    # event offsets are the positions after each EE word
    assert np.array_equal(np.nonzero(ee)[0] + 1, b.event_offsets[1:])


def test_request_sizes_cover_the_octaves():
    """Serving request sizes: in [1, 512), deterministic, every octave used
    about equally (log-uniform law)."""
    r = synth.request_sizes(0, 9000)
    assert r.min() >= 1 and r.max() < 512
    assert np.array_equal(r, synth.request_sizes(0, 9000))
    octave = np.floor(np.log2(r)).astype(int)
    counts = np.bincount(octave, minlength=9)
    assert len(counts) == 9 and counts.min() > 850 and counts.max() < 1150
