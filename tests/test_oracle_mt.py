"""The event-parallel oracle driver (OpenMP over events) against the serial
oracle: the same survivors, bit for bit, for any thread count, and the same
status on malformed input."""
import numpy as np
import pytest

from paper_1312_0917_gb300 import synth
from test_oracle_warrior import shared_cfg


@pytest.mark.parametrize("cfg,seed", [("small", 0), ("small", 3), (shared_cfg(30), 1)])
@pytest.mark.parametrize("threads", [1, 3, 0])
def test_equals_serial(orc, consts, cuts, cfg, seed, threads):
    b = synth.make_batch(cfg, seed=seed)
    cut = cuts["small"]
    rc, want = orc.run(b.words, consts, cut)
    rc2, got, times = orc.run_mt(b.words, consts, cut, threads=threads)
    assert rc == rc2 == 0
    assert got.tobytes() == want.tobytes()
    assert times["threads"] >= 1 and (threads == 0 or times["threads"] == threads)
    assert times["wall_s"] >= times["unpack_s"] >= 0 and times["fit_s"] >= 0 and times["warrior_s"] >= 0


def test_uneven_slice_and_pairwise_rule(orc, consts, cuts):
    b = synth.make_batch("uneven", seed=1, n_events=60)
    for warrior in (0, 1, -1):
        rc, want = orc.run(b.words, consts, cuts["uneven"], warrior)
        rc2, got, _ = orc.run_mt(b.words, consts, cuts["uneven"], warrior, threads=4)
        assert rc == rc2 == 0 and got.tobytes() == want.tobytes()


def test_malformed_stream_status(orc, consts):
    w = synth.make_batch("small", seed=0).words.copy()
    w[5] |= np.uint32(1 << 20)
    rc, _ = orc.run(w, consts, 1 << 40)
    rc2, got, _ = orc.run_mt(w, consts, 1 << 40, threads=2)
    assert rc == rc2 != 0 and len(got) == 0
    rc3, got3, _ = orc.run_mt(w[:-1], consts, 1 << 40)   # truncated
    assert rc3 == orc.run(w[:-1], consts, 1 << 40)[0]
