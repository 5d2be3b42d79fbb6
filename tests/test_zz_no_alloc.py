"""svt_run_static (no allocation at call time, fixed device arena) gives the
same tracks, status and counts as the context path, on two calls in a row.
Kept last in collection order so that it also runs after every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1312_0917_gb300 import binding as B, synth
from gpu_util import run_gpu, torch_words
from test_oracle_warrior import shared_cfg

pytestmark = pytest.mark.gpu


def run_static(words, consts, cut, cap):
    import torch
    d_words = torch_words(words) if len(words) else None
    d_tracks = torch.zeros(max(cap, 1) * 40, dtype=torch.uint8, device="cuda")
    sets = B.pack_constants(consts)
    n = C.c_size_t()
    st = B.lib().svt_run_static(B.ptr(d_words), len(words), sets.ctypes.data, len(sets), int(cut),
                                d_tracks.data_ptr(), cap, C.byref(n), None)
    torch.cuda.synchronize()
    out = d_tracks.cpu().numpy().view(B.TRACK_DTYPE)[: min(n.value, cap)]
    return st, n.value, out


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = B.Context(0)
    yield c
    c.close()


def test_two_calls_in_a_row_equal_the_context_path(ctx, consts, cuts):
    batches = [synth.make_batch("small", seed=0).words,
               synth.make_batch(shared_cfg(60), seed=4).words]
    for words, cut in zip(batches, (cuts["small"], cuts["small"])):
        ctx.load_constants(consts, cut)
        st0, want, stats = run_gpu(ctx, words, B.PERSISTENT)
        assert st0 == B.OK
        st, n, got = run_static(words, consts, cut, len(want) + 16)
        assert st == B.OK and n == len(want) == stats["n_tracks"]
        assert got.tobytes() == want.tobytes()


def test_limits_and_errors(consts, cuts):
    words = synth.make_batch("small", seed=1).words
    st, n, _ = run_static(words, consts, cuts["small"], 10)          # tracks do not fit
    assert st == B.E_CAPACITY and n > 10
    big = np.zeros((1 << 17) + 1, np.uint32)
    sets = B.pack_constants(consts)
    n = C.c_size_t()
    assert B.lib().svt_run_static(None, len(big), sets.ctypes.data, len(sets), 0, None, 0,
                                  C.byref(n), None) == B.E_INVAL
    st, n, _ = run_static(big, consts, cuts["small"], 16)             # words beyond the arena
    assert st == B.E_CAPACITY
    bad = words.copy()
    bad[7] |= np.uint32(1 << 20)
    st, n, _ = run_static(bad, consts, cuts["small"], 4096)
    assert st == B.E_BADWORD and n == 0
    st, n, got = run_static(words, consts, cuts["small"], 4096)      # and it still works
    assert st == B.OK and n == len(got) > 0


def _at_limit_configs():
    # 1025 events (one road each), 8199 roads (911 events of 9): both below
    # the arena's 131072 words; 1024 events x 8 roads: exactly at both limits
    return {"events": synth.Config("ev1025", 1025, ("fixed", 1), ("uniform", 1, 1)),
            "roads": synth.Config("rd8199", 911, ("fixed", 9), ("uniform", 1, 1)),
            "at_limit": synth.Config("ev1024", 1024, ("fixed", 8), ("uniform", 1, 1))}


@pytest.mark.parametrize("what", ["events", "roads"])
def test_arena_event_and_road_limits(ctx, consts, cuts, what):
    """More events or roads than the arena holds: SVT_E_CAPACITY with no
    tracks (checked on the device); the next call still equals the context
    path."""
    b = synth.make_batch(_at_limit_configs()[what], seed=6)
    assert len(b.words) < (1 << 17)
    st, n, _ = run_static(b.words, consts, cuts["small"], 1 << 14)
    assert st == B.E_CAPACITY and n == 0
    good = synth.make_batch("small", seed=2).words
    ctx.load_constants(consts, cuts["small"])
    st0, want, _ = run_gpu(ctx, good, B.PERSISTENT)
    st, n, got = run_static(good, consts, cuts["small"], len(want) + 16)
    assert st0 == st == B.OK and n == len(want)
    assert got.tobytes() == want.tobytes()


def test_batch_at_the_event_and_road_limits_equals_the_context_path(ctx, consts, cuts):
    """1024 events and 8192 roads, exactly the arena's limits: byte for byte
    the context path's tracks, twice in a row."""
    b = synth.make_batch(_at_limit_configs()["at_limit"], seed=7)
    assert b.n_events == 1024 and len(b.roads) == 8192
    ctx.load_constants(consts, cuts["small"])
    st0, want, _ = run_gpu(ctx, b.words, B.PERSISTENT)
    assert st0 == B.OK and len(want) > 0
    for _ in range(2):
        st, n, got = run_static(b.words, consts, cuts["small"], len(want) + 16)
        assert st == B.OK and n == len(want)
        assert got.tobytes() == want.tobytes()
