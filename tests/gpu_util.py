"""Helpers of the GPU tests: run a batch through the C ABI, run the oracle
(in parallel over event slices, spawned processes), compare bit for bit."""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def torch_words(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).cuda()


def run_gpu(ctx, words, mode, stream=None, d_words=None):
    """-> (status, TRACK_DTYPE host array, stats dict)"""
    from paper_1312_0917_gb300 import binding as B
    if d_words is None:
        d_words = torch_words(words) if len(words) else None
    st = ctx.unpack(d_words, len(words), stream)
    if st != B.OK:
        return st, np.zeros(0, dtype=B.TRACK_DTYPE), {}
    B.check(ctx.fit_events(mode, stream), "svt_fit_events")
    st, tracks = ctx.get_tracks(stream=stream)
    return st, tracks, ctx.get_stats(stream)


def pack_hits(coord):
    hits = np.zeros(len(coord), dtype=np.uint64)
    for l in range(5):
        hits |= coord[:, l].astype(np.uint64) << np.uint64(12 * l)
    return hits


def assert_same_tracks(gpu, orc):
    """GPU svt_track records == oracle survivors, field by field."""
    assert len(gpu) == len(orc), (len(gpu), len(orc))
    for f in ("event", "road", "comb", "chi2"):
        a, b = gpu[f].astype(np.int64), orc[f].astype(np.int64)
        if not np.array_equal(a, b):
            i = int(np.nonzero(a != b)[0][0])
            raise AssertionError("field %s differs first at %d: gpu %s oracle %s"
                                 % (f, i, gpu[i], orc[i]))
    assert np.array_equal(gpu["p"], orc["p"])
    assert np.array_equal(gpu["hits"], pack_hits(orc["coord"]))
    assert (gpu["pad"] == 0).all()


def _init_worker(root):
    if root not in sys.path:
        sys.path.insert(0, root)


def _oracle_slice(args):
    words, consts, cut, warrior = args
    import oracle
    return oracle.run(words, consts, cut, warrior)


def oracle_parallel(batch, consts, cut, n_slices=None, warrior=1):
    """Oracle over event slices of `batch` in spawned processes; event indices
    are shifted back to the batch's numbering."""
    import oracle
    oracle.build()
    E = batch.n_events
    n_proc = max(1, min(os.cpu_count() or 1, 32))
    n_slices = n_slices or min(E, 4 * n_proc)
    bounds = np.linspace(0, E, n_slices + 1).astype(int)
    jobs = [(batch.event_slice(a, b - a), consts, cut, warrior)
            for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    starts = [a for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    ctx = mp.get_context("spawn")
    with ctx.Pool(n_proc, initializer=_init_worker, initargs=(ROOT,)) as pool:
        res = pool.map(_oracle_slice, jobs)
    parts = []
    for (rc, arr), a in zip(res, starts):
        assert rc == 0, rc
        arr = arr.copy()
        arr["event"] += np.uint32(a)
        parts.append(arr)
    return np.concatenate(parts)
