"""Seeded synthetic inputs for the SVT track-fitting chain.

This module produces INPUTS only: the packed 32-bit word stream of a batch of
events and the fit-constant tables.  It holds none of the fitting arithmetic
(no fit, no chi-square, no cut, no hit-warrior), so both the CUDA path and the
CPU oracle can consume what it writes without sharing any of the method.

Word format (one 32-bit word per datum; the paper's "packed input data" of
Sec. II-A, with the field layout fixed by this library):

    bit 31      EE  end of event   (only on the last word of an event, which
                                    also carries EP)
    bit 30      EP  end of road    (on the last word of every road)
    bits 29..27 type: 0..4 silicon hit on that layer, 5 XFT curvature,
                6 XFT phi, 7 road header
    bits 26..0  payload: hit -> coordinate in bits 11..0;
                curvature / phi -> int16 in bits 15..0 (two's complement);
                header -> wedge bits 3..0, barrel bits 6..4,
                          excluded layer bits 9..7

A road is: header, curvature, phi, then its hits in any layer order.  The
d-th hit word of layer l inside a road is hit index d of that layer.

Random numbers: every quantity is a counter-based draw, splitmix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
evaluated at (seed, stream, element index), so values do not depend on how
the generation is vectorised and are identical on x86-64 and aarch64 (pure
64-bit integer arithmetic, no floating point anywhere).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

__all__ = [
    "Config", "CONFIGS", "Batch", "make_constants", "make_batch",
    "encode_roads", "request_sizes", "N_SETS", "N_LAYERS", "MAX_HITS", "MAX_ROADS",
]

N_LAYERS = 5          # silicon layers per road
MAX_HITS = 8          # hits per layer per road (format limit)
MAX_ROADS = 256       # roads per event (format limit)
N_WEDGES, N_BARRELS = 12, 6
N_SETS = N_WEDGES * N_BARRELS * N_LAYERS   # 360 constant sets

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (arbitrary distinct constants)
_S_NROADS, _S_WEDGE, _S_BARREL, _S_EXCL, _S_CURV, _S_PHI = 1, 2, 3, 4, 5, 6
_S_NHITS, _S_COORD, _S_ORDER, _S_SHARE = 7, 8, 9, 10
_S_F, _S_Q, _S_C, _S_K = 20, 21, 22, 23


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def draws(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """64-bit draws number `index` (0-based) of the splitmix64 sequence whose
    state starts at key(seed, stream) = splitmix64 output `stream` of `seed`."""
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        key = _mix(s + np.uint64(stream + 1) * _GOLDEN)[0]
        idx = np.asarray(index, dtype=np.uint64)
        return _mix(key + (idx + np.uint64(1)) * _GOLDEN)


def uniform_int(seed: int, stream: int, index, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on [lo, hi] (hi - lo < 2**32): lo + (r32 * span) >> 32."""
    span = hi - lo + 1
    assert 0 < span <= (1 << 32)
    r32 = draws(seed, stream, index) >> np.uint64(32)
    with np.errstate(over="ignore"):
        v = (r32 * np.uint64(span)) >> np.uint64(32)
    return v.astype(np.int64) + lo


@dataclass(frozen=True)
class Config:
    """Shape of one synthetic workload.

    roads: ("fixed", R) or ("geom", mean, lo, hi)  -- roads per event
    hits:  ("uniform", lo, hi) or ("skewed", cap)  -- hits per layer per road
    shared_hits: probability that a road's first hit on a layer copies the
        coordinate of the previous road's first hit on that layer (test inputs
        that make roads of one event share hits).
    """
    name: str
    n_events: int
    roads: tuple
    hits: tuple
    shared_hits: float = 0.0
    description: str = ""


CONFIGS = {
    "small": Config("small", 100, ("fixed", 8), ("uniform", 1, 2),
                    description="100 events x 8 roads, 1-2 hits per layer"),
    "scaled": Config("scaled", 3000, ("fixed", 64), ("uniform", 1, 4),
                     description="3000 events x 64 roads, 1-4 hits per layer"),
    "uneven": Config("uneven", 10000, ("geom", 32, 1, 256), ("skewed", 8),
                     description="10000 events, roads geometric(mean 32) in "
                                 "[1,256], hits P(n)=2^-n capped at 8"),
    "stress": Config("stress", 200, ("fixed", 128), ("uniform", 8, 8),
                     description="200 events x 128 roads x 8 hits on each "
                                 "of 5 layers"),
}


@dataclass
class Batch:
    """One generated batch.

    words          uint32[W] packed stream
    event_offsets  int64[E+1] word offset of each event (last = W)
    roads          structured array, one record per road (the generator's own
                   description of what it encoded)
    """
    config: Config
    seed: int
    words: np.ndarray
    event_offsets: np.ndarray
    roads: np.ndarray
    n_fits: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_events(self) -> int:
        return len(self.event_offsets) - 1

    def event_slice(self, first: int, count: int) -> np.ndarray:
        """Words of events [first, first+count) (a valid stream on its own)."""
        a, b = self.event_offsets[first], self.event_offsets[first + count]
        return self.words[a:b]


ROAD_DTYPE = np.dtype([
    ("event", np.int64), ("road", np.int64), ("wedge", np.int64),
    ("barrel", np.int64), ("excl", np.int64), ("curv", np.int64),
    ("phi", np.int64), ("n", np.int64, (N_LAYERS,)),
    ("coords", np.int64, (N_LAYERS, MAX_HITS)),
])


def make_constants(seed: int = 0) -> dict:
    """The 360 constant sets (12 wedges x 6 barrels x 5 excluded layers).

    F, C: int16 [360, 3, 6] uniform in [-4096, 4095]
    q, k: int32 [360, 3]    uniform in [-65536, 65535]
    """
    n6 = N_SETS * 18
    n3 = N_SETS * 3
    F = uniform_int(seed, _S_F, np.arange(n6), -4096, 4095).astype(np.int16)
    C = uniform_int(seed, _S_C, np.arange(n6), -4096, 4095).astype(np.int16)
    q = uniform_int(seed, _S_Q, np.arange(n3), -65536, 65535).astype(np.int32)
    k = uniform_int(seed, _S_K, np.arange(n3), -65536, 65535).astype(np.int32)
    return {"F": F.reshape(N_SETS, 3, 6), "q": q.reshape(N_SETS, 3),
            "C": C.reshape(N_SETS, 3, 6), "k": k.reshape(N_SETS, 3)}


def _roads_per_event(cfg: Config, seed: int) -> np.ndarray:
    E = cfg.n_events
    kind = cfg.roads[0]
    if kind == "fixed":
        return np.full(E, cfg.roads[1], dtype=np.int64)
    if kind == "geom":
        mean, lo, hi = cfg.roads[1:]
        assert mean == 32 and lo == 1
        # Bernoulli trials with success probability 1/32: each 64-bit draw
        # gives 12 five-bit trials; success = a zero five-bit field.  The count
        # is 1 + failures before the first success, clipped to `hi`.
        per_ev = (hi + 11) // 12
        r = draws(seed, _S_NROADS, np.arange(E * per_ev)).reshape(E, per_ev)
        shifts = (np.arange(12, dtype=np.uint64) * np.uint64(5))
        fields = (r[:, :, None] >> shifts[None, None, :]) & np.uint64(31)
        succ = (fields == 0).reshape(E, per_ev * 12)
        first = np.where(succ.any(axis=1), succ.argmax(axis=1), per_ev * 12)
        return np.minimum(1 + first, hi).astype(np.int64)
    raise ValueError(kind)


def _hits_per_layer(cfg: Config, seed: int, n_roads: int) -> np.ndarray:
    idx = np.arange(n_roads * N_LAYERS)
    kind = cfg.hits[0]
    if kind == "uniform":
        lo, hi = cfg.hits[1:]
        n = uniform_int(seed, _S_NHITS, idx, lo, hi)
    elif kind == "skewed":
        cap = cfg.hits[1]
        # n = 1 + number of trailing one bits of a draw, capped:
        # P(n) = 2^-n for n < cap, P(cap) = 2^-(cap-1).
        r = draws(seed, _S_NHITS, idx)
        n = np.ones(len(idx), dtype=np.int64)
        alive = np.ones(len(idx), dtype=bool)
        for b in range(cap - 1):
            bit = ((r >> np.uint64(b)) & np.uint64(1)).astype(bool)
            alive &= bit
            n += alive
    else:
        raise ValueError(kind)
    return n.reshape(n_roads, N_LAYERS)


def make_batch(cfg: Config | str, seed: int = 0, n_events: int | None = None) -> Batch:
    """Generate one batch of `cfg` (optionally with a different event count)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if n_events is not None:
        cfg = Config(cfg.name, n_events, cfg.roads, cfg.hits, cfg.shared_hits,
                     cfg.description)
    rpe = _roads_per_event(cfg, seed)
    R = int(rpe.sum())
    ev_of_road = np.repeat(np.arange(cfg.n_events), rpe)
    first_road = np.concatenate([[0], np.cumsum(rpe)[:-1]])
    road_in_ev = np.arange(R) - np.repeat(first_road, rpe)

    g = np.arange(R)
    wedge = uniform_int(seed, _S_WEDGE, g, 0, N_WEDGES - 1)
    barrel = uniform_int(seed, _S_BARREL, g, 0, N_BARRELS - 1)
    excl = uniform_int(seed, _S_EXCL, g, 0, N_LAYERS - 1)
    curv = uniform_int(seed, _S_CURV, g, -32768, 32767)
    phi = uniform_int(seed, _S_PHI, g, -32768, 32767)
    nh = _hits_per_layer(cfg, seed, R)
    coords = uniform_int(seed, _S_COORD, np.arange(R * N_LAYERS * MAX_HITS),
                         0, 4095).reshape(R, N_LAYERS, MAX_HITS)
    if cfg.shared_hits > 0:
        thr = int(cfg.shared_hits * (1 << 32))
        share = (draws(seed, _S_SHARE, np.arange(R * N_LAYERS)) >> np.uint64(32)) \
            .astype(np.int64).reshape(R, N_LAYERS) < thr
        share &= (road_in_ev > 0)[:, None]
        prev = np.maximum(g - 1, 0)
        src = coords[prev, :, 0].copy()
        coords[:, :, 0] = np.where(share, src, coords[:, :, 0])

    # --- emission order of the hit words inside each road -----------------
    # hits listed in (road, layer, d) order, then each road's hits are sorted
    # by a random key; the d-th emitted hit of layer l carries coords[., l, d].
    slot = np.arange(MAX_HITS)
    valid = slot[None, None, :] < nh[:, :, None]                    # R,5,8
    h_road, h_layer, h_slot = np.nonzero(valid)
    H = len(h_road)
    key = draws(seed, _S_ORDER, (h_road * N_LAYERS + h_layer) * MAX_HITS + h_slot)
    order = np.lexsort((key, h_road))                 # emission order
    e_road, e_layer = h_road[order], h_layer[order]
    # rank of each emitted hit among the same (road, layer), in emission order
    pos = np.arange(H)
    grp = np.lexsort((pos, e_layer, e_road))
    gr, gl = e_road[grp], e_layer[grp]
    start = np.ones(H, dtype=bool)
    start[1:] = (gr[1:] != gr[:-1]) | (gl[1:] != gl[:-1])
    run_id = np.cumsum(start) - 1
    run_start = np.nonzero(start)[0]
    rank_sorted = np.arange(H) - run_start[run_id]
    e_rank = np.empty(H, dtype=np.int64)
    e_rank[grp] = rank_sorted
    e_coord = coords[e_road, e_layer, e_rank]

    # --- word stream ----------------------------------------------------------
    hits_per_road = nh.sum(axis=1)
    road_len = 3 + hits_per_road
    road_off = np.concatenate([[0], np.cumsum(road_len)])
    W = int(road_off[-1])
    words = np.zeros(W, dtype=np.uint32)
    base = road_off[:-1]
    words[base] = ((7 << 27) | wedge | (barrel << 4) | (excl << 7)).astype(np.uint32)
    words[base + 1] = ((5 << 27) | (curv & 0xFFFF)).astype(np.uint32)
    words[base + 2] = ((6 << 27) | (phi & 0xFFFF)).astype(np.uint32)
    hit_first = np.concatenate([[0], np.cumsum(hits_per_road)[:-1]])
    hit_pos = base[e_road] + 3 + (np.arange(H) - hit_first[e_road])
    words[hit_pos] = ((e_layer << 27) | e_coord).astype(np.uint32)
    last = road_off[1:] - 1
    words[last] |= np.uint32(1 << 30)
    last_of_event = last[first_road + rpe - 1]
    words[last_of_event] |= np.uint32(1 << 31)
    event_offsets = np.concatenate([[0], road_off[first_road + rpe]]).astype(np.int64)

    roads = np.zeros(R, dtype=ROAD_DTYPE)
    roads["event"], roads["road"] = ev_of_road, road_in_ev
    roads["wedge"], roads["barrel"], roads["excl"] = wedge, barrel, excl
    roads["curv"], roads["phi"], roads["n"] = curv, phi, nh
    roads["coords"] = np.where(valid, coords, 0)
    n_fits = int(np.prod(nh, axis=1).sum())
    return Batch(cfg, seed, words, event_offsets, roads, n_fits)


_S_REQ = 30


def request_sizes(seed: int, n_requests: int, max_events: int = 512) -> np.ndarray:
    """Event counts of serving requests, spread evenly over octaves: octave k
    uniform in 0..log2(max_events) - 1, then a count uniform in [2^k, 2^(k+1))
    (a log-uniform law on [1, max_events) in integer arithmetic)."""
    n_oct = max(1, int(max_events).bit_length() - 1)
    i = np.arange(n_requests)
    k = uniform_int(seed, _S_REQ, 2 * i, 0, n_oct - 1)
    lo = np.left_shift(1, k)
    off = (draws(seed, _S_REQ, 2 * i + 1) >> np.uint64(32)).astype(np.int64)
    return (lo + (off * lo) // (1 << 32)).astype(np.int64)


def encode_roads(events) -> np.ndarray:
    """Encode hand-written events into a word stream.

    `events` is a list of events; an event is a list of roads; a road is a
    dict with keys wedge, barrel, excl, curv, phi and hits: a list of
    (layer, coordinate) pairs in emission order.
    """
    out = []
    for ev in events:
        for ri, rd in enumerate(ev):
            w = [(7 << 27) | rd["wedge"] | (rd["barrel"] << 4) | (rd["excl"] << 7),
                 (5 << 27) | (rd["curv"] & 0xFFFF),
                 (6 << 27) | (rd["phi"] & 0xFFFF)]
            w += [(layer << 27) | c for layer, c in rd["hits"]]
            w[-1] |= 1 << 30
            if ri == len(ev) - 1:
                w[-1] |= 1 << 31
            out += w
    return np.array(out, dtype=np.uint32)
