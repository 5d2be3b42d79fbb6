"""Pins of the oracle's combine, fit, chi-square and cut (Sec. II).

Each check reduces the fixed-point fit to something fixed independently of
the oracle's own code: constants that are multiples of 4096 turn the fit into
an exact integer matrix product (numpy), unit constants turn it into a floor
division (numpy.floor_divide), a hand-built extreme case has a closed form,
and the combinations are enumerated by itertools.product.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_1312_0917_gb300 import synth
from conftest import GOLDEN, zero_consts
from test_oracle_unpack import road


def x_vectors(fits, roads):
    """x = (hits of the four non-excluded layers ascending, curv, phi) per fit,
    built from the generator's record of each road."""
    key = {(int(r["event"]), int(r["road"])): r for r in roads}
    X = np.zeros((len(fits), 6), dtype=np.int64)
    S = np.zeros(len(fits), dtype=np.int64)
    for i, f in enumerate(fits):
        r = key[(int(f["event"]), int(f["road"]))]
        hits = [int(f["coord"][l]) for l in range(5) if l != r["excl"]]
        X[i] = hits + [int(r["curv"]), int(r["phi"])]
        S[i] = (r["wedge"] * 6 + r["barrel"]) * 5 + r["excl"]
    return X, S


@pytest.fixture(scope="module")
def batch():
    return synth.make_batch("small", seed=11)


def test_identity_rows_select_x_slots(orc, batch):
    """F rows 4096*e_j: p_i = x_j + q_i exactly (pins the order of x)."""
    for slots in [(0, 1, 2), (3, 4, 5), (5, 0, 3)]:
        c = zero_consts()
        for i, j in enumerate(slots):
            c["F"][:, i, j] = 4096
        c["q"][:] = [11, -7, 3]
        rc, fits = orc.fit_all(batch.words, c)
        assert rc == 0
        X, _ = x_vectors(fits, batch.roads)
        for i, j in enumerate(slots):
            assert np.array_equal(fits["p"][:, i], X[:, j] + c["q"][0, i])


def test_multiples_of_4096_are_exact_matmul(orc, batch):
    """F = 4096*G, C = 4096*H (G, H differ per set): p = G x + q and
    chi2 = |H x + k|^2 exactly -- an integer matrix product; also pins the
    constant-set index (wedge*6 + barrel)*5 + excluded layer."""
    rng = np.random.default_rng(7)
    G = rng.integers(-7, 8, size=(synth.N_SETS, 3, 6))
    H = rng.integers(-7, 8, size=(synth.N_SETS, 3, 6))
    c = zero_consts()
    c["F"][:] = 4096 * G
    c["C"][:] = 4096 * H
    c["q"][:] = rng.integers(-65536, 65536, size=(synth.N_SETS, 3))
    c["k"][:] = rng.integers(-65536, 65536, size=(synth.N_SETS, 3))
    rc, fits = orc.fit_all(batch.words, c)
    assert rc == 0
    X, S = x_vectors(fits, batch.roads)
    p = np.einsum("nij,nj->ni", G[S], X) + c["q"][S]
    a = np.einsum("nij,nj->ni", H[S], X) + c["k"][S]
    assert np.array_equal(fits["p"], p)
    assert np.array_equal(fits["chi2"], (a * a).sum(axis=1))


@pytest.mark.parametrize("scale", [1, 3, 2048, 4095])
def test_floor_division_on_negative_sums(orc, batch, scale):
    """F row = scale*e_j: p = floor(scale*x_j / 4096) + q (numpy floor_divide);
    curvature and phi are signed, so negative sums are exercised."""
    c = zero_consts()
    c["F"][:, 0, 4] = scale        # curvature
    c["F"][:, 1, 5] = scale        # phi
    c["F"][:, 2, 0] = scale        # first fitted hit (non-negative)
    c["C"][:, 0, 4] = -scale       # a_0 = floor(-scale*curv/4096)
    rc, fits = orc.fit_all(batch.words, c)
    X, _ = x_vectors(fits, batch.roads)
    assert (X[:, 4] < 0).any() and (X[:, 5] < 0).any()
    for i, j in enumerate((4, 5, 0)):
        assert np.array_equal(fits["p"][:, i], np.floor_divide(scale * X[:, j], 4096))
    a0 = np.floor_divide(-scale * X[:, 4], 4096)
    assert np.array_equal(fits["chi2"], a0 * a0)


def test_hand_floor_values(orc):
    """curv = -1 with F = 1: floor(-1/4096) = -1 (truncation would give 0);
    curv = -4096: exactly -1; curv = -4097: -2; phi = 4095: 0."""
    for curv, want in [(-1, -1), (-4096, -1), (-4097, -2), (4095, 0), (4096, 1)]:
        c = zero_consts()
        c["F"][:, 0, 4] = 1
        w = road([(l, 5) for l in range(5)], curv=curv, last_of_event=True)
        rc, fits = orc.fit_all(np.array(w, np.uint32), c)
        assert rc == 0 and len(fits) == 1 and fits["p"][0, 0] == want


def test_extreme_magnitudes_closed_form(orc):
    """All F = -4096, hits 4095, curv = phi = -32768:
    sum = -4096*(4*4095) + (-4096)*(-32768)*2 = 4096*49156 -> p = 49156 + q.
    All C = 4095, hits 4095, curv = phi = 32767, k = 65535:
    a = floor(4095*81914/4096) + 65535 = floor(81914 - 19.998...) + 65535
      = 81894 + 65535."""
    c = zero_consts()
    c["F"][:] = -4096
    c["q"][:] = [1, 2, 3]
    w = road([(l, 4095) for l in range(5)], curv=-32768, phi=-32768, last_of_event=True)
    rc, fits = orc.fit_all(np.array(w, np.uint32), c)
    assert list(fits["p"][0]) == [49157, 49158, 49159]
    c = zero_consts()
    c["C"][:] = 4095
    c["k"][:] = 65535
    w = road([(l, 4095) for l in range(5)], curv=32767, phi=32767, last_of_event=True)
    rc, fits = orc.fit_all(np.array(w, np.uint32), c)
    assert fits["chi2"][0] == 3 * (81894 + 65535) ** 2


def test_combinations_match_product_enumeration(orc):
    """comb runs 0..N-1 through itertools.product(d4, d3, d2, d1, d0):
    layer 0 varies fastest; N = product of the hits per layer."""
    b = synth.make_batch(synth.Config("c", 6, ("fixed", 5), ("uniform", 0, 3)), seed=2)
    rc, fits = orc.fit_all(b.words, synth.make_constants(0))
    assert rc == 0
    i = 0
    for r in b.roads:
        n = [int(v) for v in r["n"]]
        expect = []
        for d in itertools.product(*[range(n[l]) for l in (4, 3, 2, 1, 0)]):
            d = d[::-1]
            expect.append(tuple(int(r["coords"][l][d[l]]) for l in range(5)))
        N = int(np.prod(n))
        assert N == len(expect)
        got = fits[i:i + N]
        assert (got["event"] == r["event"]).all() and (got["road"] == r["road"]).all()
        assert list(got["comb"]) == list(range(N))
        assert [tuple(int(v) for v in g) for g in got["coord"]] == expect
        i += N
    assert i == len(fits)
    assert (b.roads["n"] == 0).any()         # empty layers were exercised


def test_rational_recomputation(orc, batch, consts):
    """floor(Fraction(sum F x, 4096)) + q for the generated constants."""
    from fractions import Fraction
    import math
    rc, fits = orc.fit_all(batch.words, consts)
    X, S = x_vectors(fits[:400], batch.roads)
    for n in range(400):
        s = S[n]
        for i in range(3):
            acc = sum(int(consts["F"][s, i, j]) * int(X[n, j]) for j in range(6))
            assert fits["p"][n, i] == math.floor(Fraction(acc, 4096)) + int(consts["q"][s, i])
        chi = 0
        for k in range(3):
            acc = sum(int(consts["C"][s, k, j]) * int(X[n, j]) for j in range(6))
            a = math.floor(Fraction(acc, 4096)) + int(consts["k"][s, k])
            chi += a * a
        assert fits["chi2"][n] == chi


def test_cut_is_inclusive(orc, batch, consts):
    rc, fits = orc.fit_all(batch.words, consts, cut=0)
    t = int(np.median(fits["chi2"]))
    rc, f2 = orc.fit_all(batch.words, consts, cut=t)
    assert np.array_equal(f2["pass"] == 1, f2["chi2"] <= t)
    rc, passing = orc.run(batch.words, consts, t, warrior=-1)
    assert np.array_equal(passing["comb"], f2["comb"][f2["chi2"] <= t])
    assert np.array_equal(passing["chi2"], f2["chi2"][f2["chi2"] <= t])


def test_stored_cut_is_nearest_rank_90th_percentile(orc, consts, cuts):
    """For the small workload: count(chi2 <= T) >= ceil(0.9 N) and
    count(chi2 <= T - 1) < ceil(0.9 N), checked by counting."""
    b = synth.make_batch("small", seed=0)
    rc, chi = orc.chi2_all(b.words, consts)
    T = cuts["small"]
    need = -(-9 * len(chi) // 10)
    assert (chi <= T).sum() >= need > (chi <= T - 1).sum()
    with open(os.path.join(GOLDEN, "chi2_cuts.json")) as f:
        meta = json.load(f)
    assert meta["small"]["n_fits"] == len(chi) == b.n_fits
