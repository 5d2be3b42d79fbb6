"""Hand-built batches with survivors derived by hand (no program computed them).

Every case uses constants under which chi2 has a closed form: C[s][0][0] =
4096 for every set s and all other constants zero, so a_0 = x_0 = the hit on
the lowest non-excluded layer, a_1 = a_2 = 0 and chi2 = x_0^2; F = 0, q = 0
gives p = (0, 0, 0).  All roads exclude layer 4, so x_0 is the layer-0 hit.

Each case is (name, events, cut, expected) where expected lists the
surviving (event, road, comb) triples in canonical order.
"""
import numpy as np

from paper_1312_0917_gb300 import synth

BIG_CUT = 1 << 40


def consts():
    n = synth.N_SETS
    c = {"F": np.zeros((n, 3, 6), np.int16), "q": np.zeros((n, 3), np.int32),
         "C": np.zeros((n, 3, 6), np.int16), "k": np.zeros((n, 3), np.int32)}
    c["C"][:, 0, 0] = 4096
    return c


def rd(coords_per_layer, excl=4, wedge=0, barrel=0):
    """coords_per_layer: five lists of coordinates (hit order)."""
    hits = [(l, c) for l in range(5) for c in coords_per_layer[l]]
    return {"wedge": wedge, "barrel": barrel, "excl": excl, "curv": 0, "phi": 0,
            "hits": hits}


CASES = [
    # Two combinations differing only in the excluded layer (4): same chi2,
    # four shared hits; the lower comb (0) wins.
    ("excluded_layer_pair",
     [[rd([[10], [20], [30], [40], [1, 2]])]], BIG_CUT, [(0, 0, 0)]),

    # Two roads with equal layer-0 hit -> equal chi2; they share layers 0,1,2.
    # The tie is broken by road index: road 0 wins.
    ("cross_road_tie",
     [[rd([[7], [8], [9], [100], [200]]), rd([[7], [8], [9], [101], [201]])]],
     BIG_CUT, [(0, 0, 0)]),

    # Chain A(chi2 1) - B(4) - C(9): A shares layers 1,2,3 with B; B shares
    # layers 2,3,4 with C; A and C share only layers 2,3.  B is dropped by A
    # and C is dropped by B although B itself is dropped (non-greedy rule).
    ("non_greedy_chain",
     [[rd([[1], [10], [20], [30], [99]]), rd([[2], [10], [20], [30], [98]]),
       rd([[3], [11], [20], [30], [98]])]], BIG_CUT, [(0, 0, 0)]),

    # Two shared hits are not enough: both survive.
    ("two_shared_hits",
     [[rd([[1], [10], [20], [31], [99]]), rd([[2], [10], [20], [30], [98]])]],
     BIG_CUT, [(0, 0, 0), (0, 1, 0)]),

    # The cut: chi2 = 3^2 = 9 > 8 fails, chi2 = 2^2 = 4 passes; no sharing.
    ("cut_inclusive",
     [[rd([[3], [10], [20], [30], [40]]), rd([[2], [11], [21], [31], [41]]),
       rd([[1], [12], [22], [32], [42]])]], 4, [(0, 1, 0), (0, 2, 0)]),

    # Equal coordinates inside one layer: hits 0 and 1 of layer 0 are both 5,
    # so combs 0 and 1 share all five hits and have equal chi2: comb 0 wins.
    # Comb 2 (layer-0 hit 6, chi2 36) shares layers 1..4 with comb 0: dropped.
    ("duplicate_coordinate_in_layer",
     [[rd([[5, 5, 6], [10], [20], [30], [40]])]], BIG_CUT, [(0, 0, 0)]),

    # A road with an empty layer has no combinations; events are independent
    # (the same road in event 1 is not dropped by event 0's).
    ("empty_layer_and_event_independence",
     [[rd([[1], [2], [], [4], [5]]), rd([[1], [10], [20], [30], [40]])],
      [rd([[1], [10], [20], [30], [40]])]], BIG_CUT, [(0, 1, 0), (1, 0, 0)]),

    # One road, 2x2 on layers 0 and 1: combs (d0,d1) = 0:(0,0) 1:(1,0)
    # 2:(0,1) 3:(1,1).  Layer-0 hits 3, 1 -> chi2 9, 1, 9, 1.  Every pair of
    # combinations shares layers 2,3,4, so only the lowest key survives:
    # chi2 1 at combs 1 and 3 -> comb 1.
    ("single_road_grid",
     [[rd([[3, 1], [50, 60], [20], [30], [40]])]], BIG_CUT, [(0, 0, 1)]),
]


def case_words(events):
    return synth.encode_roads(events)
