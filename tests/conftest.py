import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def consts():
    from paper_1312_0917_gb300 import synth
    return synth.make_constants(0)


@pytest.fixture(scope="session")
def cuts():
    with open(os.path.join(GOLDEN, "chi2_cuts.json")) as f:
        return {k: v["cut"] for k, v in json.load(f).items()}


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def zero_consts():
    from paper_1312_0917_gb300 import synth
    n = synth.N_SETS
    return {"F": np.zeros((n, 3, 6), np.int16), "q": np.zeros((n, 3), np.int32),
            "C": np.zeros((n, 3, 6), np.int16), "k": np.zeros((n, 3), np.int32)}


def set_index(wedge, barrel, excl):
    return (wedge * 6 + barrel) * 5 + excl
