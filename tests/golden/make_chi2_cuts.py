"""Write tests/golden/chi2_cuts.json: the chi-square cut of every workload.

The cut of a workload is the nearest-rank 90th percentile of the chi-square of
every combination (before any cut) of that workload's seed-0 batch:
T = sorted(chi2)[ceil(0.9 N) - 1].  The serving workload uses the cut of the
"scaled" workload, whose events it replays.

Only the seeded generator (inputs) and the CPU oracle (chi-square values) are
called here; nothing comes from the CUDA path.

    python tests/golden/make_chi2_cuts.py [--only small,scaled]
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1312_0917_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chi2_cuts.json")


def nearest_rank_90(chi: np.ndarray) -> int:
    n = len(chi)
    rank = (9 * n + 9) // 10          # ceil(0.9 n) with integers only
    return int(np.partition(chi, rank - 1)[rank - 1])


def cut_for(name: str, chunk_events: int = 20) -> dict:
    b = synth.make_batch(name, seed=0)
    consts = synth.make_constants(0)
    parts = []
    for e0 in range(0, b.n_events, chunk_events):
        cnt = min(chunk_events, b.n_events - e0)
        rc, chi = oracle.chi2_all(b.event_slice(e0, cnt), consts)
        assert rc == 0, rc
        parts.append(chi)
    chi = np.concatenate(parts)
    assert len(chi) == b.n_fits
    return {"cut": nearest_rank_90(chi), "n_fits": int(len(chi)),
            "n_events": b.n_events, "n_words": int(len(b.words))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="small,scaled,uneven,stress")
    args = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in args.only.split(","):
        data[name] = cut_for(name)
        print(name, data[name], flush=True)
    data["serving"] = dict(data["scaled"], source="scaled")
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
