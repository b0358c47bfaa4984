"""Writes tests/golden/exact_refs.json from oracle.exact only (brute force for 4x4,
row transfer matrix for 6x6).  Run from the repository root:

    python tests/golden/make_exact_refs.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402

TEMPS = (1.5, 2.0, 2.269185, 3.5)


def main():
    out = {"source": "oracle.exact: enumerate_averages(4, T), transfer_averages(6, T)",
           "4x4": {}, "6x6": {}}
    for T in TEMPS:
        out["4x4"][repr(T)] = exact.enumerate_averages(4, T)
        out["6x6"][repr(T)] = exact.transfer_averages(6, T)
    _, _, g = exact.density_of_states(6)
    out["6x6_total_states"] = float(g.sum())
    with open(os.path.join(HERE, "exact_refs.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
