"""Writes tests/golden/three_node.json: the exact stationary distribution of the
hand-built 3-node PBN (pbn_synth.three_node, p = 1/16) under both perturbation
readings of Sec. 2.2, by exact rational Gaussian elimination (oracle only).

The paper prints no worked numerical example; this network is hand-built so
that its probabilities (p = 1/16, selection 3/4 and 1/4) are exact in the
2^-32 quantisation the simulation uses, which makes the rational answer the
exact answer of the simulated chain as well.
"""
import json
import os
import sys
from fractions import Fraction

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
from oracle import exact_rational as er  # noqa: E402


def main():
    out = {"network": "pbn_synth.three_node(p=1/16)",
           "citation": "Sec. 2.1 (stationary distribution pi = pi P) and Sec. 2.2 (PBN with perturbations); "
                       "hand-built example, exact rational solve",
           "state_index": "s = v0 + 2 v1 + 4 v2"}
    for mode, name in ((0, "per_node"), (1, "global")):
        P = er.transition_matrix(3, er.three_node_functions(), Fraction(1, 16), mode)
        pi = er.stationary(P)
        out[name] = {"pi_num_den": [[x.numerator, x.denominator] for x in pi],
                     "pi": [float(x) for x in pi],
                     "p_v0_1": float(sum(pi[s] for s in range(8) if s & 1))}
    path = os.path.join(os.path.dirname(__file__), "three_node.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k]["p_v0_1"] for k in ("per_node", "global")}))


if __name__ == "__main__":
    main()
