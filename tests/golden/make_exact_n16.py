"""Writes tests/golden/exact_n16.json: the exact steady-state probability of
the state of interest of pbn_synth.exact_config(16) under both perturbation
readings of Sec. 2.2, by FP64 power iteration (Sec. 2.1) with the oracle's
implicit product-measure step (oracle only; the 2^16 x 2^16 matrix is never
formed).  The probabilities are the quantised ones the simulation realises."""
import json
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
import pbn_synth as S  # noqa: E402
from oracle import exact as E  # noqa: E402


def compute():
    net, soi, cfg = S.exact_config(16)
    out = {"network": "pbn_synth.exact_config(16)",
           "citation": "Sec. 2.1 (limiting distribution of an ergodic DTMC by iterating pi P) and Sec. 2.2 "
                       "(PBN with perturbations); FP64 power iteration to an L1 change below 1e-14",
           "state_of_interest": {"nodes": [int(x) for x in soi.nodes], "values": [int(x) for x in soi.values]}}
    for mode, name in ((0, "per_node"), (1, "global")):
        pi, iters = E.stationary_implicit(net, mode)
        out[name] = {"prob": float(pi[E.soi_mask(net.n, soi)].sum()), "iterations": int(iters)}
    return out


def main():
    out = compute()
    with open(os.path.join(os.path.dirname(__file__), "exact_n16.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
