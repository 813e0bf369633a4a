"""Writes the stored oracle values of tests/golden/ (run: python tests/golden/make_golden.py).

Only the FP64 oracle (oracle/gw_oracle.py) and the seeded input generator are called. The paper
prints no worked numbers that synthetic inputs could reproduce, so these fixtures freeze the
oracle's own results on the brute-force-size system. Any later change to the oracle's arithmetic
then shows up in test_golden.py and needs its own justification.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import gw_oracle as O                       # noqa: E402
from paper_2011_01400_gb300.synth import make_system   # noqa: E402

# (config, seed, head_wings): the head_wings = 0 case is also reachable by the explicit-loop
# brute-force tier (oracle/brute.py), which has no q = 0 head/wings treatment
CASES = [("tiny", 1, 1), ("tiny", 4, 0)]


def golden(cfg, seed, hw):
    s = make_system(cfg, seed=seed, head_wings=hw)
    r = O.g0w0(s)
    return dict(
        config=cfg, seed=seed, head_wings=hw,
        source="oracle/gw_oracle.py g0w0 (FP64): chi0 -> eps~ -> W^c -> Sigma_c -> two-pole QP",
        mu=float(r["mu"]),
        omega=[float(x) for x in r["omega"]],
        sigma_re=r["sigma"].real.round(15).tolist(),
        sigma_im=r["sigma"].imag.round(15).tolist(),
        e_qp=r["e_qp"].tolist(),
        gap=float(r["gap"]),
    )


def main():
    for cfg, seed, hw in CASES:
        path = os.path.join(HERE, f"oracle_{cfg}_seed{seed}_hw{hw}_g0w0.json")
        with open(path, "w") as f:
            json.dump(golden(cfg, seed, hw), f, indent=1)
        print("wrote", path)


if __name__ == "__main__":
    main()
