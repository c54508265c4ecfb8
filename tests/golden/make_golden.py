"""Writes the stored expected values under tests/golden/ by calling only the CPU oracle.

    python tests/golden/make_golden.py

pcpd_L1024_S64.txt: the L=1024, 64-sample, d=0.5, p=0.15, seed-1 fully-occupied decay run
over 2000 MCS: for each of the 32 log-spaced record times, the MCS time, the sub-step
ceil(t*L/K) and the total occupation count (R7-R9 of the design notes).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1301_6082_gb300.workloads import SMALL_L1024, log_times  # noqa: E402


def main():
    w = SMALL_L1024
    L, S = w["L"], w["S"]
    d, p = w["runs"][0]
    ts = log_times(w["mcs"], w["n_rec"])
    sub = [O.substep_of_time(L, t) for t in ts]
    st = O.init_state(L, S, w["init"], w["seed"])
    tot, _, _ = O.run(st, p, d, w["seed"], 0, sub[-1], sub)
    with open(os.path.join(HERE, "pcpd_L1024_S64.txt"), "w") as f:
        f.write("# oracle output: L=1024 S=64 d=0.5 p=0.15 seed=1 full start; written by make_golden.py\n")
        f.write("# t_mcs substep total_occupied\n")
        for t, n, c in zip(ts, sub, tot):
            f.write(f"{t} {n} {int(c)}\n")


if __name__ == "__main__":
    main()
