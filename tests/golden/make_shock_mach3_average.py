"""Writes shock_mach3_average.txt: the FP64 oracle's ensemble of time-averaged profiles of the
Mach-3 argon shock (Sec. 4.1; 100 cells over [-25, 25] upstream mean free paths, omega 0.81,
~200 particles per upstream cell, CFL 0.5), 500 steps, averages over the states after step 100,
K = 128 runs with seeds 1000..1127.  Per cell: mean and single-run standard deviation (ddof 1)
of density, x-velocity and temperature of the averaged state.  Calls only the oracle.

    python tests/golden/make_shock_mach3_average.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))                 # tests/
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))  # repository root

SEEDS = tuple(range(1000, 1128))
OUT = os.path.join(HERE, "shock_mach3_average.txt")


def main():
    import stat_util as S
    ens = S.oracle_ensemble("fp64", SEEDS)
    table = np.stack([c for k in S.QUANTITIES for c in ens[k][:2]], axis=1)
    hdr = ("Time-averaged profiles of the Mach-3 argon shock (Sec. 4.1), FP64 oracle ensemble.\n"
           "Problem: 100 cells over [-25, 25] upstream mean free paths, omega 0.81, ~200 particles per upstream cell,\n"
           f"CFL 0.5, {S.STEPS} steps, averages over the states after step {S.AVG_START};\n"
           f"K = {len(SEEDS)} runs, seeds {SEEDS[0]}..{SEEDS[-1]}; written by tests/golden/make_shock_mach3_average.py.\n"
           "Columns per cell: mean_rho sd_rho mean_u sd_u mean_T sd_T (sd = single-run standard deviation, ddof 1)")
    np.savetxt(OUT, table, fmt="%.10e", header=hdr)


if __name__ == "__main__":
    main()
