"""Writes the oracle regression fixtures of this directory.  Calls only the oracle and the seeded
input generators; rerun it only for a change of the oracle's arithmetic that cites the passage of
the paper (or the documented reading of it) that justifies the change.

config1_xyz.txt: X, Y, Z of the plain-method workload (one 3 mHz Galactic binary, A = 1e-22,
iota = 0.5, phi0 = 0, lambda = 1.0, beta = 0.3, psi = 0.4; static triangle of 2.5e9 m arms;
dt = 10 s, N = 65 536, order 25; TDI-2, summed delays) at 12 output indices."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

N, DT, T0, P = 65536, 10.0, 0.0, 25
IDX = np.array([0, 1, 2, 100, 4095, 4096, 32767, 32768, 50000, 65533, 65534, 65535])


def config1_xyz():
    src = synth.config1_source()
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, P)
    orb = synth.orbit_static(T0 - 2e5, T0 + N * DT + 2e5)
    o = oracle.Orbit(orb.t_knots, orb.pos, orb.delays)
    return oracle.response_at(P, 2, DT, T0, N, o, o, hp, hc, t0h, src.lam, src.beta, src.psi, IDX)


if __name__ == "__main__":
    x = config1_xyz()
    with open(os.path.join(HERE, "config1_xyz.txt"), "w") as f:
        f.write("# index X Y Z (plain-method workload, order 25, TDI-2; written by make_golden.py)\n")
        for k, i in enumerate(IDX):
            f.write("%d %.17e %.17e %.17e\n" % (i, x[0, k], x[1, k], x[2, k]))
