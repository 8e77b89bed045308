"""Pin of the inversion flop model used for the LU/inverse roofline.

The paper prints, per system, the time of one QMC step, the share of it spent
in the inversion (Table 3) and the inversion GFlop/s (Table 2).  Dividing
2 (N_up^3 + N_dn^3) flop by (share x step time) must reproduce the printed
GFlop/s; the alternatives 2/3 N^3 (LU only) and 8/3 N^3 do not.
"""
import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_2_3.json")


def test_inversion_is_two_n_cubed_per_spin_matrix():
    g = json.load(open(GOLD))
    nu, nd = np.array(g["n_up"], float), np.array(g["n_dn"], float)
    for coef, ok in ((2.0, True), (2.0 / 3.0, False), (8.0 / 3.0, False)):
        fits = []
        for cpu in ("core2", "sandy_bridge"):
            t = np.array(g[cpu]["step_s"]) * np.array(g[cpu]["inversion_share"])
            printed = np.array(g[cpu]["inversion_gflops"])
            ratio = coef * (nu ** 3 + nd ** 3) / t / 1e9 / printed
            fits.append(bool(np.all((ratio > 0.75) & (ratio < 1.33))))
        # the model must fit both processors; a wrong model misses on at least one
        assert all(fits) == ok, (coef, fits)
