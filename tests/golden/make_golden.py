"""Writes the stored expected values under tests/golden/ from the FP64
oracle (oracle/) alone.  The paper prints no worked example (only the
constants of Eq. 3), so every stored value here is the oracle's; a change
to one of these files is a change to the oracle's arithmetic and names the
passage that justifies it.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle  # noqa: E402

# the 64-element binary: recipe of the initial state, Eqs. 4-6 parameters
BINARY_64 = dict(n_donor=40, n_accretor=24, q=0.5, f_donor=0.8, f_accretor=0.5, sigma_v=1e-3,
                 seed=11, stream=0)
PARAMS_64 = dict(G=1.0, eps=0.01, beta=0.5, dt=1e-3)
STEPS_64 = 10


def _fmt(v):
    return repr(float(v))


def write_roche():
    lines = ["# Eq. 3 Roche-lobe radius r_L(q) with the printed coefficient 0.69 and",
             "# Eggleton's 0.6, and the L1 point of Eq. 2 (Kopal's normalised potential,",
             "# star 1 at the origin, star 2 at x = 1, q = m_2 / m_1).",
             "# Written by tests/golden/make_golden.py from the FP64 oracle.",
             "# q  r_L(q; 0.69)  r_L(q; 0.6)  x_L1(q)"]
    for q in (0.1, 0.2, 0.3, 0.5, 1.0, 2.0, 5.0):
        lines.append(" ".join([_fmt(q), _fmt(oracle.roche_rL(q, 0.69)),
                               _fmt(oracle.roche_rL(q, 0.6)),
                               _fmt(oracle.roche_L1(q))]))
    open(os.path.join(HERE, "roche.txt"), "w").write("\n".join(lines) + "\n")


def write_binary_64():
    x, v, m, R, g = oracle.make_ic(BINARY_64["n_donor"], BINARY_64["n_accretor"], BINARY_64["q"],
                                   f_donor=BINARY_64["f_donor"],
                                   f_accretor=BINARY_64["f_accretor"],
                                   sigma_v=BINARY_64["sigma_v"], seed=BINARY_64["seed"],
                                   stream=BINARY_64["stream"])
    p = PARAMS_64
    a = oracle.forces(x, v, m, R, g, G=p["G"], eps=p["eps"], beta=p["beta"])
    rx, rv, ra = oracle.run(x, v, m, R, g, G=p["G"], eps=p["eps"], beta=p["beta"], dt=p["dt"],
                            nsteps=STEPS_64, n_donor=BINARY_64["n_donor"],
                            grow_f0=BINARY_64["f_donor"])
    head = ["# 64-element binary: " + " ".join(f"{k}={v}" for k, v in BINARY_64.items()),
            "# parameters: " + " ".join(f"{k}={v}" for k, v in PARAMS_64.items()) +
            f" steps={STEPS_64} (no donor growth)",
            "# Eqs. 4-6 accelerations at the initial state (a0), then the kick-drift-kick",
            "# state after the steps (x, v, a); one element per line, in particle order.",
            "# Written by tests/golden/make_golden.py from the FP64 oracle.",
            "# a0x a0y a0z  x y z  vx vy vz  ax ay az"]
    rows = [" ".join(_fmt(t) for t in (*a[i], *rx[i], *rv[i], *ra[i])) for i in range(len(x))]
    open(os.path.join(HERE, "binary_64.txt"), "w").write("\n".join(head + rows) + "\n")


if __name__ == "__main__":
    oracle.build()
    write_roche()
    write_binary_64()
    print("wrote", os.path.join(HERE, "roche.txt"), os.path.join(HERE, "binary_64.txt"))
