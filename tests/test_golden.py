"""Stored expected values (tests/golden/, written from the FP64 oracle by
tests/golden/make_golden.py; the paper prints no worked example).

The oracle must keep reproducing them (a change to its arithmetic shows up
here first), and the library's host-side Roche-geometry functions (Eqs. 2,
3) match them without a GPU.  The GPU tests compare the CUDA path with the
same stored forces and trajectory.
"""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _golden_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def load_binary_64():
    """(description, parameters, steps, a0 (64,3), x, v, a after the steps)."""
    g = _golden_module()
    t = np.loadtxt(os.path.join(GOLDEN, "binary_64.txt"))
    return g.BINARY_64, g.PARAMS_64, g.STEPS_64, t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12]


def test_oracle_reproduces_roche_values(orc):
    t = np.loadtxt(os.path.join(GOLDEN, "roche.txt"))
    for q, rl69, rl6, xl1 in t:
        assert orc.roche_rL(q, 0.69) == pytest.approx(rl69, rel=1e-14)
        assert orc.roche_rL(q, 0.6) == pytest.approx(rl6, rel=1e-14)
        assert orc.roche_L1(q) == pytest.approx(xl1, abs=1e-14)


def test_library_host_roche_functions_match_the_stored_values():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody as nbm
    t = np.loadtxt(os.path.join(GOLDEN, "roche.txt"))
    for q, rl69, rl6, xl1 in t:
        assert nbm.nb_roche_rL(q, 0.69) == pytest.approx(rl69, rel=1e-14)
        assert nbm.nb_roche_rL(q, 0.6) == pytest.approx(rl6, rel=1e-14)
        assert nbm.nb_roche_L1(q) == pytest.approx(xl1, abs=1e-14)


def test_oracle_reproduces_binary_64(orc):
    desc, p, steps, a0, x, v, a = load_binary_64()
    ox, ov, om, oR, og = orc.make_ic(desc["n_donor"], desc["n_accretor"], desc["q"],
                                     f_donor=desc["f_donor"], f_accretor=desc["f_accretor"],
                                     sigma_v=desc["sigma_v"], seed=desc["seed"],
                                     stream=desc["stream"])
    ra0 = orc.forces(ox, ov, om, oR, og, G=p["G"], eps=p["eps"], beta=p["beta"])
    rx, rv, ra = orc.run(ox, ov, om, oR, og, G=p["G"], eps=p["eps"], beta=p["beta"], dt=p["dt"],
                         nsteps=steps, n_donor=desc["n_donor"], grow_f0=desc["f_donor"])
    for got, want in ((ra0, a0), (rx, x), (rv, v), (ra, a)):
        assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
    # the fixture exercises both terms: without the contact term (gamma = 0)
    # the start's accelerations would be far smaller
    grav = orc.forces(ox, ov, om, oR, np.zeros_like(og), G=p["G"], eps=p["eps"], beta=p["beta"])
    assert np.abs(a0 - grav).max() > 10.0 * np.abs(grav).max()
