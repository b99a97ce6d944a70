"""The contact kernel's two layouts (Eqs. 5/6): one thread per element, or
three threads per element with one z-plane of the 27 neighbour cells each.

Both take each plane's contributions in the same order and add the three
plane sums in plane order, so they must give the same bits: the forces of a
state, a whole trajectory (whose contact decisions feed back into the state),
a batch of independent systems, and a run that switches layout half-way.
The three-lane forces are also checked against the FP64 oracle directly, and
the FP64 force path and the energy diagnostic (which always run one thread
per element) against the oracle with three lanes selected.
"""
import numpy as np
import pytest

import synth
from nbtest import oracle_ic, rms_rel, workload_kwargs

pytestmark = pytest.mark.gpu

BINARY = dict(n_donor=6000, n_accretor=2500, q=0.4, f_donor=0.9, f_accretor=0.5,
              sigma_v=1e-3, seed=4, stream=0)
BINARY_P = dict(eps=0.005, dt=5e-4, beta=0.5)


@pytest.fixture(scope="module")
def nbm():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _make(nbm, desc, params, **kw):
    return nbm.System(nbm.nb_desc_default(**desc), nbm.nb_params_default(**params), **kw)


def test_lanes_are_validated(nbm):
    with _make(nbm, BINARY, BINARY_P) as s:
        assert s.contact_lanes() == 0  # automatic until selected or tuned
        for bad in (2, 4, -1):
            with pytest.raises(nbm.NbError) as ei:
                s.set_contact_lanes(bad)
            assert ei.value.status == nbm.NB_EINVAL
        s.set_contact_lanes(3)
        assert s.contact_lanes() == 3
        s.set_contact_lanes(1)
        assert s.contact_lanes() == 1
        s.set_contact_lanes(0)
        assert s.contact_lanes() == 0


def test_three_lanes_match_oracle(nbm, orc):
    p = dict(BINARY_P, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    with _make(nbm, BINARY, BINARY_P) as s:
        s.set_contact_lanes(3)
        a = s.forces()
    ox, ov, om, oR, og = oracle_ic(orc, BINARY, p)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=p["eps"], beta=p["beta"])
    assert rms_rel(a, ref) <= 1e-5


def test_layouts_bitwise_same_forces_and_trajectory(nbm):
    """Forces of the initial state, 60 steps (graph-replayed), and a run that
    changes layout every 20 steps: the same bits throughout, and the same as
    the automatic choice."""
    res = {}
    for lanes in (1, 3, 0, "switch"):
        with _make(nbm, BINARY, BINARY_P) as s:
            s.set_contact_lanes(1 if lanes == "switch" else lanes)
            a0 = s.forces()
            for k in range(3):
                if lanes == "switch":
                    s.set_contact_lanes(3 if k % 2 == 0 else 1)
                s.step(20)
            s.sync()
            xv, a, meta = s.get_state()
            res[lanes] = (a0, xv, a, s.forces())
    for key in (3, 0, "switch"):
        for u, w in zip(res[1], res[key]):
            assert np.array_equal(u, w), key


def test_layouts_bitwise_in_a_batch(nbm):
    """A batch of small and large systems (few and many candidates per
    element): the same bits with either layout, and each system's forces
    the same as the system alone."""
    systems = synth.sweep_systems(12, seed=3, nmin=512, nmax=20000)
    descs = [nbm.nb_desc_default(**x) for x in systems]
    params = [nbm.nb_params_default(**BINARY_P) for _ in systems]
    out = {}
    for lanes in (1, 3):
        with nbm.Batch(descs, params) as b:
            b.set_contact_lanes(lanes)
            b.step(15)
            b.sync()
            out[lanes] = [b.forces(k) for k in range(len(systems))]
    for u, w in zip(out[1], out[3]):
        assert np.array_equal(u, w)
    with nbm.System(descs[5], params[5]) as s:
        s.set_contact_lanes(3)
        s.step(15)
        s.sync()
        assert np.array_equal(s.forces(), out[1][5])


def test_growing_donor_full_size_with_three_lanes(nbm, orc):
    """The 65,536-element binary with the growing donor, 200 steps with three
    lanes against the same with one: the same state bit for bit, and its
    accelerations against the oracle on sampled rows."""
    desc, params = workload_kwargs("binary_64k")
    states = {}
    for lanes in (1, 3):
        with _make(nbm, desc, params) as s:
            s.set_contact_lanes(lanes)
            s.step(200)
            s.sync()
            xv, _, meta = s.get_state()
            states[lanes] = (xv, s.forces(), meta.step)
    assert np.array_equal(states[1][0], states[3][0])
    assert np.array_equal(states[1][1], states[3][1])
    xv, a, k = states[3]
    n, nd = len(xv), desc["n_donor"]
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    R = np.array(oR)
    R[:nd] *= orc.donor_scale(k, desc["f_donor"], desc["expand_rate"], desc["expand_steps"])
    rows = np.unique(np.concatenate([[0, nd - 1, nd, n - 1],
                                     (synth.u01(9, 1, 256) * n).astype(np.int64)]))
    ref = orc.forces_rows(rows, xv[:, :3], xv[:, 3:], om, R, og, G=1.0, eps=params["eps"],
                          beta=params["beta"])
    assert rms_rel(a[rows], ref) <= 1e-6


def test_fp64_path_and_energy_ignore_the_layout(nbm, orc):
    """With three lanes selected, the FP64 force path and the energy
    diagnostic (one thread per element, FP64 contact magnitudes) still match
    the oracle, and give the same bits as with one lane."""
    p = dict(BINARY_P, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    ox, ov, om, oR, og = oracle_ic(orc, BINARY, p)
    got = {}
    for lanes in (1, 3):
        with _make(nbm, BINARY, dict(BINARY_P, force_prec=64)) as s:
            s.set_contact_lanes(lanes)
            a = s.forces()
            d = s.diagnostics()
        got[lanes] = (a, d["e_rep"], d["e_grav"])
    assert np.array_equal(got[1][0], got[3][0])
    assert got[1][1] == got[3][1] and got[1][2] == got[3][2]
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=p["eps"], beta=p["beta"])
    assert rms_rel(got[3][0], ref) <= 1e-12
    od = orc.diagnostics(ox, ov, om, oR, og, G=1.0, eps=p["eps"], n_donor=BINARY["n_donor"])
    assert got[3][1] == pytest.approx(od["E_rep"], rel=1e-10)


def test_tuner_picks_a_layout_and_keeps_the_bits(nbm):
    """nb_autotune times both contact layouts and selects one (1 or 3, no
    longer automatic); the forces are the same bits as before tuning with
    the same pair variant, and the batch tuner does the same."""
    with _make(nbm, BINARY, BINARY_P) as s:
        s.set_contact_lanes(1)
        tuned = s.autotune(1)
        lanes = s.contact_lanes()
        assert lanes in (1, 3)
        a_tuned = s.forces()
        s.set_contact_lanes(4 - lanes)  # the other layout
        assert np.array_equal(s.forces(), a_tuned)
    with _make(nbm, BINARY, BINARY_P) as s:
        s.set_pair_cfg(*[tuned[k] for k in ("tile", "i_per_thread", "threads", "min_blocks",
                                            "nr_slots", "i_packed", "shared_rcp", "symmetric")])
        assert np.array_equal(s.forces(), a_tuned)
    systems = synth.sweep_systems(6, seed=5, nmin=1024, nmax=8192)
    with nbm.Batch([nbm.nb_desc_default(**x) for x in systems],
                   [nbm.nb_params_default(**BINARY_P) for _ in systems]) as b:
        b.autotune(1)
        assert b.contact_lanes() in (1, 3)
