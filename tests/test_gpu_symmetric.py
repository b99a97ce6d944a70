"""The pair term with each unordered pair evaluated once (both elements get
their share, Newton's third law) against the FP64 oracle, through the C ABI.

The symmetric layout splits a system into blocks of threads x i-per-thread
elements; these cases span several blocks, a ragged last block, blocks whose
elements carry different masses (the donor/accretor boundary inside a block,
per-element masses) and uniform blocks, with and without contacts.
Tolerances are those of the one-sided FP32 path (1e-5 RMS-relative per
step, 1e-4 on positions).
"""
import numpy as np
import pytest

import synth
from nbtest import oracle_ic, rms_rel, workload_kwargs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nbm():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _sym_variants():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return [c for c in nbody.nb_pair_cfg_variants() if c[7]]


ONE_SIDED = (128, 8, 128, 2, 0, 0, 6, 0)


def _make(nbm, desc, params, **kw):
    return nbm.System(nbm.nb_desc_default(**desc), nbm.nb_params_default(**params), **kw)


def _cloud_system(nbm, n, seed, contacts=True):
    x, v = synth.cloud(n, seed, radius=0.4, speed=0.2)
    st = synth.Stream(seed, 11)
    m = 0.5 + st.uniform(n)
    R = (0.01 + 0.01 * st.uniform(n)) if contacts else np.zeros(n)
    gam = (1.0 + st.uniform(n)) if contacts else np.zeros(n)
    desc = dict(n_donor=n // 2, n_accretor=n - n // 2, q=0.5)
    params = dict(eps=0.003, dt=1e-3, beta=0.35)
    s = _make(nbm, desc, params, xv_in=np.concatenate([x, v], 1),
              mrg_in=np.stack([m, R, gam], 1))
    return s, (x, v, m, R, gam)


BINARY = dict(n_donor=6000, n_accretor=2500, q=0.4, f_donor=0.9, f_accretor=0.5,
              sigma_v=1e-3, seed=3, stream=0)
BINARY_P = dict(eps=0.005, dt=5e-4, beta=0.5)


@pytest.mark.parametrize("cfg", _sym_variants())
@pytest.mark.parametrize("n,contacts", [(3000, True), (4097, False), (5120, True)])
def test_symmetric_forces_per_element_masses(nbm, orc, cfg, n, contacts):
    s, (x, v, m, R, gam) = _cloud_system(nbm, n, 40 + n, contacts)
    with s:
        s.set_pair_cfg(*cfg)
        a = s.forces()
    ref = orc.forces(x, v, m, R, gam, G=1.0, eps=0.003, beta=0.35)
    assert rms_rel(a, ref) <= 1e-5
    assert np.abs(a - ref).max() <= 5e-4 * np.abs(ref).max()


@pytest.mark.parametrize("cfg", _sym_variants())
def test_symmetric_forces_binary(nbm, orc, cfg):
    """Uniform-mass blocks of each star and one block holding both."""
    with _make(nbm, BINARY, BINARY_P) as s:
        s.set_pair_cfg(*cfg)
        a = s.forces()
        a_one = None
        s.set_pair_cfg(*ONE_SIDED)
        a_one = s.forces()
    p = dict(BINARY_P, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    ox, ov, om, oR, og = oracle_ic(orc, BINARY, p)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=p["eps"], beta=p["beta"])
    assert rms_rel(a, ref) <= 1e-5
    # the two FP32 orders of summation agree far inside the tolerance
    assert rms_rel(a, a_one) <= 2e-6


def test_symmetric_momentum_balance(nbm):
    """Gravity only: every evaluation hands equal and opposite forces to the
    two elements, so sum m a vanishes to FP32 rounding of the shares."""
    s, (x, v, m, R, gam) = _cloud_system(nbm, 6000, 77, contacts=False)
    with s:
        s.set_pair_cfg(*_sym_variants()[0])
        a = s.forces()
    p = (m[:, None] * a).sum(0)
    scale = np.abs(m[:, None] * a).sum(0)
    assert np.all(np.abs(p) <= 1e-6 * scale)


def test_symmetric_trajectory(nbm, orc):
    """100 steps of a 3,500-element binary with contacts and donor growth."""
    desc = dict(n_donor=2600, n_accretor=900, q=0.3, f_donor=0.9, f_accretor=0.5,
                expand_rate=1e-3, expand_steps=60, sigma_v=1e-3, seed=6, stream=0)
    params = dict(eps=0.005, dt=5e-4, beta=0.5)
    with _make(nbm, desc, params) as s:
        s.set_pair_cfg(*_sym_variants()[0])
        s.step(100)
        s.sync()
        xv, a, meta = s.get_state()
        assert meta.step == 100
    p = dict(params, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    ox, ov, om, oR, og = oracle_ic(orc, desc, p)
    rx, rv, ra = orc.run(ox, ov, om, oR, og, G=1.0, eps=0.005, beta=0.5, dt=5e-4, nsteps=100,
                         n_donor=2600, grow_f0=0.9, grow_rate=1e-3, grow_cap=60)
    assert np.abs(xv[:, :3] - rx).max() <= 1e-4
    assert np.sqrt(((xv[:, :3] - rx) ** 2).mean()) <= 1e-5


def test_symmetric_alone_vs_batch_bitwise(nbm):
    import torch
    systems = [
        (dict(n_donor=3000, n_accretor=1100, q=0.4, f_donor=0.9, f_accretor=0.5, sigma_v=1e-3,
              seed=1), dict(eps=0.005, dt=5e-4, beta=0.5)),
        (dict(n_donor=700, n_accretor=700, q=0.9, f_donor=0.7, f_accretor=0.6, sigma_v=2e-3,
              seed=2), dict(eps=0.008, dt=8e-4, beta=0.7)),
        (dict(n_donor=5000, n_accretor=2000, q=0.2, f_donor=0.95, f_accretor=0.4,
              expand_rate=1e-3, expand_steps=-1, sigma_v=1e-3, seed=3),
         dict(eps=0.004, dt=4e-4, beta=0.3)),
    ]
    cfg = _sym_variants()[0]
    descs = [nbm.nb_desc_default(**d) for d, _ in systems]
    params = [nbm.nb_params_default(**p) for _, p in systems]
    stream = torch.cuda.Stream()
    with nbm.Batch(descs, params, stream=stream) as b:
        b.set_pair_cfg(*cfg)
        b.step(5)
        b.step(5)
        b.sync()
        mixed = [b.get_state(s) for s in range(len(systems))]
    for s, (d, p) in enumerate(systems):
        with _make(nbm, d, p) as one:
            one.set_pair_cfg(*cfg)
            one.step(10)
            one.sync()
            xv, a, meta = one.get_state()
        assert np.array_equal(mixed[s][0], xv), f"system {s}: state differs"
        assert np.array_equal(mixed[s][1], a), f"system {s}: accelerations differ"


def test_symmetric_checkpoint_resume_bitwise(nbm):
    cfg = _sym_variants()[0]
    with _make(nbm, BINARY, BINARY_P) as s:
        s.set_pair_cfg(*cfg)
        s.step(4)
        s.sync()
        xv, a, meta = s.get_state()
        s.step(6)
        s.sync()
        ref = s.get_state()
    with _make(nbm, BINARY, BINARY_P) as r:
        r.set_pair_cfg(*cfg)
        r.set_state(xv, a, meta)
        r.step(6)
        r.sync()
        got = r.get_state()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("cfg", _sym_variants())
def test_symmetric_diagnostics_energy(nbm, orc, cfg):
    """The potential of the energy diagnostic: the rotating variants run it
    on their own symmetric items (each unordered pair once, fixed-point
    sums), the others as a one-sided pass; either way E_grav matches the
    oracle, and the forces of the step passes that follow are unchanged."""
    with _make(nbm, BINARY, BINARY_P) as s:
        s.set_pair_cfg(*cfg)
        a0 = s.forces()
        d = s.diagnostics()
        a = s.forces()
    p = dict(BINARY_P, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    ox, ov, om, oR, og = oracle_ic(orc, BINARY, p)
    od = orc.diagnostics(ox, ov, om, oR, og, G=1.0, eps=p["eps"], n_donor=BINARY["n_donor"])
    assert d["e_grav"] == pytest.approx(od["E_grav"], rel=1e-6)
    assert d["e_rep"] == pytest.approx(od["E_rep"], rel=1e-10)
    assert np.array_equal(a, a0)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=p["eps"], beta=p["beta"])
    assert rms_rel(a, ref) <= 1e-5


def test_symmetric_potential_mixed_masses_and_coincident_elements(nbm, orc):
    """Per-element masses (no uniform tile or block), two coincident elements
    (the pair contributes nothing) and several blocks: the symmetric
    potential pass's E_grav against the oracle's, for the default variant."""
    n = 5000
    x, v = synth.cloud(n, 77, radius=0.4, speed=0.2)
    x[4321] = x[17]  # coincident, in different blocks
    m = 0.5 + synth.u01(77, 3, n)
    desc = dict(n_donor=n // 2, n_accretor=n - n // 2, q=0.5)
    params = dict(eps=0.003, dt=1e-3, beta=0.35, flags=nbm.NB_GRAVITY_ONLY)
    mrg = np.stack([m, np.zeros(n), np.zeros(n)], 1)
    with _make(nbm, desc, params, xv_in=np.concatenate([x, v], 1), mrg_in=mrg) as s:
        assert s.pair_cfg()["symmetric"] == 3
        d = s.diagnostics()
    eg, _ = orc.potential(x, m, np.zeros(n), np.zeros(n), G=1.0, eps=0.003)
    assert d["e_grav"] == pytest.approx(float(np.sum(eg)), rel=1e-6)


@pytest.mark.parametrize("name,nrows", [("binary_64k", 256), ("binary_1m", 128)])
def test_symmetric_full_size_sampled(nbm, orc, name, nrows):
    """At the benchmark's sizes, in the symmetric launch shape the tuner
    picks there: sampled rows against the oracle."""
    desc, params = workload_kwargs(name)
    cfg = (256, 8, 128, 2, 0, 0, 0, 1)
    assert cfg in _sym_variants()
    with _make(nbm, desc, params) as s:
        s.set_pair_cfg(*cfg)
        a = s.forces()
        n = s.n
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    nd = desc["n_donor"]
    rows = np.unique(np.concatenate([
        [0, 1, 1023, 1024, nd - 1, nd, nd + 1, n - 1025, n - 1024, n - 1],
        (synth.u01(7, 9, nrows) * n).astype(np.int64)]))
    ref = orc.forces_rows(rows, ox, ov, om, oR, og, G=1.0, eps=params["eps"],
                          beta=params["beta"])
    assert rms_rel(a[rows], ref) <= 1e-5


@pytest.mark.parametrize("n", [1, 2, 3, 1023, 1024, 1025, 2047, 2048, 2049, 3071, 3073])
def test_symmetric_block_boundaries(nbm, orc, n):
    """Sizes around whole blocks of 1,024 (ragged last block, one element
    past a block, a single block), per-element masses and contacts."""
    s, (x, v, m, R, gam) = _cloud_system(nbm, n, 500 + n, contacts=True)
    with s:
        s.set_pair_cfg(256, 8, 128, 2, 0, 0, 2, 1)
        a = s.forces()
    if n == 1:
        assert np.all(a == 0.0)
        return
    ref = orc.forces(x, v, m, R, gam, G=1.0, eps=0.003, beta=0.35)
    assert rms_rel(a, ref) <= 1e-5
    assert np.abs(a - ref).max() <= 5e-4 * np.abs(ref).max()


def test_symmetric_tiny_and_large_systems_in_one_batch(nbm):
    """Systems of 1, 3, 257 and 5,000 elements with the symmetric kernel:
    each bitwise equal to itself alone."""
    import torch
    systems = [
        (dict(n_donor=1, n_accretor=0, q=0.5, f_donor=0.8, f_accretor=0.5, seed=21),
         dict(eps=0.01, dt=1e-3, beta=0.5)),
        (dict(n_donor=2, n_accretor=1, q=0.5, f_donor=0.8, f_accretor=0.5, seed=22),
         dict(eps=0.01, dt=1e-3, beta=0.5)),
        (dict(n_donor=200, n_accretor=57, q=0.6, f_donor=0.8, f_accretor=0.5, seed=23),
         dict(eps=0.006, dt=5e-4, beta=0.4)),
        (dict(n_donor=3600, n_accretor=1400, q=0.3, f_donor=0.9, f_accretor=0.5, seed=24),
         dict(eps=0.005, dt=5e-4, beta=0.5)),
    ]
    cfg = (256, 8, 128, 2, 0, 0, 2, 1)
    descs = [nbm.nb_desc_default(**d) for d, _ in systems]
    params = [nbm.nb_params_default(**p) for _, p in systems]
    with nbm.Batch(descs, params, stream=torch.cuda.Stream()) as b:
        b.set_pair_cfg(*cfg)
        b.step(4)
        b.sync()
        mixed = [b.get_state(s) for s in range(len(systems))]
    for s, (d, p) in enumerate(systems):
        with _make(nbm, d, p) as one:
            one.set_pair_cfg(*cfg)
            one.step(4)
            one.sync()
            xv, a, _ = one.get_state()
        assert np.array_equal(mixed[s][0], xv), f"system {s}: state differs"
        assert np.array_equal(mixed[s][1], a), f"system {s}: accelerations differ"


@pytest.mark.parametrize("name,nrows", [("binary_64k", 256), ("binary_1m", 128)])
def test_full_size_in_the_tuned_configuration(nbm, orc, name, nrows):
    """At the benchmark's sizes, in the pair configuration the tuner picks
    (the launch configuration the benchmark times): sampled rows against
    the oracle."""
    desc, params = workload_kwargs(name)
    with _make(nbm, desc, params) as s:
        best = s.autotune(2)
        a = s.forces()
        n = s.n
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    nd = desc["n_donor"]
    rows = np.unique(np.concatenate([
        [0, 1, 1023, 1024, nd - 1, nd, nd + 1, n - 1],
        (synth.u01(13, 9, nrows) * n).astype(np.int64)]))
    ref = orc.forces_rows(rows, ox, ov, om, oR, og, G=1.0, eps=params["eps"],
                          beta=params["beta"])
    assert rms_rel(a[rows], ref) <= 1e-5, f"tuned configuration {best}"


def test_energy_drift_long_run(nbm, orc):
    """1,000 elastic steps (beta = 1) of a 4,096-element binary on the
    default (symmetric) path: the total energy's drift stays within a small
    multiple of the FP64 oracle's own drift on the same problem (the two
    trajectories separate chaotically, so energies are compared in size,
    not value by value)."""
    desc = dict(n_donor=3072, n_accretor=1024, q=0.4, f_donor=0.85, f_accretor=0.5,
                sigma_v=1e-3, seed=9, stream=0)
    params = dict(eps=0.005, dt=2e-4, beta=1.0)
    nsteps = 1000
    with _make(nbm, desc, params) as s:
        d0 = s.diagnostics()
        s.step(nsteps)
        s.sync()
        d1 = s.diagnostics()
    p = dict(params, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    ox, ov, om, oR, og = oracle_ic(orc, desc, p)
    e0 = orc.diagnostics(ox, ov, om, oR, og, G=1.0, eps=0.005)["E_tot"]
    rx, rv, _ = orc.run(ox, ov, om, oR, og, G=1.0, eps=0.005, beta=1.0, dt=2e-4, nsteps=nsteps,
                        n_donor=3072)
    e1 = orc.diagnostics(rx, rv, om, oR, og, G=1.0, eps=0.005)["E_tot"]
    assert d0["e_tot"] == pytest.approx(e0, rel=1e-6)
    drift_gpu = abs(d1["e_tot"] - d0["e_tot"]) / abs(e0)
    drift_orc = abs(e1 - e0) / abs(e0)
    assert drift_gpu <= 3.0 * max(drift_orc, 1e-5), (drift_gpu, drift_orc)


def test_symmetric_plan_memory_is_linear_in_n(nbm, orc):
    """The symmetric kernel sums both sides of every pair into one fixed-point
    accumulator per element (no slot per (block, element)): a
    1,048,576-element system takes well under 1 GB of device memory in the
    default symmetric configuration and runs it with only 1.5 GB of the
    device left free; its forces match the oracle on sampled rows."""
    import torch
    desc, params = workload_kwargs("binary_1m")
    free, _ = torch.cuda.mem_get_info()
    leave = 1536 << 20
    if free < leave + (1 << 30):
        pytest.skip("not enough device memory to set the case up")
    hold = torch.empty(free - leave, dtype=torch.uint8, device="cuda")
    try:
        with _make(nbm, desc, params) as s:
            cfg = s.pair_cfg()
            a = s.forces()
            n = s.n
            dev_bytes = s.info.device_bytes
    finally:
        del hold
        torch.cuda.empty_cache()
    assert cfg["symmetric"] == 3
    assert dev_bytes < 1e9, dev_bytes
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    nd = desc["n_donor"]
    rows = np.unique(np.concatenate([[0, nd - 1, nd, n - 1],
                                     (synth.u01(5, 19, 96) * n).astype(np.int64)]))
    ref = orc.forces_rows(rows, ox, ov, om, oR, og, G=1.0, eps=params["eps"],
                          beta=params["beta"])
    assert rms_rel(a[rows], ref) <= 1e-5


def test_fixed_point_sums_are_order_independent(nbm):
    """The persistent CTAs claim work items in an order that varies from run
    to run; the fixed-point sums make every evaluation bit-for-bit the same
    (here: five evaluations of a 20,000-element system, several blocks and
    both-sided items per row)."""
    s, _ = _cloud_system(nbm, 20000, 91)
    with s:
        first = s.forces()
        for _ in range(4):
            assert np.array_equal(s.forces(), first)


@pytest.mark.parametrize("eps", [0.0, 1e-7])
def test_small_softening_runs_one_sided_items(nbm, orc, eps):
    """Softening too small for the fixed-point layout (eps = 0, and eps = 1e-7
    for a binary of extent ~1): the symmetric plan gives the system one-sided
    items summed into partial slots.  The forces still match the oracle, and
    the system gives the same bits alone and in a batch next to a system
    summed in fixed point; in that batch the potential pass runs both kinds
    of items in one launch and each system's E_grav matches the oracle's."""
    desc = dict(n_donor=2000, n_accretor=1000, q=0.5, f_donor=0.8, f_accretor=0.5,
                sigma_v=1e-3, seed=8, stream=0)
    params = dict(eps=eps, dt=5e-4, beta=0.5)
    with _make(nbm, desc, params) as s:
        assert s.pair_cfg()["symmetric"] == 3
        a = s.forces()
        s.step(3)
        s.sync()
        alone = s.get_state()
    p = dict(params, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    ox, ov, om, oR, og = oracle_ic(orc, desc, p)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=eps, beta=0.5)
    assert rms_rel(a, ref) <= 1e-5
    with nbm.Batch([nbm.nb_desc_default(**BINARY), nbm.nb_desc_default(**desc)],
                   [nbm.nb_params_default(**BINARY_P), nbm.nb_params_default(**params)]) as b:
        assert np.array_equal(b.forces(1), a)
        # the potential pass of the mixed launch: system 0's symmetric items
        # (fixed point), system 1's one-sided items (partial slots)
        d1 = b.diagnostics(1)
        og1, _ = orc.potential(ox, om, np.zeros(len(om)), np.zeros(len(om)), G=1.0, eps=eps)
        assert d1["e_grav"] == pytest.approx(float(np.sum(og1)), rel=1e-6)
        d0 = b.diagnostics(0)
        p0 = dict(BINARY_P, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
        bx, _, bm, _, _ = oracle_ic(orc, BINARY, p0)
        og0, _ = orc.potential(bx, bm, np.zeros(len(bm)), np.zeros(len(bm)), G=1.0,
                               eps=BINARY_P["eps"])
        assert d0["e_grav"] == pytest.approx(float(np.sum(og0)), rel=1e-6)
        # diagnostics leave the trajectory as it was
        b.step(3)
        b.sync()
        mixed = b.get_state(1)
    assert np.array_equal(mixed[0], alone[0]) and np.array_equal(mixed[1], alone[1])


@pytest.mark.parametrize("cfg", [None, ONE_SIDED], ids=["default", "one-sided"])
def test_momenta_conserved_over_a_long_run(nbm, cfg):
    """Gravity and contact forces are central and the kick-drift-kick update
    keeps x x v unchanged under the drift, so total linear and angular
    momentum are conserved up to rounding: 4,000 steps of a 16,384-element
    binary with a growing donor (the violent start of the pinned initial
    conditions included), FP32 pair term."""
    desc = dict(n_donor=12288, n_accretor=4096, q=0.3, f_donor=0.9, f_accretor=0.5,
                sigma_v=1e-3, seed=3, stream=0, expand_rate=6.25e-5, expand_steps=8000)
    params = dict(eps=0.005, dt=1e-3, beta=0.5)
    with _make(nbm, desc, params) as s:
        if cfg is not None:
            s.set_pair_cfg(*cfg)
        d0 = s.diagnostics()
        s.step(4000)
        d1 = s.diagnostics()
    assert d1["n_nonfinite"] == 0
    assert d1["step"] == 4000
    lz0 = d0["l"][2]
    assert abs(d1["l"][2] - lz0) <= 1e-6 * abs(lz0)
    assert max(abs(p) for p in d1["p"]) <= 1e-6
    for c in (0, 1):
        assert abs(d1["l"][c] - d0["l"][c]) <= 1e-6 * abs(lz0)
