"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (from the arithmetic: FP32 coordinates relative to the system's
reference point carry ~3e-8 relative rounding, the MUFU square root and
reciprocal ~1 ulp, tile sums of <= 256 terms are compensated across tiles):
  * FP32 pair term: per-step accelerations within 1e-5 RMS-relative.
  * FP64 pair term: within 1e-12 RMS-relative (summation order only).
  * 100 steps of the 1,024-element binary: positions within 1e-4 (max abs).
  * Initial conditions: both sides build them from the same recipe and the
    same SplitMix64 draws; equal to 1e-14.
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


def _make(nbm, desc, params, **kw):
    d = nbm.nb_desc_default(**desc)
    p = nbm.nb_params_default(**params)
    return nbm.System(d, p, **kw)


def _state(sys_):
    xv, a, meta = sys_.get_state()
    return xv[:, :3], xv[:, 3:], a, meta


# ---------------------------------------------------------------- initial state
def test_initial_conditions_match_oracle(nbm, orc):
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        x, v, a, meta = _state(s)
        ox, ov, om, oR, og = oracle_ic(orc, desc, params)
        assert np.abs(x - ox).max() < 1e-14
        assert np.abs(v - ov).max() < 1e-14
        info = s.info
        assert info.m_donor == pytest.approx(om[0], rel=1e-15)
        assert info.r_donor0 == pytest.approx(oR[0], rel=1e-14)
        assert info.gamma_accretor == pytest.approx(og[-1], rel=1e-13)
        assert meta.step == 0


# ---------------------------------------------------------------- one force evaluation
@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-12)])
def test_forces_binary_1k(nbm, orc, prec, tol):
    desc, params = workload_kwargs("binary_1k")
    params = dict(params, force_prec=prec)
    with _make(nbm, desc, params) as s:
        a = s.forces()
        x, v, a_stored, _ = _state(s)
        ox, ov, om, oR, og = oracle_ic(orc, desc, params)
        ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=params["eps"], beta=params["beta"])
        assert rms_rel(a, ref) <= tol
        # the stored a^0 equals the evaluation at the same state
        assert np.array_equal(a, a_stored)


def _random_system(nbm, n, seed, prec, spread=0.3):
    """A cloud of n elements with per-element masses, radii and strengths
    chosen so that many pairs overlap (both contact branches)."""
    x, v = synth.cloud(n, seed, radius=spread, speed=0.2)
    st = synth.Stream(seed, 11)
    m = 0.5 + st.uniform(n)
    R = (0.02 + 0.02 * st.uniform(n)) * (spread / 0.3) * max(1.0, (64.0 / max(n, 1)) ** (1 / 3))
    gam = 1.0 + st.uniform(n)
    nd = n // 2
    desc = dict(n_donor=nd, n_accretor=n - nd, q=0.5, f_donor=0.8, f_accretor=0.5)
    params = dict(eps=0.003, dt=1e-3, beta=0.35, force_prec=prec)
    xv = np.concatenate([x, v], 1)
    mrg = np.stack([m, R, gam], 1)
    return _make(nbm, desc, params, xv_in=xv, mrg_in=mrg), (x, v, m, R, gam)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 63, 64, 65, 255, 256, 257, 1000, 2049])
@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-12)])
def test_forces_ragged_sizes(nbm, orc, n, prec, tol):
    s, (x, v, m, R, gam) = _random_system(nbm, n, 100 + n, prec)
    with s:
        a = s.forces()
        ref = orc.forces(x, v, m, R, gam, G=1.0, eps=0.003, beta=0.35)
        if n == 1:
            assert np.all(a == 0.0)
        else:
            assert rms_rel(a, ref) <= tol
            # and element by element against the largest acceleration
            assert np.abs(a - ref).max() <= 50 * tol * np.abs(ref).max()


def test_contact_branches_exercised(orc):
    x, v = synth.cloud(257, 357, radius=0.3, speed=0.2)
    st = synth.Stream(357, 11)
    st.uniform(257)
    R = (0.02 + 0.02 * st.uniform(257))
    conv = div = 0
    for i in range(257):
        d = x - x[i]
        r = np.sqrt((d * d).sum(1))
        c = (r < R + R[i]) & (r > 0)
        dv = ((v - v[i]) * d).sum(1)
        conv += int((c & (dv < 0)).sum())
        div += int((c & (dv >= 0)).sum())
    assert conv > 50 and div > 50


# ---------------------------------------------------------------- trajectories
def test_trajectory_binary_1k_100_steps(nbm, orc):
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        s.step(100)
        s.sync()
        x, v, a, meta = _state(s)
        assert meta.step == 100
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    rx, rv, ra = orc.run(ox, ov, om, oR, og, G=1.0, eps=params["eps"], beta=params["beta"],
                         dt=params["dt"], nsteps=100, n_donor=desc["n_donor"])
    assert np.abs(x - rx).max() <= 1e-4
    assert np.sqrt(((x - rx) ** 2).mean()) <= 1e-5


def test_trajectory_fp64_path(nbm, orc):
    desc, params = workload_kwargs("binary_1k")
    params = dict(params, force_prec=64)
    with _make(nbm, desc, params) as s:
        s.step(20)
        s.sync()
        x, v, a, _ = _state(s)
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    rx, rv, ra = orc.run(ox, ov, om, oR, og, G=1.0, eps=params["eps"], beta=params["beta"],
                         dt=params["dt"], nsteps=20, n_donor=desc["n_donor"])
    assert np.abs(x - rx).max() <= 1e-9


def test_donor_expansion_trajectory(nbm, orc):
    """Donor radius grows each step (rate in r_L per step, capped)."""
    desc = dict(n_donor=1536, n_accretor=512, q=0.3, f_donor=0.9, f_accretor=0.5,
                expand_rate=5e-3, expand_steps=30, sigma_v=1e-3, seed=4, stream=0)
    params = dict(eps=0.005, dt=5e-4, beta=0.5)
    with _make(nbm, desc, params) as s:
        s.step(40)
        s.sync()
        x, v, a, meta = _state(s)
        d = s.diagnostics()
    ox, ov, om, oR, og = oracle_ic(orc, desc, dict(params, G=1.0, kappa_gamma=8.0, rl_coeff=0.69))
    rx, rv, ra = orc.run(ox, ov, om, oR, og, G=1.0, eps=0.005, beta=0.5, dt=5e-4, nsteps=40,
                         n_donor=1536, grow_f0=0.9, grow_rate=5e-3, grow_cap=30)
    assert np.abs(x - rx).max() <= 1e-4
    assert d["r_donor"] == pytest.approx(orc.donor_scale(40, 0.9, 5e-3, 30), rel=1e-15)


# ---------------------------------------------------------------- full sizes, sampled
@pytest.mark.parametrize("name,nrows", [("binary_64k", 384), ("binary_1m", 192)])
def test_forces_full_size_sampled(nbm, orc, name, nrows):
    desc, params = workload_kwargs(name)
    with _make(nbm, desc, params) as s:
        a = s.forces()
        x, v, _, _ = _state(s)
        n = s.n
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    assert np.abs(x - ox).max() < 1e-14
    nd = desc["n_donor"]
    rows = np.unique(np.concatenate([
        [0, 1, nd - 1, nd, nd + 1, n - 1],
        (synth.u01(5, 9, nrows) * n).astype(np.int64)]))
    ref = orc.forces_rows(rows, ox, ov, om, oR, og, G=1.0, eps=params["eps"], beta=params["beta"])
    assert rms_rel(a[rows], ref) <= 1e-5


def _grown_radii(orc, R0, n_donor, desc, k):
    """Element radii of step k: donor radii scaled by the growth law, the
    accretor's fixed."""
    R = np.array(R0, dtype=np.float64)
    R[:n_donor] *= orc.donor_scale(k, desc["f_donor"], desc["expand_rate"], desc["expand_steps"])
    return R


def test_binary_64k_growing_donor_sampled(nbm, orc):
    """The 65,536-element binary (q = 0.3, eps 0.005, dt 5e-4) with the donor
    growing from 0.9 to 1.15 r_L over 10^4 steps, stepped on the GPU at full
    size.  At steps 25, 50, 1,000 and 10,000 (the donor at 1.15 r_L, many
    elements pressed from all sides): the accelerations at the state (x^k,
    v^k) with the radii of step k, and the stored a^k of the integrator at
    (x^k, v^{k-1/2}), against the oracle on sampled rows -- 320 random rows,
    the donor/accretor index boundary and the 64 donor elements nearest the
    accretor (the donor's surface facing L1, where its growth acts first).
    At the first two, while the start's overlaps still push hard, the
    initial radii would give forces farther from the oracle than the
    tolerance: the growth is visible."""
    desc, params = workload_kwargs("binary_64k")
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    nd, dt = desc["n_donor"], params["dt"]
    with _make(nbm, desc, params) as s:
        n = s.n
        k = 0
        for k_next in (25, 50, 1000, 10000):
            s.step(k_next - k)
            s.sync()
            k = k_next
            x, v, a_stored, meta = _state(s)
            assert meta.step == k
            a = s.forces()
            near_l1 = np.argsort(x[:nd, 0])[:64]  # donor centre at +x, accretor at -x
            rows = np.unique(np.concatenate([
                [0, 1, nd - 1, nd, nd + 1, n - 1], near_l1,
                (synth.u01(7, k, 320) * n).astype(np.int64)]))
            Rk = _grown_radii(orc, oR, nd, desc, k)
            kw = dict(G=1.0, eps=params["eps"], beta=params["beta"])
            ref = orc.forces_rows(rows, x, v, om, Rk, og, **kw)
            # 1e-5 is the stated tolerance; the contact depth and distance in
            # double-float keep the compressed late states near 3e-7 (FP32
            # depths reached 5e-6 at step 10,000)
            assert rms_rel(a[rows], ref) <= 1e-6
            # the integrator's a^k used the half-step velocity v^{k-1/2}
            vh = v - 0.5 * dt * a_stored
            ref_h = orc.forces_rows(rows, x, vh, om, Rk, og, **kw)
            assert rms_rel(a_stored[rows], ref_h) <= 1e-6
            if k <= 50:
                # the growth is visible at this tolerance: the initial radii
                # give accelerations farther off than the tolerance
                ref0 = orc.forces_rows(rows, x, v, om, oR, og, **kw)
                assert rms_rel(ref0, ref) > 1e-4
            assert s.diagnostics()["r_donor"] == pytest.approx(
                orc.donor_scale(k, desc["f_donor"], desc["expand_rate"], desc["expand_steps"]),
                rel=1e-15)


# ---------------------------------------------------------------- diagnostics
def test_diagnostics_match_oracle(nbm, orc):
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        s.step(10)
        d = s.diagnostics()
        x, v, _, _ = _state(s)
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    ref = orc.diagnostics(x, v, om, oR, og, eps=params["eps"], n_donor=desc["n_donor"], q=desc["q"])
    assert d["step"] == 10
    assert d["e_kin"] == pytest.approx(ref["E_kin"], rel=1e-12)
    assert d["e_rep"] == pytest.approx(ref["E_rep"], rel=1e-10)
    assert d["e_grav"] == pytest.approx(ref["E_grav"], rel=1e-6)  # FP32 pair potential
    assert np.allclose(d["p"], ref["P"], rtol=0, atol=1e-14)
    assert np.allclose(d["l"], ref["L"], rtol=1e-12, atol=1e-15)
    assert np.allclose(d["com"], ref["com"], rtol=0, atol=1e-14)
    assert np.allclose(d["com_donor"], ref["com_donor"], rtol=0, atol=1e-14)
    assert d["separation"] == pytest.approx(ref["separation"], rel=1e-13)
    assert d["n_past_L1"] == ref["n_past_L1"]
    assert d["n_in_accretor_lobe"] == ref["n_in_acc_lobe"]
    assert d["n_unbound"] == ref["n_unbound"]
    assert d["m_unbound"] == pytest.approx(ref["m_unbound"], rel=1e-12, abs=1e-300)
    assert d["n_nonfinite"] == 0


def test_mass_transfer_accounting_matches_oracle(nbm, orc):
    """Donor elements past L1, inside the accretor's lobe and unbound, after
    the violent first steps of the 1,024-element binary (elements are
    ejected) and for a hand-placed state with elements moved into the
    accretor's lobe."""
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        s.step(60)
        d = s.diagnostics()
        x, v, _, _ = _state(s)
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    ref = orc.diagnostics(x, v, om, oR, og, eps=params["eps"], n_donor=desc["n_donor"], q=desc["q"])
    assert ref["n_unbound"] > 0  # the pinned IC recipe ejects elements
    for k_lib, k_ref in [("n_past_L1", "n_past_L1"), ("n_in_accretor_lobe", "n_in_acc_lobe"),
                         ("n_unbound", "n_unbound")]:
        assert d[k_lib] == ref[k_ref], k_lib
    # elements moved into the accretor's lobe
    x2 = x.copy()
    ca = ref["com_accretor"]
    x2[:20] = ca + 0.02 * (np.arange(20)[:, None] % 3 - 1.0)
    xv = np.concatenate([x2, v], 1)
    with _make(nbm, desc, params, xv_in=xv) as s:
        d2 = s.diagnostics()
    ref2 = orc.diagnostics(x2, v, om, oR, og, eps=params["eps"], n_donor=desc["n_donor"],
                           q=desc["q"])
    assert d2["n_in_accretor_lobe"] == ref2["n_in_acc_lobe"] >= 10


# ---------------------------------------------------------------- determinism, checkpoints
def test_runs_are_bitwise_reproducible(nbm):
    desc, params = workload_kwargs("binary_1k")
    out = []
    for _ in range(2):
        with _make(nbm, desc, params) as s:
            s.step(25)
            out.append(_state(s))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_checkpoint_resume_bitwise(nbm):
    desc, params = workload_kwargs("binary_1k")
    desc = dict(desc, expand_rate=1e-3, expand_steps=25)
    with _make(nbm, desc, params) as s:
        s.step(40)
        x_ref, v_ref, a_ref, _ = _state(s)
    with _make(nbm, desc, params) as s:
        s.step(15)
        xv, a, meta = s.get_state()
    with _make(nbm, desc, params) as s2:
        s2.set_state(xv, a, meta)
        s2.step(25)
        x2, v2, a2, meta2 = _state(s2)
    assert meta2.step == 40
    assert np.array_equal(x_ref, x2) and np.array_equal(v_ref, v2) and np.array_equal(a_ref, a2)


def test_set_state_rejects_nonfinite_and_keeps_state(nbm):
    """A checkpoint with a non-finite value is refused (NB_EINVAL naming the
    first bad row) and the system's state is left as it was; page-locked
    output arrays are filled in place."""
    import torch
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        s.step(3)
        xv, a, meta = s.get_state()
        bad = xv.copy()
        bad[700, 4] = np.nan
        bad[900, 0] = np.inf
        with pytest.raises(nbm.NbError) as ei:
            s.set_state(bad, a, meta)
        assert ei.value.status == nbm.NB_EINVAL and "xv_in[700]" in str(ei.value)
        n = s.n
        pxv = torch.empty((n, 6), dtype=torch.float64, pin_memory=True).numpy()
        pa = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        _, _, meta2 = s.get_state(out=(pxv, pa))
        assert meta2.step == 3
        assert np.array_equal(pxv, xv) and np.array_equal(pa, a)


def test_caller_arrays_of_the_wrong_size_are_refused(nbm):
    """The library reads and writes exactly n rows through caller pointers;
    the binding refuses arrays of another size before any call (the state is
    left as it was)."""
    import torch
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        xv, a, meta = s.get_state()
        with pytest.raises(ValueError):
            s.set_state(xv[:-1], None, meta)
        with pytest.raises(ValueError):
            s.set_state(xv, a[:, :2], meta)
        with pytest.raises(ValueError):
            s.forces(out=np.empty((s.n, 2)))
        with pytest.raises(ValueError):
            s.forces(out=torch.empty(3 * s.n - 3, dtype=torch.float64, device="cuda"))
        with pytest.raises(ValueError):
            s.forces(out=torch.empty(3 * s.n, dtype=torch.float32, device="cuda"))
        xv2, a2, _ = s.get_state()
        assert np.array_equal(xv, xv2) and np.array_equal(a, a2)
        dev = torch.empty(3 * s.n, dtype=torch.float64, device="cuda")
        s.forces(out=dev)
        assert np.array_equal(dev.cpu().numpy().reshape(-1, 3), s.forces())


def test_steps_split_across_calls_bitwise(nbm):
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        s.step(12)
        r1 = _state(s)
    with _make(nbm, desc, params) as s:
        for _ in range(3):
            s.step(4)
        r2 = _state(s)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


# ---------------------------------------------------------------- failure detection
def test_nonfinite_state_is_reported(nbm):
    """An element whose drift overflows to infinity is flagged by the update
    kernel and reported by nb_sync as NB_ENONFINITE (no GPU fault)."""
    n = 8
    x, v = synth.cloud(n, 3, radius=0.5)
    v[3] = [1e308, 0.0, 0.0]
    desc = dict(n_donor=4, n_accretor=4, q=1.0)
    params = dict(eps=0.01, dt=10.0, flags=nbm.NB_GRAVITY_ONLY)
    with _make(nbm, desc, params, xv_in=np.concatenate([x, v], 1)) as s:
        s.step(1)
        with pytest.raises(nbm.NbError) as ei:
            s.sync()
        assert ei.value.status == nbm.NB_ENONFINITE
        assert s.diagnostics()["n_nonfinite"] >= 1


def test_gravity_only_flag(nbm, orc):
    desc, params = workload_kwargs("binary_1k")
    params = dict(params, flags=nbm.NB_GRAVITY_ONLY)
    with _make(nbm, desc, params) as s:
        a = s.forces()
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    ref = orc.forces(ox, ov, om, oR, np.zeros_like(og), G=1.0, eps=params["eps"])
    assert rms_rel(a, ref) <= 1e-5


# ---------------------------------------------------------------- launch variants
def _variants():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody.nb_pair_cfg_variants()


@pytest.mark.parametrize("cfg", _variants())
def test_every_pair_variant_matches_oracle(nbm, orc, cfg):
    """Each built (tile, i per thread, threads, blocks) variant, on a ragged
    size with per-element masses (per-pair mass path) and on the binary
    (uniform-mass tiles)."""
    s, (x, v, m, R, gam) = _random_system(nbm, 2049, 77, 32)
    with s:
        s.set_pair_cfg(*cfg)
        a = s.forces()
    ref = orc.forces(x, v, m, R, gam, G=1.0, eps=0.003, beta=0.35)
    assert rms_rel(a, ref) <= 1e-5
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        s.set_pair_cfg(*cfg)
        a = s.forces()
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=params["eps"], beta=params["beta"])
    assert rms_rel(a, ref) <= 1e-5


def test_autotune_keeps_parity(nbm, orc):
    desc, params = workload_kwargs("binary_1k")
    with _make(nbm, desc, params) as s:
        best = s.autotune(2)
        assert (best["tile"], best["i_per_thread"], best["threads"], best["min_blocks"],
                best["nr_slots"], best["i_packed"], best["shared_rcp"],
                best["symmetric"]) in _variants()
        assert best["ms"] > 0
        cfg = s.pair_cfg()
        assert cfg["tile"] == best["tile"]
        a = s.forces()
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=params["eps"], beta=params["beta"])
    assert rms_rel(a, ref) <= 1e-5


def test_graph_replay_equals_direct_launches(nbm):
    """Multi-step calls on a non-default stream replay a captured CUDA graph;
    the result is bitwise that of direct launches on the default stream."""
    import torch
    desc, params = workload_kwargs("binary_1k")
    desc = dict(desc, expand_rate=1e-3, expand_steps=-1)
    with _make(nbm, desc, params) as s:
        s.step(7)
        s.step(7)
        r_direct = _state(s)
    stream = torch.cuda.Stream()
    with _make(nbm, desc, params, stream=stream) as s:
        s.step(7)
        s.step(7)
        s.sync()
        r_graph = _state(s)
    for a, b in zip(r_direct[:3], r_graph[:3]):
        assert np.array_equal(a, b)
    assert r_graph[3].step == 14


def test_bounded_device_wait_times_out_cleanly(nbm, orc):
    """A device wait on a barrier that nothing completes gives up after its
    budget and reports NB_ETIMEOUT; the context stays usable."""
    import time
    t0 = time.perf_counter()
    st = nbm.nb_selftest_device_wait(20_000_000)  # ~10 ms of SM clocks
    assert st == nbm.NB_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    test_forces_binary_1k(nbm, orc, 32, 1e-5)


@pytest.mark.parametrize("cfg", [(128, 8, 128, 2, 0, 0, 8), (256, 8, 128, 2, 0, 0, 6),
                                 (256, 8, 128, 2, 0, 0, 2, 1)])
def test_shared_reciprocal_falls_back_without_softening(nbm, orc, cfg):
    """With eps < 1e-4 the shared-reciprocal variants use the plain
    reciprocal (the product of two denominators could underflow); the
    result still matches the oracle, here with eps = 0."""
    n = 1500
    x, v = synth.cloud(n, 91, radius=0.5, speed=0.2)
    m = 0.5 + synth.u01(91, 3, n)
    desc = dict(n_donor=n // 2, n_accretor=n - n // 2, q=0.5)
    params = dict(eps=0.0, dt=1e-3, beta=0.5, flags=nbm.NB_GRAVITY_ONLY)
    mrg = np.stack([m, np.zeros(n), np.zeros(n)], 1)
    with _make(nbm, desc, params, xv_in=np.concatenate([x, v], 1), mrg_in=mrg) as s:
        s.set_pair_cfg(*cfg)
        a = s.forces()
    ref = orc.forces(x, v, m, np.zeros(n), np.zeros(n), G=1.0, eps=0.0)
    assert rms_rel(a, ref) <= 1e-5


def test_unit_rate_probe(nbm):
    """The measured issue rates behind the roofline are those of a
    Blackwell SM at its clock: 16 MUFU results and 128 FP32 lanes per clock
    (per second here, so bounded with the clock range of the part)."""
    import torch
    r = nbm.nb_measure_unit_rates(torch.cuda.Stream())
    assert r["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    for k in ("mufu_sqrt_per_s_sm", "mufu_rcp_per_s_sm"):
        assert 12.0 * 1.0e9 <= r[k] <= 17.0 * 2.2e9, r
    assert 96.0 * 1.0e9 <= r["fp32_lanes_per_s_sm"] <= 130.0 * 2.2e9, r
    # the two MUFU operations and the FP32 lanes keep the SM's 1 : 8 ratio
    ratio = r["fp32_lanes_per_s_sm"] / r["mufu_rcp_per_s_sm"]
    assert 7.0 <= ratio <= 9.0, r
    # the symmetric kernel's instruction mix from registers: at most the
    # bound of the separate pipes (15 FP32 lanes and 2 MUFU per evaluation)
    mix = r["pair_mix_evals_per_s_sm"]
    bound = min(r["fp32_lanes_per_s_sm"] / 15.0,
                1.0 / (1.0 / r["mufu_sqrt_per_s_sm"] + 1.0 / r["mufu_rcp_per_s_sm"]))
    assert 0.3 * bound <= mix <= 1.02 * bound, r


# ---------------------------------------------------------------- stored values
@pytest.mark.parametrize("prec,ftol,xtol", [(32, 1e-5, 1e-5), (64, 1e-12, 1e-11)])
def test_stored_binary_64(nbm, prec, ftol, xtol):
    """The 64-element binary of tests/golden/binary_64.txt (written from the
    FP64 oracle): the library's forces at the start and its state after the
    stored number of steps, against the stored values."""
    from test_golden import load_binary_64
    desc, p, steps, a0, x, v, a = load_binary_64()
    params = dict(eps=p["eps"], dt=p["dt"], beta=p["beta"], G=p["G"], force_prec=prec)
    with _make(nbm, dict(desc), params) as s:
        got0 = s.forces()
        s.step(steps)
        s.sync()
        xv, _, meta = s.get_state()
    assert meta.step == steps
    assert rms_rel(got0, a0) <= ftol
    assert np.abs(xv[:, :3] - x).max() <= xtol
    assert rms_rel(xv[:, 3:], v) <= 100 * ftol
