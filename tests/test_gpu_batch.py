"""Batched and served forms through the C ABI.

* A system advanced inside a batch (one kernel launch per phase for all
  systems) gives bitwise the state it gives alone.
* A batch's forces match the FP64 oracle per system.
* The server (continuous batching) returns, for every run, the result of
  running it alone; its admission respects the device-memory budget.
"""
import numpy as np
import pytest

from nbtest import oracle_ic, rms_rel

pytestmark = pytest.mark.gpu

SYSTEMS = [
    dict(desc=dict(n_donor=512, n_accretor=512, q=0.5, f_donor=0.8, f_accretor=0.5,
                   sigma_v=1e-3, seed=1),
         params=dict(eps=0.01, dt=1e-3, beta=0.5)),
    dict(desc=dict(n_donor=1900, n_accretor=600, q=0.3, f_donor=0.9, f_accretor=0.5,
                   expand_rate=2e-3, expand_steps=-1, sigma_v=1e-3, seed=2),
         params=dict(eps=0.005, dt=5e-4, beta=0.3)),
    dict(desc=dict(n_donor=350, n_accretor=350, q=0.9, f_donor=0.7, f_accretor=0.6,
                   sigma_v=2e-3, seed=3),
         params=dict(eps=0.008, dt=8e-4, beta=0.7)),
]


@pytest.fixture(scope="module")
def nbm():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _descs(nbm, systems):
    return ([nbm.nb_desc_default(**s["desc"]) for s in systems],
            [nbm.nb_params_default(**s["params"]) for s in systems])


CFG_FIELDS = ("tile", "i_per_thread", "threads", "min_blocks", "nr_slots", "i_packed",
              "shared_rcp", "symmetric")


def _alone(nbm, s, nsteps, stream=None, cfg=None):
    """The run alone; with cfg (a pair configuration as a dict), a^0 is
    re-evaluated with it before stepping, as a server does at admission."""
    with nbm.System(nbm.nb_desc_default(**s["desc"]), nbm.nb_params_default(**s["params"]),
                    stream=stream) as sysm:
        if cfg is not None:
            sysm.set_pair_cfg(*[cfg[f] for f in CFG_FIELDS])
            xv, _, meta = sysm.get_state()
            sysm.set_state(xv, None, meta)
        sysm.step(nsteps)
        sysm.sync()
        xv, a, meta = sysm.get_state()
        d = sysm.diagnostics()
    return xv, a, meta, d


def test_batch_alone_vs_mix_bitwise(nbm):
    import torch
    descs, params = _descs(nbm, SYSTEMS)
    stream = torch.cuda.Stream()
    with nbm.Batch(descs, params, stream=stream) as b:
        b.step(6)
        b.step(6)
        b.sync()
        mixed = [b.get_state(s) for s in range(len(SYSTEMS))]
    for s, sysdef in enumerate(SYSTEMS):
        xv, a, meta, _ = _alone(nbm, sysdef, 12)
        assert mixed[s][2].step == 12
        assert np.array_equal(mixed[s][0], xv), f"system {s} positions/velocities differ"
        assert np.array_equal(mixed[s][1], a), f"system {s} accelerations differ"


def test_batch_forces_match_oracle(nbm, orc):
    descs, params = _descs(nbm, SYSTEMS)
    with nbm.Batch(descs, params) as b:
        for s, sysdef in enumerate(SYSTEMS):
            a = b.forces(s)
            d = dict(sysdef["desc"])
            d.setdefault("stream", 0)
            p = dict(sysdef["params"], G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
            ox, ov, om, oR, og = oracle_ic(orc, d, p)
            ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=p["eps"], beta=p["beta"])
            assert rms_rel(a, ref) <= 1e-5


def test_batch_diagnostics_per_system(nbm):
    descs, params = _descs(nbm, SYSTEMS)
    with nbm.Batch(descs, params) as b:
        b.step(3)
        for s, sysdef in enumerate(SYSTEMS):
            d = b.diagnostics(s)
            _, _, _, ref = _alone(nbm, sysdef, 3)
            assert d["step"] == 3
            for k in ("e_kin", "e_grav", "e_rep"):
                assert d[k] == ref[k]
            assert np.array_equal(d["p"], ref["p"]) and np.array_equal(d["l"], ref["l"])


def _server_requests():
    reqs = []
    for k in range(6):
        s = SYSTEMS[k % 3]
        reqs.append((s, 5 + 4 * k))
    return reqs


def test_server_results_equal_alone(nbm):
    import torch
    stream = torch.cuda.Stream()
    srv = nbm.nb_server_create(4 << 30, 3, 4096, 32, stream)
    try:
        cfg = nbm.nb_server_pair_cfg(srv)
        info = nbm.nb_server_info(srv)
        assert info["nslots"] == 3 and info["slot_n"] >= 4096
        tickets = []
        for s, nsteps in _server_requests():
            d = nbm.nb_desc_default(**s["desc"])
            p = nbm.nb_params_default(**s["params"])
            tickets.append(nbm.nb_submit(srv, d, p, nsteps))
        nbm.nb_server_drain(srv, 120.0)
        results = [nbm.nb_poll(srv, t) for t in tickets]
    finally:
        nbm.nb_server_destroy(srv)
    for (s, nsteps), r in zip(_server_requests(), results):
        assert r["status"] == nbm.NB_OK
        assert r["steps"] == nsteps
        assert r["t_submit"] <= r["t_start"] <= r["t_finish"]
        _, _, _, ref = _alone(nbm, s, nsteps, cfg=cfg)
        d = r["diag"]
        assert d["step"] == nsteps
        assert d["e_kin"] == ref["e_kin"]
        assert np.array_equal(d["p"], ref["p"]) and np.array_equal(d["l"], ref["l"])
        assert np.array_equal(d["com"], ref["com"])
        assert d["n_past_L1"] == ref["n_past_L1"]
        assert np.isnan(d["e_grav"])


def test_server_admits_by_request_bytes(nbm):
    """Admission counts each run's own device bytes against the budget.  The
    budget holds one run of the largest size (4,096 elements) but not that
    run and a 1,024-element one: the three small runs queued behind the large
    one (long enough for several admission rounds to pass while it runs)
    wait until it is retired, then all three run at once."""
    with pytest.raises(nbm.NbError) as ei:
        nbm.nb_server_create(1000, 4, 4096, 32)
    assert ei.value.status == nbm.NB_EBUDGET
    probe = nbm.nb_server_create(1 << 30, 8, 4096, 32)
    try:
        per_big = nbm.nb_server_stats_read(probe)["max_request_bytes"]
    finally:
        nbm.nb_server_destroy(probe)
    budget = int(per_big * 1.1)
    big = dict(desc=dict(n_donor=3000, n_accretor=1000, q=0.4, f_donor=0.9, f_accretor=0.5,
                         sigma_v=1e-3, seed=5), params=dict(eps=0.006, dt=5e-4, beta=0.5))
    small = SYSTEMS[0]  # 1,024 elements: a quarter of the large run's bytes
    srv = nbm.nb_server_create(budget, 8, 4096, 32)
    try:
        assert nbm.nb_server_info(srv)["nslots"] == 8
        t_big = nbm.nb_submit(srv, nbm.nb_desc_default(**big["desc"]),
                              nbm.nb_params_default(**big["params"]), 400)
        t_small = [nbm.nb_submit(srv, nbm.nb_desc_default(**small["desc"]),
                                 nbm.nb_params_default(**small["params"]), 8) for _ in range(3)]
        with pytest.raises(nbm.NbError) as ei:
            nbm.nb_submit(srv, nbm.nb_desc_default(n_donor=5000, n_accretor=5000),
                          nbm.nb_params_default(), 1)
        assert ei.value.status == nbm.NB_EBUDGET
        with pytest.raises(nbm.NbError) as ei:
            nbm.nb_poll(srv, 999999)
        assert ei.value.status == nbm.NB_ENOTFOUND
        for bad in (-1.0, float("nan")):
            with pytest.raises(nbm.NbError) as ei:
                nbm.nb_server_drain(srv, bad)
            assert ei.value.status == nbm.NB_EINVAL
        nbm.nb_server_drain(srv, float("inf"))  # no limit: returns when all are done
        rb = nbm.nb_poll(srv, t_big)
        rs = [nbm.nb_poll(srv, t) for t in t_small]
        st = nbm.nb_server_stats_read(srv)
    finally:
        nbm.nb_server_destroy(srv)
    assert rb["status"] == nbm.NB_OK and all(r["status"] == nbm.NB_OK for r in rs)
    for r in rs:
        assert r["t_start"] >= rb["t_finish"]
    # the three small runs were in flight together
    assert max(r["t_start"] for r in rs) < min(r["t_finish"] for r in rs)
    assert rs[0]["diag"]["e_kin"] == rs[1]["diag"]["e_kin"] == rs[2]["diag"]["e_kin"]
    assert st["peak_requests"] == 3
    assert st["peak_bytes"] <= budget
    assert st["admissions_deferred"] > 0
    assert st["requests_running"] == 0 and st["bytes_in_use"] == 0


def test_server_many_small_runs_share_the_arena(nbm):
    """Runs much smaller than the largest size take only their own room:
    with max_n = 65,536 and a budget of two such runs, eight 1,024-element
    runs are all in flight at once (fixed slots of max_n would hold two)."""
    probe = nbm.nb_server_create(1 << 30, 16, 65536, 32)
    try:
        per_big = nbm.nb_server_stats_read(probe)["max_request_bytes"]
    finally:
        nbm.nb_server_destroy(probe)
    srv = nbm.nb_server_create(int(2.2 * per_big), 16, 65536, 32)
    s = SYSTEMS[0]
    runs = [dict(s, desc=dict(s["desc"], seed=40 + k)) for k in range(8)]
    try:
        cfg = nbm.nb_server_pair_cfg(srv)
        # long enough (several chunks of steps) that all eight are admitted
        # before the first one finishes
        tickets = [nbm.nb_submit(srv, nbm.nb_desc_default(**r["desc"]),
                                 nbm.nb_params_default(**r["params"]), 400) for r in runs]
        nbm.nb_server_drain(srv, 120.0)
        res = [nbm.nb_poll(srv, t) for t in tickets]
        st = nbm.nb_server_stats_read(srv)
    finally:
        nbm.nb_server_destroy(srv)
    assert all(r["status"] == nbm.NB_OK and r["steps"] == 400 for r in res)
    assert st["peak_requests"] == 8
    assert st["peak_elements"] == 8 * 1024
    # wherever a run sat in the arena, its result is the run alone
    for k in (0, 5):
        _, _, _, ref = _alone(nbm, runs[k], 400, cfg=cfg)
        assert res[k]["diag"]["e_kin"] == ref["e_kin"]
        assert np.array_equal(res[k]["diag"]["com"], ref["com"])


def test_server_large_slots_use_symmetric_kernel(nbm):
    """Slots of >= 16,384 elements run the symmetric pair kernel; a run's
    result equals the run alone with the server's configuration."""
    import torch
    stream = torch.cuda.Stream()
    big = [
        dict(desc=dict(n_donor=12000, n_accretor=5000, q=0.4, f_donor=0.9, f_accretor=0.5,
                       sigma_v=1e-3, seed=7), params=dict(eps=0.005, dt=5e-4, beta=0.5)),
        dict(desc=dict(n_donor=3000, n_accretor=2000, q=0.7, f_donor=0.8, f_accretor=0.5,
                       expand_rate=1e-3, expand_steps=-1, sigma_v=1e-3, seed=8),
             params=dict(eps=0.008, dt=5e-4, beta=0.4)),
    ]
    srv = nbm.nb_server_create(8 << 30, 2, 17000, 32, stream)
    try:
        cfg = nbm.nb_server_pair_cfg(srv)
        assert cfg["symmetric"] >= 1
        tickets = [nbm.nb_submit(srv, nbm.nb_desc_default(**b["desc"]),
                                 nbm.nb_params_default(**b["params"]), 7 + 5 * k)
                   for k, b in enumerate(big)]
        nbm.nb_server_drain(srv, 120.0)
        results = [nbm.nb_poll(srv, t) for t in tickets]
    finally:
        nbm.nb_server_destroy(srv)
    fields = ("tile", "i_per_thread", "threads", "min_blocks", "nr_slots", "i_packed",
              "shared_rcp", "symmetric")
    for k, (b, r) in enumerate(zip(big, results)):
        assert r["status"] == nbm.NB_OK
        with nbm.System(nbm.nb_desc_default(**b["desc"]), nbm.nb_params_default(**b["params"])) as s:
            s.set_pair_cfg(*[cfg[f] for f in fields])
            # a^0 re-evaluated with the server's configuration
            xv, _, meta = s.get_state()
            s.set_state(xv, None, meta)
            s.step(7 + 5 * k)
            s.sync()
            d = s.diagnostics()
        assert r["diag"]["e_kin"] == d["e_kin"]
        assert np.array_equal(r["diag"]["p"], d["p"]) and np.array_equal(r["diag"]["com"], d["com"])


def test_server_shortest_work_first_keeps_results(nbm):
    """Two runs large enough to fill a step each: once both are admitted the
    one with less work left runs alone and the other waits; both results
    equal the runs alone (paused and resumed steps are bitwise invisible)."""
    import torch
    stream = torch.cuda.Stream()
    big = dict(n_donor=82000, n_accretor=28000, q=0.3, f_donor=0.9, f_accretor=0.5,
               sigma_v=1e-3, seed=11)
    p = dict(eps=0.005, dt=5e-4, beta=0.5)
    srv = nbm.nb_server_create(16 << 30, 2, 110000, 32, stream)
    try:
        cfg = nbm.nb_server_pair_cfg(srv)
        t_long = nbm.nb_submit(srv, nbm.nb_desc_default(**big), nbm.nb_params_default(**p), 150)
        t_short = nbm.nb_submit(srv, nbm.nb_desc_default(**dict(big, seed=12)),
                                nbm.nb_params_default(**p), 6)
        nbm.nb_server_drain(srv, 300.0)
        r_long, r_short = nbm.nb_poll(srv, t_long), nbm.nb_poll(srv, t_short)
    finally:
        nbm.nb_server_destroy(srv)
    assert r_long["status"] == r_short["status"] == nbm.NB_OK
    assert r_short["t_finish"] < r_long["t_finish"]
    fields = ("tile", "i_per_thread", "threads", "min_blocks", "nr_slots", "i_packed",
              "shared_rcp", "symmetric")
    for desc, steps, r in [(big, 150, r_long), (dict(big, seed=12), 6, r_short)]:
        with nbm.System(nbm.nb_desc_default(**desc), nbm.nb_params_default(**p)) as s:
            s.set_pair_cfg(*[cfg[f] for f in fields])
            xv, _, meta = s.get_state()
            s.set_state(xv, None, meta)
            s.step(steps)
            s.sync()
            d = s.diagnostics()
        assert r["steps"] == steps and r["diag"]["step"] == steps
        assert r["diag"]["e_kin"] == d["e_kin"]
        assert np.array_equal(r["diag"]["com"], d["com"])


def test_batch_set_state_one_system(nbm):
    """A checkpoint restored into one system of a batch rewinds that system
    only; each system then matches its own run alone, bitwise."""
    import torch
    descs, params = _descs(nbm, SYSTEMS)
    stream = torch.cuda.Stream()
    with nbm.Batch(descs, params, stream=stream) as b:
        b.step(4)
        b.sync()
        saved = b.get_state(1)
        b.step(3)
        b.sync()
        b.set_state(1, *saved)           # system 1 back to step 4, the others at 7
        b.step(5)
        b.sync()
        got = [b.get_state(s) for s in range(len(SYSTEMS))]
    for s, steps in [(0, 12), (1, 9), (2, 12)]:
        xv, a, meta, _ = _alone(nbm, SYSTEMS[s], steps)
        assert got[s][2].step == steps
        assert np.array_equal(got[s][0], xv) and np.array_equal(got[s][1], a), s


def test_server_fp64(nbm):
    """A server running the FP64 pair path returns, per run, the result of
    the run alone with the FP64 path."""
    srv = nbm.nb_server_create(1 << 30, 2, 4096, 64)
    try:
        reqs = [(SYSTEMS[0], 6), (SYSTEMS[2], 9)]
        tickets = [nbm.nb_submit(srv, nbm.nb_desc_default(**s["desc"]),
                                 nbm.nb_params_default(**dict(s["params"], force_prec=64)), n)
                   for s, n in reqs]
        nbm.nb_server_drain(srv, 120.0)
        res = [nbm.nb_poll(srv, t) for t in tickets]
        # a run of the other precision is refused at admission, promptly
        t = nbm.nb_submit(srv, nbm.nb_desc_default(**SYSTEMS[0]["desc"]),
                          nbm.nb_params_default(**SYSTEMS[0]["params"]), 2)
        t0 = nbm.nb_server_clock(srv)
        nbm.nb_server_drain(srv, 60.0)
        assert nbm.nb_server_clock(srv) - t0 < 10.0
        assert nbm.nb_poll(srv, t)["status"] == nbm.NB_EINVAL
    finally:
        nbm.nb_server_destroy(srv)
    for (s, n), r in zip(reqs, res):
        assert r["status"] == nbm.NB_OK
        one = dict(s, params=dict(s["params"], force_prec=64))
        _, _, _, ref = _alone(nbm, one, n)
        assert r["diag"]["e_kin"] == ref["e_kin"]
        assert np.array_equal(r["diag"]["com"], ref["com"])
