"""Scenario presets (after the paper's Fig. 5 runs) and the eccentric-orbit
initial state through the C ABI: the library builds the same initial state
as the oracle, its forces match, and a short run stays finite with the
donor's elements starting to cross L1 where the donor overfills its lobe."""
import numpy as np
import pytest

from nbtest import oracle_ic, rms_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nbm():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _as_dicts(d, p):
    desc = {k: getattr(d, k) for k in ("n_donor", "n_accretor", "q", "f_donor", "f_accretor",
                                        "sigma_v", "seed", "stream", "ecc")}
    params = {k: getattr(p, k) for k in ("G", "eps", "beta", "kappa_gamma", "rl_coeff", "flags")}
    return desc, params


@pytest.mark.parametrize("which", [0, 1, 2])
def test_preset_matches_oracle_and_runs(nbm, orc, which, tmp_path):
    d, p = nbm.nb_preset(which, 2048)
    desc, params = _as_dicts(d, p)
    with nbm.System(d, p) as s:
        a = s.forces()
        xv0, _, _ = s.get_state()
        s.step(40)
        s.sync()
        diag = s.diagnostics()
        nbm.dump_state(s, str(tmp_path / "snap.npz"))
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    assert np.abs(xv0[:, :3] - ox).max() < 1e-14
    ref = orc.forces(ox, ov, om, oR, og, G=params["G"], eps=params["eps"], beta=params["beta"])
    assert rms_rel(a, ref) <= 1e-5
    assert diag["step"] == 40 and diag["n_nonfinite"] == 0
    snap = np.load(tmp_path / "snap.npz")
    assert snap["xv"].shape == (2048, 6) and int(snap["step"]) == 40


def test_eccentric_initial_state_matches_oracle(nbm, orc):
    desc = dict(n_donor=600, n_accretor=400, q=0.5, f_donor=0.7, f_accretor=0.5, sigma_v=1e-3,
                seed=5, stream=0, ecc=0.3)
    params = dict(eps=0.01, dt=5e-4, beta=0.5, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    with nbm.System(nbm.nb_desc_default(**desc), nbm.nb_params_default(**params)) as s:
        xv, _, _ = s.get_state()
        a = s.forces()
        s.step(30)
        s.sync()
        x30, _, _ = s.get_state()
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    assert np.abs(xv[:, :3] - ox).max() < 1e-14 and np.abs(xv[:, 3:] - ov).max() < 1e-14
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=0.01, beta=0.5)
    assert rms_rel(a, ref) <= 1e-5
    rx, _, _ = orc.run(ox, ov, om, oR, og, G=1.0, eps=0.01, beta=0.5, dt=5e-4, nsteps=30,
                       n_donor=600)
    assert np.abs(x30[:, :3] - rx).max() <= 1e-4
    with pytest.raises(nbm.NbError):
        nbm.System(nbm.nb_desc_default(ecc=1.0), nbm.nb_params_default())
