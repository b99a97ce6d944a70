"""Degenerate cases of the method on the GPU, against the FP64 oracle.

* Coincident elements (r = 0): the pair has no direction and contributes
  nothing to either element, gravity or contact (the oracle skips d^2 = 0).
* A whole system at one point: every acceleration is exactly zero.
* Eq. 6 at its extremes: beta = 1 (elastic contact) and beta = 0 (no
  repulsion while separating).
* G = 0 with contacts: the contact term alone.
* q = 1: both stars of equal element mass, one mass run over the system.

Each case runs the default pair kernel (each unordered pair once), the
one-sided kernel and the FP64 path.
"""
import numpy as np
import pytest

import synth
from nbtest import oracle_ic, rms_rel

pytestmark = pytest.mark.gpu

SYMMETRIC = (256, 12, 128, 2, 0, 0, 2, 3)
ONE_SIDED = (256, 8, 128, 2, 0, 0, 6, 0)
PATHS = [("symmetric", 32, SYMMETRIC), ("one-sided", 32, ONE_SIDED), ("fp64", 64, None)]


@pytest.fixture(scope="module")
def nbm():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _forces(nbm, x, v, m, R, gam, prec, cfg, **params):
    n = x.shape[0]
    desc = nbm.nb_desc_default(n_donor=n // 2, n_accretor=n - n // 2, q=0.5)
    p = nbm.nb_params_default(dt=1e-3, force_prec=prec, **params)
    with nbm.System(desc, p, xv_in=np.concatenate([x, v], 1),
                    mrg_in=np.stack([m, R, gam], 1)) as s:
        if cfg is not None:
            s.set_pair_cfg(*cfg)
        return s.forces()


def _cloud(n, seed, contacts=True):
    x, v = synth.cloud(n, seed, radius=0.3, speed=0.2)
    st = synth.Stream(seed, 13)
    m = 0.5 + st.uniform(n)
    R = (0.01 + 0.01 * st.uniform(n)) if contacts else np.zeros(n)
    gam = (1.0 + st.uniform(n)) if contacts else np.zeros(n)
    return x, v, m, R, gam


@pytest.mark.parametrize("path,prec,cfg", PATHS, ids=[p[0] for p in PATHS])
def test_coincident_elements_contribute_nothing(nbm, orc, path, prec, cfg):
    """Every 7th element is placed exactly on its predecessor (with its own
    velocity, radius and strength): those pairs drop out of both terms."""
    n = 3000
    x, v, m, R, gam = _cloud(n, 41)
    x[1::7] = x[0::7][: len(x[1::7])]
    a = _forces(nbm, x, v, m, R, gam, prec, cfg, eps=0.004, beta=0.4)
    ref = orc.forces(x, v, m, R, gam, G=1.0, eps=0.004, beta=0.4)
    assert np.all(np.isfinite(a))
    tol = 1e-5 if prec == 32 else 1e-12
    assert rms_rel(a, ref) <= tol
    # the duplicated pairs themselves: same as with the partner removed
    k = 7 * 11
    keep = np.ones(n, dtype=bool)
    keep[k + 1] = False
    ref_k = orc.forces_rows([k], x[keep], v[keep], m[keep], R[keep], gam[keep], G=1.0,
                            eps=0.004, beta=0.4)[0]
    assert np.abs(a[k] - ref_k).max() <= 50 * tol * np.abs(ref_k).max()


@pytest.mark.parametrize("path,prec,cfg", PATHS, ids=[p[0] for p in PATHS])
def test_system_at_one_point_has_zero_acceleration(nbm, path, prec, cfg):
    n = 600
    x = np.tile([[0.1, -0.2, 0.05]], (n, 1))
    v = synth.cloud(n, 5, speed=0.1)[1]
    a = _forces(nbm, x, v, np.ones(n), np.full(n, 0.02), np.ones(n), prec, cfg, eps=0.0,
                beta=0.5)
    assert np.array_equal(a, np.zeros_like(a))


@pytest.mark.parametrize("beta", [0.0, 1.0])
@pytest.mark.parametrize("path,prec,cfg", PATHS, ids=[p[0] for p in PATHS])
def test_restitution_extremes(nbm, orc, path, prec, cfg, beta):
    n = 2500
    x, v, m, R, gam = _cloud(n, 43)
    a = _forces(nbm, x, v, m, R, gam, prec, cfg, eps=0.003, beta=beta)
    ref = orc.forces(x, v, m, R, gam, G=1.0, eps=0.003, beta=beta)
    assert rms_rel(a, ref) <= (1e-5 if prec == 32 else 1e-12)


@pytest.mark.parametrize("path,prec,cfg", PATHS, ids=[p[0] for p in PATHS])
def test_contact_term_alone(nbm, orc, path, prec, cfg):
    """G = 0: only Eqs. 5/6 act (and every element without an overlap has
    exactly zero acceleration)."""
    n = 2500
    x, v, m, R, gam = _cloud(n, 47)
    a = _forces(nbm, x, v, m, R, gam, prec, cfg, G=0.0, eps=0.003, beta=0.5)
    ref = orc.forces(x, v, m, R, gam, G=0.0, eps=0.003, beta=0.5)
    assert np.any(ref != 0.0)
    assert np.array_equal(a[np.all(ref == 0.0, axis=1)], np.zeros((int(np.sum(
        np.all(ref == 0.0, axis=1))), 3)))
    assert rms_rel(a, ref) <= (1e-5 if prec == 32 else 1e-12)


@pytest.mark.parametrize("path,prec,cfg", PATHS, ids=[p[0] for p in PATHS])
def test_equal_mass_binary(nbm, orc, path, prec, cfg):
    """q = 1: every element carries the same mass; forces at step 0 and
    positions after 20 steps against the oracle."""
    desc = dict(n_donor=2048, n_accretor=2048, q=1.0, f_donor=0.9, f_accretor=0.9,
                sigma_v=1e-3, seed=9, stream=0, expand_rate=0.0, expand_steps=-1)
    params = dict(eps=0.005, dt=5e-4, beta=0.5, G=1.0, kappa_gamma=8.0, rl_coeff=0.69,
                  force_prec=prec)
    with nbm.System(nbm.nb_desc_default(**desc), nbm.nb_params_default(**params)) as s:
        if cfg is not None:
            s.set_pair_cfg(*cfg)
        a0 = s.forces()
        s.step(20)
        s.sync()
        xv, _, _ = s.get_state()
    ox, ov, om, oR, og = oracle_ic(orc, desc, params)
    ref = orc.forces(ox, ov, om, oR, og, G=1.0, eps=0.005, beta=0.5)
    assert rms_rel(a0, ref) <= (1e-5 if prec == 32 else 1e-12)
    rx, _, _ = orc.run(ox, ov, om, oR, og, G=1.0, eps=0.005, beta=0.5, dt=5e-4, nsteps=20,
                       n_donor=2048, grow_f0=0.9)
    assert np.abs(xv[:, :3] - rx).max() <= (1e-4 if prec == 32 else 1e-9)
