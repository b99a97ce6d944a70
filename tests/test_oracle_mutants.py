"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake into a copy of oracle/nb_oracle.c (a
wrong sign, a dropped or transposed term, a misread equation), compiles it,
and runs the pins of test_oracle_pins.py against it: at least one pin must
fail.  The numpy diagnostics of oracle/oracle.py get the same treatment
(a planted copy of the module bound to the real compiled oracle).  The
planted copies live in a temporary directory; the real oracle is untouched.
"""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "nb_oracle.c")

# (name, text in nb_oracle.c, replacement)
MUTANTS = [
    ("Eq5 bracket read as printed (r^2/12)", "r * r * r / 12.0", "r * r / 12.0"),
    ("softening added to r^2", "F = G * m[i] * m[j] / ((r + eps) * (r + eps));",
     "F = G * m[i] * m[j] / (r * r + eps * eps);"),
    ("repulsion with the wrong sign", "F -= c * gij * orc_lens_V(r, Rij);",
     "F += c * gij * orc_lens_V(r, Rij);"),
    ("beta applied while converging", "double c = (closing < 0.0) ? 1.0 : beta;",
     "double c = (closing < 0.0) ? beta : 1.0;"),
    ("pair radius summed, not averaged", "double Rij = 0.5 * (R[i] + R[j]);",
     "double Rij = (R[i] + R[j]);"),
    ("pair strength summed, not averaged", "double gij = 0.5 * (gam[i] + gam[j]);",
     "double gij = (gam[i] + gam[j]);"),
    ("force not divided by m_i", "f = F / (m[i] * r);", "f = F / r;"),
    ("x difference transposed", "double dx = x[3 * j + 0] - x[3 * i + 0];\n        double dy",
     "double dx = x[3 * i + 0] - x[3 * j + 0];\n        double dy"),
    ("full first kick", "for (i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * a[i];   /* kick  */\n"
     "        for (i = 0; i < 3 * n; ++i) x[i] += dt * v[i];",
     "for (i = 0; i < 3 * n; ++i) v[i] += dt * a[i];   /* kick  */\n"
     "        for (i = 0; i < 3 * n; ++i) x[i] += dt * v[i];"),
    ("Eq3 log of q^(2/3)", "coeff * q23 + log(1.0 + q13)", "coeff * q23 + log(1.0 + q23)"),
    ("Eq2 second term without q (as printed)", "2.0 * q / ((1.0 + q) * r2)",
     "2.0 / ((1.0 + q) * r2)"),
    ("L1 equation sign", "(1.0 + q) * mid - q;", "(1.0 + q) * mid + q;"),
    ("lens potential without r^4 term", "\n                   - r * r * r * r / 48.0);",
     ");"),
    ("donor centre at q/(1+q)", "cx_d = rp / (1.0 + q);", "cx_d = rp * q / (1.0 + q);"),
    ("periapsis rate with (1-e) squared", "(1.0 - ecc) * (1.0 - ecc) * (1.0 - ecc)));",
     "(1.0 - ecc) * (1.0 - ecc)));"),
    ("element radius N^-1/2", "Re_d = n_d > 0 ? Rs_d / cbrt((double)n_d) : 0.0;",
     "Re_d = n_d > 0 ? Rs_d / sqrt((double)n_d) : 0.0;"),
    ("coincident elements not skipped", "if (!(d2 > 0.0)) continue;               "
     "/* i == j or coincident */", "if (j == i) continue;"),
    ("potential softened on r^2", "eg -= 0.5 * G * m[i] * m[j] / (r + eps);",
     "eg -= 0.5 * G * m[i] * m[j] / sqrt(d2 + eps * eps);"),
    ("potential pairs counted twice", "eg -= 0.5 * G * m[i] * m[j] / (r + eps);",
     "eg -= G * m[i] * m[j] / (r + eps);"),
    ("repulsion energy with the wrong sign",
     "er += 0.5 * 0.5 * (gam[i] + gam[j]) * orc_lens_U(r, 0.5 * (R[i] + R[j]));",
     "er -= 0.5 * 0.5 * (gam[i] + gam[j]) * orc_lens_U(r, 0.5 * (R[i] + R[j]));"),
    ("repulsion energy with the summed radius", "orc_lens_U(r, 0.5 * (R[i] + R[j]))",
     "orc_lens_U(r, (R[i] + R[j]))"),
]


def _pins():
    spec = importlib.util.spec_from_file_location("oracle_pins", os.path.join(HERE,
                                                                             "test_oracle_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return [
        (mod.test_lens_volume_is_sphere_overlap, {}),
        (mod.test_lens_potential, {}),
        (mod.test_L1_symmetry_and_stationarity, {}),
        (mod.test_eq3_paczynski_limit, {}),
        (mod.test_eq3_form_matches_roche_lobe_volume, {"q": 0.3}),
        (mod.test_forces_zero_distance_pair, {}),
        (mod.test_forces_brute_force, {"n": 8, "seed": 4}),
        (mod.test_forces_conservation, {}),
        (mod.test_forces_gradient_of_potential, {}),
        (mod.test_softened_circular_orbit, {}),
        (mod.test_head_on_restitution_is_sqrt_beta, {}),
        (mod.test_kdk_time_reversible, {}),
        (mod.test_ic_recipe, {}),
        (mod.test_eccentric_ic_follows_kepler, {}),
    ]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_detect_planted_mistake(tmp_path, name, old, new):
    from oracle import oracle
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique for {name!r}"
    mutant = tmp_path / "nb_oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mutant), str(tmp_path / "libmutant.so"))
    orc = oracle.load_variant(lib)
    failed = []
    for fn, kw in _pins():
        try:
            fn(orc, **kw)
        except Exception as e:  # a pin failed (or the planted code broke it)
            failed.append(f"{fn.__name__}: {type(e).__name__}")
            break
    assert failed, f"no pin caught the planted mistake: {name}"


def test_control_unmodified_copy_passes_every_pin(tmp_path):
    """The harness itself: an unmodified copy compiled and loaded the same
    way passes all the pins above, so a caught mutant is caught by a pin."""
    from oracle import oracle
    copy = tmp_path / "nb_oracle_copy.c"
    copy.write_text(open(SRC).read())
    orc = oracle.load_variant(oracle.compile_source(str(copy), str(tmp_path / "libcopy.so")))
    for fn, kw in _pins():
        fn(orc, **kw)


# mistakes planted in the numpy diagnostics of oracle.py
PY_MUTANTS = [
    ("L1 plane side flipped", "past = proj < xl1 * sep", "past = proj > xl1 * sep"),
    ("L1 of the inverse mass ratio", "xl1 = roche_L1(q) if rl_L1 is None else rl_L1",
     "xl1 = roche_L1(1.0 / q) if rl_L1 is None else rl_L1"),
    ("lobe test inverted", "inlobe[k] = roche_phi(q, xi, yi, zi) >= phi_c",
     "inlobe[k] = roche_phi(q, xi, yi, zi) <= phi_c"),
    ("unbound test inverted", "unb = e > 0", "unb = e < 0"),
    ("kinetic energy without the half", '"E_kin": float(0.5 * np.sum(m * np.sum(v * v, axis=1))),',
     '"E_kin": float(np.sum(m * np.sum(v * v, axis=1))),'),
    ("angular momentum as v x x", '"L": (m[:, None] * np.cross(x, v)).sum(axis=0),',
     '"L": (m[:, None] * np.cross(v, x)).sum(axis=0),'),
    ("centre of mass unweighted", '"com": (m[:, None] * x).sum(axis=0) / m.sum(),',
     '"com": x.mean(axis=0),'),
]


def _py_pins():
    spec = importlib.util.spec_from_file_location("oracle_pins", os.path.join(HERE,
                                                                             "test_oracle_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return [mod.test_diagnostics_L1_count, mod.test_diagnostics_lobe_and_unbound,
            mod.test_diagnostics_two_body_closed_form,
            mod.test_energy_bounded_elastic_and_decreasing_inelastic]


@pytest.mark.parametrize("name,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_detect_planted_mistake_in_diagnostics(tmp_path, name, old, new):
    from oracle import oracle
    lib = oracle.build()
    src = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    assert src.count(old) == 1, f"mutation site not unique for {name!r}"
    path = tmp_path / "oracle_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_py_mutant", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB_OVERRIDE = lib
    failed = []
    for fn in _py_pins():
        try:
            fn(mod)
        except Exception as e:
            failed.append(f"{fn.__name__}: {type(e).__name__}")
            break
    assert failed, f"no pin caught the planted mistake: {name}"


def test_control_unmodified_diagnostics_pass_every_pin(tmp_path):
    from oracle import oracle
    lib = oracle.build()
    path = tmp_path / "oracle_copy.py"
    path.write_text(open(os.path.join(ROOT, "oracle", "oracle.py")).read())
    spec = importlib.util.spec_from_file_location("oracle_py_copy", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB_OVERRIDE = lib
    for fn in _py_pins():
        fn(mod)
