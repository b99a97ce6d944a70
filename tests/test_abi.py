"""The C ABI library loads and exports every entry point include/nbody.h
declares; host-only calls behave; without a GPU the compute calls fail
loudly (no CPU fallback)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(nb_[A-Za-z0-9_]+)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2303_12166_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(lib_path):
    names = _declared()
    assert {"nb_create_system", "nb_step", "nb_forces", "nb_diagnostics"} <= names
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_calls(lib_path, orc):
    from paper_2303_12166_gb300 import nbody as nbm
    assert nbm.nb_abi_version() == 1
    assert nbm.nb_status_str(nbm.NB_EINVAL) == "invalid argument"
    p = nbm.nb_params_default()
    assert (p.G, p.eps, p.dt, p.beta, p.kappa_gamma, p.rl_coeff, p.force_prec) == \
        (1.0, 0.01, 1e-3, 0.5, 8.0, 0.69, 32)
    d = nbm.nb_desc_default()
    assert (d.n_donor, d.n_accretor, d.q) == (512, 512, 0.5)
    # the library's Eq. 3 and L1 agree with the oracle's
    for q in [0.1, 0.2, 0.3, 0.5, 1.0, 2.0, 5.0]:
        assert nbm.nb_roche_rL(q) == pytest.approx(orc.roche_rL(q), rel=1e-14)
        assert nbm.nb_roche_L1(q) == pytest.approx(orc.roche_L1(q), abs=1e-14)


def test_pair_variant_table(lib_path):
    """The variant table is readable without a GPU and every entry respects
    the slot split: Newton-Raphson plus shared-reciprocal slots <= i per
    thread, the shared reciprocal only on the j-packed kernel, and the
    symmetric kernel without Newton-Raphson reciprocals and with
    whole tiles per block."""
    from paper_2303_12166_gb300 import nbody as nbm
    v = nbm.nb_pair_cfg_variants()
    assert len(v) >= 20 and len(set(v)) == len(v)
    assert any(c[7] for c in v) and any(not c[7] for c in v)
    for tile, bi, nt, minb, nr, ipk, shr, sym in v:
        assert tile in (64, 128, 256) and nt % 32 == 0 and minb >= 1
        assert nr >= 0 and shr >= 0 and (nr * (2 if ipk else 1) + shr) <= bi
        assert not (ipk and shr)
        if sym:
            assert nr == 0 and not (ipk and shr) and (nt * bi) % tile == 0
    with pytest.raises(nbm.NbError) as ei:
        nbm._check(nbm._lib.nb_pair_cfg_variants(None, 1, ctypes.byref(nbm._I32())), "x")
    assert ei.value.status == nbm.NB_EINVAL


def test_invalid_parameters_rejected(lib_path):
    from paper_2303_12166_gb300 import nbody as nbm
    cases = [dict(dt=0.0), dict(beta=1.5), dict(eps=-1.0), dict(force_prec=16)]
    for bad in cases:
        with pytest.raises(nbm.NbError) as ei:
            nbm.nb_create_system(nbm.nb_desc_default(), nbm.nb_params_default(**bad))
        assert ei.value.status == nbm.NB_EINVAL
    for bad in [dict(n_donor=0, n_accretor=0), dict(q=0.0), dict(f_donor=-1.0),
                dict(expand_rate=-1e-3, expand_steps=-1)]:
        with pytest.raises(nbm.NbError) as ei:
            nbm.nb_create_system(nbm.nb_desc_default(**bad), nbm.nb_params_default())
        assert ei.value.status == nbm.NB_EINVAL


def test_no_gpu_fails_loudly(lib_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2303_12166_gb300 import nbody as nbm
    with pytest.raises(nbm.NbError) as ei:
        nbm.nb_create_system(nbm.nb_desc_default(n_donor=8, n_accretor=8), nbm.nb_params_default())
    assert ei.value.status in (nbm.NB_ECUDA, nbm.NB_ENOMEM)


def test_caller_arrays_are_size_checked_before_the_call():
    """Arrays handed to the library by pointer must hold exactly n rows: the
    binding refuses other sizes before calling (no handle or GPU needed)."""
    import numpy as np
    from paper_2303_12166_gb300 import nbody as nbm
    desc = nbm.nb_desc_default(n_donor=40, n_accretor=24)
    params = nbm.nb_params_default()
    with pytest.raises(ValueError):
        nbm.nb_create_system(desc, params, xv_in=np.zeros((63, 6)))
    with pytest.raises(ValueError):
        nbm.nb_create_system(desc, params, mrg_in=np.zeros((64, 2)))
    with pytest.raises(ValueError):
        nbm.nb_submit(None, desc, params, 1, xv_in=np.zeros(64 * 6 + 1))
    with pytest.raises(ValueError):  # a valid xv_in with a bad mrg_in
        nbm.nb_create_system(desc, params, xv_in=np.zeros((64, 6)), mrg_in=np.zeros(5))
    # the descriptor keeps no pointer after a refused call
    assert not desc.xv_in and not desc.mrg_in


CASES_IC = [
    (dict(n_donor=512, n_accretor=512, q=0.5, f_donor=0.8, f_accretor=0.5, sigma_v=1e-3,
          seed=0, stream=0), dict()),
    (dict(n_donor=300, n_accretor=120, q=0.25, f_donor=0.95, f_accretor=0.3, sigma_v=3e-3,
          seed=7, stream=4, ecc=0.4), dict(kappa_gamma=5.0, rl_coeff=0.6, flags=2)),
    (dict(n_donor=3, n_accretor=0, q=2.0, f_donor=0.5, f_accretor=0.5, sigma_v=0.0,
          seed=1, stream=0), dict(G=0.7)),
]


@pytest.mark.parametrize("desc,params", CASES_IC)
def test_library_initial_state_matches_the_oracle(orc, desc, params):
    """The library's host-side initial-condition recipe (no GPU) against the
    oracle's, element by element."""
    from paper_2303_12166_gb300 import nbody as nbm
    xv, mrg = nbm.nb_initial_state(nbm.nb_desc_default(**desc), nbm.nb_params_default(**params))
    p = nbm.nb_params_default(**params)
    ox, ov, om, oR, og = orc.make_ic(desc["n_donor"], desc["n_accretor"], desc["q"],
                                     f_donor=desc["f_donor"], f_accretor=desc["f_accretor"],
                                     sigma_v=desc["sigma_v"], seed=desc["seed"],
                                     stream=desc["stream"], G=p.G, kappa_gamma=p.kappa_gamma,
                                     rl_coeff=p.rl_coeff, ecc=desc.get("ecc", 0.0),
                                     no_spin=bool(p.flags & 2))
    assert np.abs(xv[:, :3] - ox).max() < 1e-14
    assert np.abs(xv[:, 3:] - ov).max() < 1e-14
    assert np.allclose(mrg[:, 0], om, rtol=1e-15, atol=0)
    assert np.allclose(mrg[:, 1], oR, rtol=1e-14, atol=0)
    assert np.allclose(mrg[:, 2], og, rtol=1e-13, atol=0)


def test_initial_state_refuses_invalid_descriptions():
    from paper_2303_12166_gb300 import nbody as nbm
    with pytest.raises(nbm.NbError) as ei:
        nbm.nb_initial_state(nbm.nb_desc_default(q=-1.0), nbm.nb_params_default())
    assert ei.value.status == nbm.NB_EINVAL
    with pytest.raises(ValueError):
        nbm.nb_initial_state(nbm.nb_desc_default(n_donor=0, n_accretor=0),
                             nbm.nb_params_default())


def test_binding_covers_every_declared_entry_point():
    """The Python binding marshals every call include/nbody.h declares (it
    adds no computation of its own: each wrapper ends in the library call)."""
    src = open(os.path.join(ROOT, "paper_2303_12166_gb300", "nbody.py")).read()
    missing = [n for n in sorted(_declared()) if f'"{n}"' not in src and f"_lib.{n}" not in src]
    assert not missing, missing
