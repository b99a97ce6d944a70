"""FP64 CPU oracle of the element model (arXiv:2303.12166) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``nb_oracle.c`` (plain C,
FP64, no fast-math); this wrapper compiles it with gcc, loads it with ctypes
and adds the O(N) diagnostics in plain numpy.

Each function names the passage of the paper it follows:

* ``roche_rL``        -- Eq. 3 (coefficient printed as 0.69).
* ``roche_phi``       -- Eq. 2, read as Kopal's normalised Roche potential.
* ``roche_L1``        -- inner Lagrangian point, the zero of dphi/dx (Eq. 2).
* ``lens_V``/``lens_U`` -- bracket of Eqs. 5/6 (read with r^3/12) and its
  potential.
* ``forces``          -- Eqs. 4-6 by direct summation.
* ``run``             -- leap-frog (kick-drift-kick) with donor expansion
  (methodology section: radius of the donor's elements grows).
* ``make_ic``         -- element mass and radius from the star's mass, radius
  and element count (methodology section); star radius from Eq. 3.
* ``diagnostics``     -- energies, momentum, angular momentum, centres of
  mass, donor elements past the L1 plane.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libnb_oracle.so")
_lock = threading.Lock()
_lib = None
_LIB_OVERRIDE = None  # set on a separately loaded copy of this module (see load_variant)


def load_variant(lib_path: str):
    """A separate instance of this module bound to another compiled oracle
    library (used by the tests that plant mistakes in copies of the oracle)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(f"oracle_variant_{abs(hash(lib_path))}",
                                                  os.path.abspath(__file__))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB_OVERRIDE = lib_path
    return mod

_D = ctypes.c_double
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_P = ctypes.c_void_p


def compile_source(src: str, lib_path: str) -> str:
    """Compile a C file with the oracle's flags into a shared library."""
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           "-shared", "-fPIC", "-std=c99", "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


def build(force: bool = False) -> str:
    """Compile nb_oracle.c into oracle/_build/libnb_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build() if _LIB_OVERRIDE is None else _LIB_OVERRIDE)
        lib.orc_roche_rL.restype = _D
        lib.orc_roche_rL.argtypes = [_D, _D]
        lib.orc_roche_phi.restype = _D
        lib.orc_roche_phi.argtypes = [_D, _D, _D, _D]
        lib.orc_roche_L1.restype = _D
        lib.orc_roche_L1.argtypes = [_D]
        lib.orc_lens_V.restype = _D
        lib.orc_lens_V.argtypes = [_D, _D]
        lib.orc_lens_U.restype = _D
        lib.orc_lens_U.argtypes = [_D, _D]
        lib.orc_donor_scale.restype = _D
        lib.orc_donor_scale.argtypes = [_I64, _D, _D, _I64]
        lib.orc_forces.restype = None
        lib.orc_forces.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _D, _D, _P]
        lib.orc_forces_rows.restype = None
        lib.orc_forces_rows.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _D, _D, _I64, _P, _P]
        lib.orc_potential.restype = None
        lib.orc_potential.argtypes = [_I64, _P, _P, _P, _P, _D, _D, _P, _P]
        lib.orc_run.restype = None
        lib.orc_run.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _D, _D, _D, _D,
                                _I64, _I64, _D, _D, _I64, _P, _P, _P]
        lib.orc_make_ic.restype = None
        lib.orc_make_ic.argtypes = [_I64, _I64, _D, _D, _D, _D, _D, _U64, _U64,
                                    ctypes.c_int, _D, _D, _D, _D, _P, _P, _P, _P, _P]
        lib.orc_splitmix_u01.restype = None
        lib.orc_splitmix_u01.argtypes = [_U64, _U64, _I64, _P]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_set_threads.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    """Set the OpenMP thread count used by the O(N^2) loops."""
    _load().orc_set_threads(int(n))


# ---------------------------------------------------------------- Roche geometry
def roche_rL(q: float, coeff: float = 0.69) -> float:
    """Eq. 3: Roche-lobe radius (units of a) for mass ratio q (this star / companion)."""
    return float(_load().orc_roche_rL(float(q), float(coeff)))


def roche_phi(q: float, x: float, y: float, z: float) -> float:
    """Eq. 2 (Kopal form): m1 at origin, m2 at (1,0,0), q = m2/m1, corotating frame."""
    return float(_load().orc_roche_phi(float(q), float(x), float(y), float(z)))


def roche_L1(q: float) -> float:
    """Inner Lagrangian point: distance from m1 (origin) toward m2, units of a."""
    return float(_load().orc_roche_L1(float(q)))


# ---------------------------------------------------------------- contact term
def lens_V(r: float, R: float) -> float:
    """Bracket of Eqs. 5/6 times pi: overlap volume pi(4/3R^3 - R^2 r + r^3/12)."""
    return float(_load().orc_lens_V(float(r), float(R)))


def lens_U(r: float, R: float) -> float:
    """Integral of lens_V from r to 2R: pi(R^4 - 4/3R^3 r + R^2 r^2/2 - r^4/48)."""
    return float(_load().orc_lens_U(float(r), float(R)))


def donor_scale(k: int, f0: float, rate: float, cap: int) -> float:
    """Donor element radius at step k over its initial value: (f0+rate*min(k,cap))/f0."""
    return float(_load().orc_donor_scale(int(k), float(f0), float(rate), int(cap)))


# ---------------------------------------------------------------- Eqs. 4-6
def forces(x, v, m, R, gam, G=1.0, eps=0.0, beta=1.0):
    """Eqs. 4-6: FP64 accelerations (n,3) by direct summation over all j != i."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    v = _f64(v, (n, 3))
    m = _f64(m, (n,))
    R = _f64(R, (n,))
    gam = _f64(gam, (n,))
    a = np.zeros((n, 3), dtype=np.float64)
    _load().orc_forces(n, _ptr(x), _ptr(v), _ptr(m), _ptr(R), _ptr(gam),
                       float(G), float(eps), float(beta), _ptr(a))
    return a


def forces_rows(rows, x, v, m, R, gam, G=1.0, eps=0.0, beta=1.0):
    """Eqs. 4-6 for the listed elements only: (len(rows), 3)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    v = _f64(v, (n, 3))
    m = _f64(m, (n,))
    R = _f64(R, (n,))
    gam = _f64(gam, (n,))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise IndexError("row out of range")
    a = np.zeros((rows.size, 3), dtype=np.float64)
    _load().orc_forces_rows(n, _ptr(x), _ptr(v), _ptr(m), _ptr(R), _ptr(gam), float(G),
                            float(eps), float(beta), rows.size, _ptr(rows), _ptr(a))
    return a


def potential(x, m, R, gam, G=1.0, eps=0.0):
    """Per-element shares of E_grav and E_rep; their sums are the pair energies."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    m = _f64(m, (n,))
    R = _f64(R, (n,))
    gam = _f64(gam, (n,))
    eg = np.zeros(n)
    er = np.zeros(n)
    _load().orc_potential(n, _ptr(x), _ptr(m), _ptr(R), _ptr(gam), float(G),
                          float(eps), _ptr(eg), _ptr(er))
    return eg, er


# ---------------------------------------------------------------- leap-frog
def run(x, v, m, R0, gam, *, G=1.0, eps=0.0, beta=1.0, dt=1e-3, nsteps=1,
        k0=0, n_donor=0, grow_f0=1.0, grow_rate=0.0, grow_cap=-1, a0=None):
    """Kick-drift-kick leap-frog for ``nsteps`` steps from step index ``k0``.

    Donor elements (indices < n_donor) have radius R0 * donor_scale(k).
    Returns (x, v, a) at step k0 + nsteps as new arrays.
    """
    x = _f64(x, (-1, 3)).copy()
    n = x.shape[0]
    v = _f64(v, (n, 3)).copy()
    m = _f64(m, (n,))
    R0 = _f64(R0, (n,))
    gam = _f64(gam, (n,))
    a = np.zeros((n, 3))
    work = np.zeros(4 * n)
    a_in = None if a0 is None else _f64(a0, (n, 3))
    _load().orc_run(n, int(n_donor), _ptr(x), _ptr(v), _ptr(m), _ptr(R0), _ptr(gam),
                    float(G), float(eps), float(beta), float(dt), int(k0), int(nsteps),
                    float(grow_f0), float(grow_rate), int(grow_cap),
                    None if a_in is None else _ptr(a_in), _ptr(a), _ptr(work))
    return x, v, a


# ---------------------------------------------------------------- initial conditions
def make_ic(n_donor, n_accretor, q, *, sep=1.0, f_donor=0.8, f_accretor=0.5,
            sigma_v=1e-3, seed=0, stream=0, no_spin=False, G=1.0, kappa_gamma=8.0,
            rl_coeff=0.69, ecc=0.0):
    """Two uniform spheres of equal-mass elements starting at periapsis of an
    orbit of semi-major axis ``sep`` and eccentricity ``ecc`` (see nb_oracle.c)."""
    n = int(n_donor) + int(n_accretor)
    x = np.zeros((n, 3))
    v = np.zeros((n, 3))
    m = np.zeros(n)
    R = np.zeros(n)
    gam = np.zeros(n)
    _load().orc_make_ic(int(n_donor), int(n_accretor), float(q), float(sep),
                        float(f_donor), float(f_accretor), float(sigma_v),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream) & 0xFFFFFFFFFFFFFFFF,
                        1 if no_spin else 0, float(G), float(kappa_gamma),
                        float(rl_coeff), float(ecc), _ptr(x), _ptr(v), _ptr(m), _ptr(R),
                        _ptr(gam))
    return x, v, m, R, gam


def splitmix_u01(seed, stream, n):
    out = np.zeros(int(n))
    _load().orc_splitmix_u01(int(seed) & 0xFFFFFFFFFFFFFFFF,
                             int(stream) & 0xFFFFFFFFFFFFFFFF, int(n), _ptr(out))
    return out


# ---------------------------------------------------------------- diagnostics
def diagnostics(x, v, m, R, gam, *, G=1.0, eps=0.0, n_donor=0, q=None, rl_L1=None):
    """FP64 diagnostics of a state.

    E_kin = 1/2 sum m v^2; E_grav = -sum_{i<j} G m_i m_j/(r+eps) (Eq. 4's
    potential); E_rep = sum_{contacts} gamma_ij U(r; R_ij) (potential of the
    Eq. 5 repulsion); P = sum m v; L = sum m x cross v; centres of mass of the
    whole system and of each star's original elements.  With ``q`` given
    (donor mass / accretor mass), for the donor's elements:

    * ``n_past_L1``/``m_past_L1``: on the accretor's side of the plane through
      L1 (Eq. 2) normal to the line between the star centres;
    * ``n_in_acc_lobe``/``m_in_acc_lobe``: inside the accretor's Roche lobe,
      i.e. on that side of the plane with phi >= phi(L1), phi the normalised
      potential of Eq. 2 in the frame with the accretor's centre at the
      origin, the donor's at x = 1 (the current separation as unit), z along
      the orbital axis +z;
    * ``n_unbound``/``m_unbound``: with positive energy per unit mass in the
      field of the two stars taken as point masses at their centres,
      1/2 |v - v_cm|^2 - G M_a/|x - c_a| - G M_d/|x - c_d| > 0.
    """
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    v = _f64(v, (n, 3))
    m = _f64(m, (n,))
    eg, er = potential(x, m, R, gam, G=G, eps=eps)
    out = {
        "E_kin": float(0.5 * np.sum(m * np.sum(v * v, axis=1))),
        "E_grav": float(np.sum(eg)),
        "E_rep": float(np.sum(er)),
        "P": (m[:, None] * v).sum(axis=0),
        "L": (m[:, None] * np.cross(x, v)).sum(axis=0),
        "com": (m[:, None] * x).sum(axis=0) / m.sum(),
    }
    out["E_tot"] = out["E_kin"] + out["E_grav"] + out["E_rep"]
    nd = int(n_donor)
    if 0 < nd < n:
        cd = (m[:nd, None] * x[:nd]).sum(axis=0) / m[:nd].sum()
        ca = (m[nd:, None] * x[nd:]).sum(axis=0) / m[nd:].sum()
        out["com_donor"] = cd
        out["com_accretor"] = ca
        d = cd - ca
        sep = float(np.sqrt(d @ d))
        out["separation"] = sep
        if q is not None:
            xl1 = roche_L1(q) if rl_L1 is None else rl_L1
            proj = (x[:nd] - ca) @ (d / sep)
            past = proj < xl1 * sep
            out["n_past_L1"] = int(past.sum())
            out["m_past_L1"] = float(m[:nd][past].sum())
            # Roche frame: x along the axis, z the orbital axis, y = z cross x
            ex = d / sep
            ez = np.array([0.0, 0.0, 1.0]) - ex[2] * ex
            ez = ez / np.sqrt(ez @ ez)
            ey = np.cross(ez, ex)
            rel = (x[:nd] - ca) / sep
            phi_c = roche_phi(q, xl1, 0.0, 0.0)
            inlobe = np.zeros(nd, dtype=bool)
            for k in range(nd):
                xi, yi, zi = rel[k] @ ex, rel[k] @ ey, rel[k] @ ez
                if xi < xl1:
                    inlobe[k] = roche_phi(q, xi, yi, zi) >= phi_c
            out["n_in_acc_lobe"] = int(inlobe.sum())
            out["m_in_acc_lobe"] = float(m[:nd][inlobe].sum())
            Ma, Md = m[nd:].sum(), m[:nd].sum()
            vcm = (m[:, None] * v).sum(axis=0) / m.sum()
            dv = v[:nd] - vcm
            ra = np.linalg.norm(x[:nd] - ca, axis=1)
            rd = np.linalg.norm(x[:nd] - cd, axis=1)
            with np.errstate(divide="ignore"):  # an element at a centre is bound
                e = 0.5 * np.sum(dv * dv, axis=1) - G * Ma / ra - G * Md / rd
            unb = e > 0
            out["n_unbound"] = int(unb.sum())
            out["m_unbound"] = float(m[:nd][unb].sum())
    return out
