"""A single system split by element rows over two "devices", run through the
library on one GPU.

The schedule is the multi-GPU layout of a single system: each rank owns the
contiguous rows `dist.row_range` gives it, kicks and drifts them, the ranks
all-gather positions and velocities once per step after the drift (the pair
term needs every x_j, the contact test every v_j), and each rank evaluates
the accelerations of its own rows against all n elements with
`nb_forces_rows`.  Here the two ranks are two handles of the same system on
one GPU, the all-gather is a host concatenation written into both handles
with `nb_set_state`, and the kicks and drifts are the update's FP64
arithmetic (v + (dt/2) a, x + dt v, no fused multiply-add) on the host.

The result must be the single-system trajectory of `nb_step` bit for bit:
every row's acceleration comes from the same work items as in a full pass
(the one-sided kernel's partial slots, or the symmetric kernel's integer
fixed-point sums, whose value does not depend on which items ran in which
order).
"""
import numpy as np
import pytest

from paper_2303_12166_gb300.dist import row_range

pytestmark = pytest.mark.gpu

DESC = dict(n_donor=4500, n_accretor=1700, q=0.35, f_donor=0.9, f_accretor=0.5,
            expand_rate=2e-3, expand_steps=-1, sigma_v=1e-3, seed=13, stream=0)
PARAMS = dict(eps=0.005, dt=5e-4, beta=0.5)
STEPS = 8
ONE_SIDED = (128, 8, 128, 2, 0, 0, 6, 0)


@pytest.fixture(scope="module")
def nbm():
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _system(nbm, cfg):
    s = nbm.System(nbm.nb_desc_default(**DESC), nbm.nb_params_default(**PARAMS))
    if cfg is not None:
        s.set_pair_cfg(*cfg)
        xv, _, meta = s.get_state()
        s.set_state(xv, None, meta)  # a^0 with this configuration
    return s


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("cfg", [None, ONE_SIDED], ids=["symmetric", "one-sided"])
def test_row_split_matches_one_system_bitwise(nbm, cfg, world):
    with _system(nbm, cfg) as ref:
        ref.step(STEPS)
        ref.sync()
        xv_ref, a_ref, meta_ref = ref.get_state()
        n = ref.n
    ranks = [_system(nbm, cfg) for _ in range(world)]
    try:
        rows = [row_range(n, world, r) for r in range(world)]
        xv, _, meta = ranks[0].get_state()
        x, v = xv[:, :3].copy(), xv[:, 3:].copy()
        hdt, dt = 0.5 * PARAMS["dt"], PARAMS["dt"]
        a = [h.forces_rows(lo, hi) for h, (lo, hi) in zip(ranks, rows)]
        zeros = np.zeros((n, 3))
        for k in range(STEPS):
            for (lo, hi), ar in zip(rows, a):
                v[lo:hi] = v[lo:hi] + hdt * ar
                x[lo:hi] = x[lo:hi] + dt * v[lo:hi]
            # all-gather of x and v: every rank holds every row of step k + 1
            meta.step = k + 1
            for h in ranks:
                h.set_state(np.concatenate([x, v], 1), zeros, meta)
            a = [h.forces_rows(lo, hi) for h, (lo, hi) in zip(ranks, rows)]
            for (lo, hi), ar in zip(rows, a):
                v[lo:hi] = v[lo:hi] + hdt * ar
    finally:
        for h in ranks:
            h.close()
    assert meta_ref.step == STEPS
    assert np.array_equal(x, xv_ref[:, :3])
    assert np.array_equal(v, xv_ref[:, 3:])
    assert np.array_equal(np.concatenate(a), a_ref)


def test_forces_rows_are_the_rows_of_a_full_evaluation(nbm):
    """Any row range, block-aligned or not, gives bit for bit the rows of
    nb_forces; a range outside 0 .. n is refused."""
    with _system(nbm, None) as s:
        full = s.forces()
        n = s.n
        for lo, hi in [(0, n), (0, 1), (n - 1, n), (1000, 1537), (3071, 4609), (17, 6000)]:
            assert np.array_equal(s.forces_rows(lo, hi), full[lo:hi]), (lo, hi)
        with pytest.raises(ValueError):
            s.forces_rows(5, 5)
        # the C entry point checks the range as well
        out = np.zeros((1, 3))
        st = nbm._lib.nb_forces_rows(nbm._P(s.h), n, n + 1, out.ctypes.data_as(nbm._P), 0)
        assert st == nbm.NB_EINVAL
