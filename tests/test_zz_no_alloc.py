"""The allocation-free pair-term entry point (nb_pair_forces_noalloc).

It exists for callers that may not allocate device memory (a host framework
that owns the device memory through its own pool, a latency-critical thread
that may not block on the device-wide synchronisation of cudaFree).  Its
scratch is a fixed array inside the library, shared by every call, so the
test makes two calls in a row -- with different sizes, so that anything left
over from the first call would show in the second -- and checks each against
the existing entry point (nb_forces of a system with the contact term off)
within the FP32 pair-term tolerance of the other tests.  The buffers are
allocated by the test, not by the library.
"""
import numpy as np
import pytest

import synth
from nbtest import rms_rel

pytestmark = pytest.mark.gpu

G, EPS = 1.3, 0.004


def _elements(n, seed):
    x, v = synth.cloud(n, seed, radius=0.4)
    m = 0.5 + synth.u01(seed, 3, n)
    return x, v, m


def _reference(nbm, x, v, m):
    """Pair term from the existing entry point: a system holding these
    elements with zero radii and the contact term switched off."""
    n = len(m)
    desc = nbm.nb_desc_default(n_donor=n // 2, n_accretor=n - n // 2)
    params = nbm.nb_params_default(G=G, eps=EPS, flags=nbm.NB_GRAVITY_ONLY)
    mrg = np.stack([m, np.zeros(n), np.zeros(n)], 1)
    with nbm.System(desc, params, xv_in=np.concatenate([x, v], 1), mrg_in=mrg) as s:
        return s.forces()


def test_noalloc_matches_existing_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody as nbm

    stream = torch.cuda.Stream()
    got = []
    for n, seed in [(3000, 5), (1029, 6)]:
        x, v, m = _elements(n, seed)
        ref = _reference(nbm, x, v, m)
        xyzm = torch.tensor(np.concatenate([x, m[:, None]], 1), dtype=torch.float64,
                            device="cuda")
        acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
        a = acc.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rms_rel(a, ref) <= 1e-5
        got.append((n, xyzm, a))

    # the first size again: same result, bit for bit
    n, xyzm, a0 = got[0]
    acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
    assert np.array_equal(acc.cpu().numpy(), a0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2303_12166_gb300 import nbody as nbm
    big = nbm.NB_NOALLOC_MAX_N + 1
    xyzm = torch.zeros((big, 4), dtype=torch.float64, device="cuda")
    acc = torch.zeros((big, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(nbm.NbError) as ei:
        nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), big, G, EPS, acc.data_ptr())
    assert ei.value.status == nbm.NB_EINVAL
    assert "outside" in str(ei.value)
