"""The allocation-free pair-term entry point (nb_pair_forces_noalloc).

It exists for callers that may not allocate device memory (a host framework
that owns the device memory through its own pool, a latency-critical thread
that may not block on the device-wide synchronisation of cudaFree).  Its
scratch is a fixed array inside the library, shared by every call, so the
test makes calls in a row -- with different sizes, so that anything left
over from one call would show in the next -- and checks each against the
FP64 oracle's pair term (Eq. 4 with the contact term off: zero radii and
strengths) within the FP32 pair-term tolerance of the other tests, at the
edges of the scratch (n = 1, 2 and NB_NOALLOC_MAX_N) and in between.  It
also checks the result against the library's own entry point (nb_forces of
a system with the contact term off), that a repeated call gives the same
bits, and that calls after the first leave the device's free memory as it
was.  The buffers are allocated by the test, not by the library.
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


def _oracle(orc, x, v, m):
    """Eq. 4 alone in FP64: every element with zero radius and strength, so
    no pair is in contact."""
    n = len(m)
    return orc.forces(x, v, m, np.zeros(n), np.zeros(n), G=G, eps=EPS, beta=1.0)


def _library(nbm, x, v, m):
    """The same pair term from the existing entry point: a system holding
    these elements with zero radii and the contact term switched off."""
    n = len(m)
    desc = nbm.nb_desc_default(n_donor=n // 2, n_accretor=n - n // 2)
    params = nbm.nb_params_default(G=G, eps=EPS, flags=nbm.NB_GRAVITY_ONLY)
    mrg = np.stack([m, np.zeros(n), np.zeros(n)], 1)
    with nbm.System(desc, params, xv_in=np.concatenate([x, v], 1), mrg_in=mrg) as s:
        return s.forces()


@pytest.fixture(scope="module")
def nbm():
    pytest.importorskip("torch")
    from paper_2303_12166_gb300 import build
    build.build()
    from paper_2303_12166_gb300 import nbody
    return nbody


def _call(torch, nbm, xyzm, n, stream):
    acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    # the NaN fill runs on torch's stream; the call runs on `stream`
    torch.cuda.synchronize()
    nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
    return acc.cpu().numpy()


def test_noalloc_matches_oracle_at_its_edges(nbm, orc):
    import torch
    stream = torch.cuda.Stream()
    got = {}
    sizes = [(nbm.NB_NOALLOC_MAX_N, 7), (2, 8), (3000, 5), (1, 9), (1029, 6)]
    for n, seed in sizes:
        x, v, m = _elements(n, seed)
        xyzm = torch.tensor(np.concatenate([x, m[:, None]], 1), dtype=torch.float64,
                            device="cuda")
        a = _call(torch, nbm, xyzm, n, stream)
        assert np.all(np.isfinite(a))
        if n == 1:
            assert np.all(a == 0.0)
        else:
            ref = _oracle(orc, x, v, m)
            assert rms_rel(a, ref) <= 1e-5
            assert np.abs(a - ref).max() <= 50 * 1e-5 * np.abs(ref).max()
        got[n] = (xyzm, a, (x, v, m))

    # the existing entry point gives the same pair term
    x, v, m = got[3000][2]
    assert rms_rel(got[3000][1], _library(nbm, x, v, m)) <= 1e-5

    # the largest size again, after the smaller ones: the same bits
    n = nbm.NB_NOALLOC_MAX_N
    xyzm, a0, _ = got[n]
    assert np.array_equal(_call(torch, nbm, xyzm, n, stream), a0)


def test_noalloc_calls_leave_free_memory_unchanged(nbm):
    """After the first call on the device (which loads the library's device
    code and places its scratch array), later calls take no device memory."""
    import torch
    stream = torch.cuda.Stream()
    n = 5000
    x, v, m = _elements(n, 11)
    xyzm = torch.tensor(np.concatenate([x, m[:, None]], 1), dtype=torch.float64, device="cuda")
    acc = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
    free = []
    for _ in range(3):
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
    assert len(set(free)) == 1, free


def test_noalloc_rejects_sizes_beyond_its_scratch(nbm):
    import torch
    big = nbm.NB_NOALLOC_MAX_N + 1
    xyzm = torch.zeros((big, 4), dtype=torch.float64, device="cuda")
    acc = torch.zeros((big, 3), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(nbm.NbError) as ei:
        nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), big, G, EPS, acc.data_ptr())
    assert ei.value.status == nbm.NB_EINVAL
    assert "outside" in str(ei.value)


def test_noalloc_refuses_a_capturing_stream(nbm):
    """The call ends with a copy to host memory and a stream synchronisation,
    neither of which a stream capture allows: it refuses a stream that is
    capturing instead of breaking the caller's capture."""
    import torch
    n = 64
    xyzm = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    xyzm[:, 3] = 1.0
    acc = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    # the first call (device code loaded, scratch address looked up) is made
    # before any capture
    nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=stream):
        try:
            nbm.nb_pair_forces_noalloc(xyzm.data_ptr(), n, G, EPS, acc.data_ptr(), stream)
        except nbm.NbError as e:
            refused = e
    assert refused is not None and refused.status == nbm.NB_EINVAL
    assert "captur" in str(refused)
