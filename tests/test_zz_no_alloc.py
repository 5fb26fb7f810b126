"""mh_pair_eval_noalloc: the evaluation with no device allocation.

Some callers may not call cudaMalloc at all (a solver embedded in a host
application that owns every byte of device memory, or a latency-critical loop
that cannot take an allocation's implicit synchronisation).  This entry point
serves them from a fixed scratch array inside the library.  The test calls it
through the C ABI twice in a row, on different inputs, and compares each
result with mh_pair_eval's at the tolerances of the other parity tests.  It
lives in its own file, named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from helpers import kepler_traj, rel_rows
from paper_2006_02501_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_02501_gb300.build import build
    build()
    from paper_2006_02501_gb300 import _capi
    return _capi.lib()


def _call(fn, P, prec, m, traj, eps, i0=0, i1=None):
    N = len(m)
    i1 = N if i1 is None else i1
    rows = np.ascontiguousarray(traj[:, :P + 1].transpose(1, 2, 0).reshape((P + 1) * 3, N))
    dm = torch.from_numpy(np.ascontiguousarray(m)).cuda()
    dr = torch.from_numpy(rows).cuda()
    out = torch.full(((P + 1) * 3, i1 - i0), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(P, prec, N, dm.data_ptr(), dr.data_ptr(), eps, 1.0, i0, i1, out.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy().reshape(P + 1, 3, i1 - i0).transpose(2, 0, 1)


CASES = [  # (P, precision, tolerance on a, on the higher derivatives)
    (3, 0, 1e-12, 1e-12),
    (5, 0, 1e-12, 1e-12),
    (3, 1, 2e-6, 5e-5),
]


@pytest.mark.parametrize("P,prec,tol_a,tol_k", CASES)
def test_noalloc_matches_allocating_entry_point_twice(L, P, prec, tol_a, tol_k):
    for call, (seed, N, i0, i1) in enumerate([(21, 3000, 0, 3001), (22, 1700, 100, 900)]):
        m, x, v = I.smbh_disc(seed=seed, N=N)
        traj = kepler_traj(m, x, v, min(P, 3))
        if P > 3:
            rng = np.random.default_rng(seed)
            traj = np.concatenate([traj, rng.normal(size=(len(m), P - 3, 3))], axis=1)
        rc_ref, ref = _call(L.mh_pair_eval, P, prec, m, traj, 1e-4, i0, i1)
        rc, got = _call(L.mh_pair_eval_noalloc, P, prec, m, traj, 1e-4, i0, i1)
        assert rc_ref == 0 and rc == 0, (call, L.mh_last_error())
        assert np.all(np.isfinite(got))
        assert rel_rows(got[:, 0], ref[:, 0]) < tol_a, call
        for k in range(1, P + 1):
            assert rel_rows(got[:, k], ref[:, k], 1e-6) < tol_k, (call, k)


def test_noalloc_shrinks_the_split_to_fit(L):
    """A problem whose normal plan does not fit the fixed scratch: the precision
    form on 400000 bodies (its FP32 input rows take 30 MB of the 32 MiB) for
    2000 bodies, whose j-split must shrink from the planner's to at most 16 slots
    of 192 KB.  The result still matches mh_pair_eval's, twice in a row."""
    m, x, v = I.smbh_disc(seed=23, N=399999)
    traj = kepler_traj(m, x, v, 3)
    for i0 in (1000, 250000):
        rc_ref, ref = _call(L.mh_pair_eval, 3, 1, m, traj, 1e-4, i0, i0 + 2000)
        rc, got = _call(L.mh_pair_eval_noalloc, 3, 1, m, traj, 1e-4, i0, i0 + 2000)
        assert rc_ref == 0 and rc == 0, L.mh_last_error()
        assert rel_rows(got[:, 0], ref[:, 0]) < 2e-6
        for k in range(1, 4):
            assert rel_rows(got[:, k], ref[:, k], 1e-6) < 5e-5, k


def test_noalloc_matches_oracle(L, orc):
    """The allocation-free path against the CPU oracle directly (FP64, P = 3, a
    range of bodies that spans several i-tiles with a ragged end), at 1e-12."""
    m, x, v = I.smbh_disc(seed=24, N=2999)
    traj = kepler_traj(m, x, v, 3)
    rc, got = _call(L.mh_pair_eval_noalloc, 3, 0, m, traj, 1e-4, 37, 1337)
    assert rc == 0, L.mh_last_error()
    ref = orc.evaluate(m, traj, 1e-4, i0=37, i1=1337)
    for k in range(4):
        assert rel_rows(got[:, k], ref[:, k], 1e-6) < 1e-12, k


def test_noalloc_rejects_oversize_problem(L):
    # 6 * 3 * 300000 doubles of one partial-sum slot exceed the 32 MiB scratch
    p = ctypes.c_void_p(16)        # never dereferenced: the size check comes first
    rc = L.mh_pair_eval_noalloc(5, 0, 300000, p, p, 1e-4, 1.0, 0, 300000, p, None)
    assert rc == -1
    assert b"32 MiB" in L.mh_last_error()
