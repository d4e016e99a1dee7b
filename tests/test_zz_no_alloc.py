"""The allocation-free Rayleigh-Ritz entry point against the allocating one.

``pbs_small_rr_noalloc`` serves callers that cannot call cudaMalloc: its work
space is a fixed device array inside the library.  Fed with the Gram matrices
from ``pbs_gram``, its coefficients must reproduce ``pbs_rayleigh_ritz`` on
the same span, on two calls in a row (the shared array keeps the previous
call's contents, which must not leak into the next result).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pbs.Context(0) as c:
        yield c


def _span(geom, q, seed):
    r = np.random.default_rng(seed)
    # smooth-ish columns: low Fourier modes plus noise keep the Ritz values spread out
    S = r.standard_normal((q, geom.D)) + 1j * r.standard_normal((q, geom.D))
    return torch.from_numpy(np.ascontiguousarray(S)).cuda()


@pytest.mark.parametrize("q,p", [(12, 6), (30, 10), (80, 16)])
def test_noalloc_matches_rayleigh_ritz_twice(ctx, q, p):
    n = 16
    geom = pbs.Geometry(gi.rod_eps(n, n))
    k = (0.6, -0.3)
    opts = pbs.default_opts(precision=pbs.PBS_FP64)
    stream = torch.cuda.current_stream()
    for call in range(2):
        S = _span(geom, q, seed=100 + call)
        X_ref = torch.zeros((p, geom.D), dtype=torch.complex128, device="cuda")
        th_ref = ctx.rayleigh_ritz(geom, opts, k, q, S.data_ptr(), p, False, X_ref.data_ptr(), stream)
        GM = torch.zeros((q, q), dtype=torch.complex128, device="cuda")
        GA = torch.zeros((q, q), dtype=torch.complex128, device="cuda")
        ctx.gram(geom, k, q, S.data_ptr(), GM.data_ptr(), GA.data_ptr(), stream)
        C = torch.full((p, q), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        theta = torch.zeros(p, dtype=torch.float64, device="cuda")
        info = torch.full((2,), 99, dtype=torch.int32, device="cuda")
        pbs.small_rr_noalloc(GM.data_ptr(), GA.data_ptr(), q, p, C.data_ptr(), theta.data_ptr(), info.data_ptr(),
                             stream)
        torch.cuda.synchronize()
        assert info.cpu().tolist() == [0, q]
        assert np.allclose(theta.cpu().numpy(), th_ref, rtol=1e-12, atol=0)
        # C is column-major q x p on the device: row j of the (p, q) tensor is column j
        X = (C @ S)  # (p, q) @ (q, D): X[j] = sum_i C[i, j] S[i]
        assert torch.allclose(X, X_ref, rtol=0, atol=1e-10 * float(X_ref.abs().max()))


def test_noalloc_rejects_sizes_beyond_its_array(ctx):
    dummy = torch.zeros(8, dtype=torch.complex128, device="cuda")
    th = torch.zeros(8, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    for q, p in [(97, 4), (40, 33), (4, 5), (0, 1)]:
        with pytest.raises(pbs.PbsError) as e:
            pbs.small_rr_noalloc(dummy.data_ptr(), dummy.data_ptr(), q, p, dummy.data_ptr(), th.data_ptr(),
                                 info.data_ptr())
        assert e.value.status == pbs.PBS_EINVAL
