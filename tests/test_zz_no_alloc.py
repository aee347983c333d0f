"""helm_subdomain_solve_noalloc: the subdomain solve for callers that cannot
allocate device memory when they call it.

It must give the same answer as the allocating entry point
helm_subdomain_solve, on the same kernel, call after call -- the shared
static scratch keeps the previous call's contents, so two calls in a row with
different subdomains and right-hand sides must both be right -- and it must
refuse sizes beyond its fixed scratch with HELM_ERR_ARG.  For every precision
it is also checked against the oracle's direct solve of the same local PML
problem, with the tolerances of the other subdomain-solve tests.  The file
sorts last so that a run stopping at the first failure has run every other
test first; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import ddm as OD

pytestmark = pytest.mark.gpu

# against the allocating entry point (same kernel, same inputs: rounding only)
TOL_SAME = {0: 1e-12, 1: 1e-6, 2: 1e-6, 3: 1e-6}
# against the oracle's local direct solve (as in test_gpu_parity)
TOL_ORACLE = {0: 1e-11, 1: 1e-4, 2: 1e-2, 3: 1e-2}


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2002_05327_gb300 as H
    from paper_2002_05327_gb300.build import build
    build()
    return H


def _call(H, ctx, s, R, U):
    """Through the C ABI: device pointers in and out, no allocation inside."""
    return H.lib().helm_subdomain_solve_noalloc(ctx.ptr, int(s), int(R.shape[0]),
                                                 ctypes.c_void_p(R.data_ptr()),
                                                 ctypes.c_void_p(U.data_ptr()))


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return max(float(np.linalg.norm(a[r] - b[r]) / np.linalg.norm(b[r])) for r in range(b.shape[0]))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_allocating_solve_twice_in_a_row(H, prec):
    import torch
    wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=3)
    part = OD.Partition(wl)
    ctx = H.helm_setup_workload(wl, precision=prec)
    H.helm_factor(ctx)
    rng = np.random.default_rng(7 + prec)
    for s in (5, 0):  # two calls in a row, different windows and sources
        lo, hi = H.helm_window_info(ctx, s)
        shape = (3,) + tuple(reversed([b - a for a, b in zip(lo, hi)]))
        R = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        ref = H.helm_subdomain_solve(ctx, s, R)
        Rd = torch.from_numpy(R).cuda()
        Ud = torch.empty_like(Rd)
        assert _call(H, ctx, s, Rd, Ud) == H.HELM_OK, H.lib().helm_last_error()
        got = Ud.cpu().numpy()
        assert _rel(got, ref) < TOL_SAME[prec], (s, _rel(got, ref))
        direct = part.local_solve(part.subs[(s % 4, s // 4)], R)
        assert _rel(got, direct) < TOL_ORACLE[prec], (s, _rel(got, direct))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(H):
    """A request one right-hand side beyond the 64 MiB scratch is refused before
    any device work; R and U are real buffers of that size, so even a broken
    check would stay inside memory the test owns."""
    import torch
    wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=1)
    ctx = H.helm_setup_workload(wl, precision=0)
    H.helm_factor(ctx)
    lo, hi = H.helm_window_info(ctx, 0)
    win = int(np.prod([b - a for a, b in zip(lo, hi)]))
    too_many = (64 << 20) // (win * 16) + 1
    R = torch.zeros((too_many, win), dtype=torch.complex128, device="cuda")
    U = torch.zeros_like(R)
    rc = H.lib().helm_subdomain_solve_noalloc(ctx.ptr, 0, too_many, ctypes.c_void_p(R.data_ptr()),
                                              ctypes.c_void_p(U.data_ptr()))
    assert rc == H.HELM_ERR_ARG
    assert b"maximum" in H.lib().helm_last_error()
    with pytest.raises(ValueError):
        H.helm_subdomain_solve_noalloc(ctx, 0, R[:1].reshape(1, 1, win))
    ctx.close()
