"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is element-wise, right-hand side by right-hand side
(tests/parity.py): the relative L2 error of each right-hand side and its
relative max error max|u - ref| / max|ref| must both be within the tolerance,
so that a wrong value at a few nodes (a transfer strip, a corner, a seam)
cannot hide under a norm over the whole output.

Tolerances, from the arithmetic and set at 2-4x the worst case measured on
GB300 over every case below (raw DDM against the oracle's Algorithm 3.1/4.1):
  * FP64 path (HELM_PREC_F64): 1e-12 (measured <= 1.2e-14).  Both sides solve
    the same complex128 systems; only the elimination order differs.
  * complex64 SIMT path (HELM_PREC_MIXED): 1e-5 (measured <= 5.5e-6).
    complex64 factors carry a unit roundoff of 6e-8, amplified by the block
    recurrence and the local condition numbers of the PML blocks.
  * Tensor-core paths (TF32, FP16 with power-of-two scales): 3e-3 (measured
    <= 7.5e-4).  Both keep 10 mantissa bits (unit roundoff 4.9e-4) in every
    block product.
  * After FP64 GMRES (the product's answer): 1e-6 per right-hand side against
    the global direct solve, the bound the method promises after refinement.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from parity import assert_close
from oracle import adjoint as OA
from oracle import ddm as OD
from oracle import helmholtz as OH

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 3e-3, 3: 3e-3, 4: 3e-3, 5: 3e-3}
PRECS = [0, 1, 2, 3, 4, 5]


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2002_05327_gb300 as H
    from paper_2002_05327_gb300.build import build
    build()
    return H


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ctx(H, wl, prec, **kw):
    """prec 0/1/2 = FP64 / complex64 / TF32 tensor cores (tcgen05 where the
    blocks allow it, in the twisted two-ended form where every subdomain has
    at least 4 lines); 3 = TF32 forced onto the mma.sync kernel; 4 = TF32 on
    the one-ended tcgen05 kernel; 5 = FP16 operands with power-of-two scales
    in the twisted tcgen05 kernel (two tiles up to 256 block rows, three up to
    384; TF32 elsewhere)."""
    if prec == 3:
        prec, kw = 2, dict(kw, tc_kernel=1)
    elif prec == 4:
        prec, kw = 2, dict(kw, tc_kernel=2)
    elif prec == 5:
        prec = 3
    c = H.helm_setup_workload(wl, precision=prec, **kw)
    H.helm_factor(c)
    return c


CASES = {
    "2d-layered-3x2": lambda: W.small_2d(),
    "2d-layered-4x3-5rhs": lambda: W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=5),
    "2d-1x1": lambda: W.small_2d(nx=30, ny=26, nbx=1, nby=1, nrhs=1),
    "2d-strip-3x1": lambda: W.small_2d(nx=45, ny=20, nbx=3, nby=1, nrhs=2),
    # blocks of more than 128 rows: the tensor-core solve runs as a 2-CTA cluster
    "2d-wide-2x2": lambda: W.small_2d(nx=260, ny=48, nbx=2, nby=2, pml=8, overlap=4, sub_pml=8,
                                      nrhs=10),
    # blocks of 300 rows: three M = 128 tiles in the FP16 twisted kernel
    "2d-300row-2x2": lambda: W.small_2d(nx=560, ny=48, nbx=2, nby=2, pml=8, overlap=4, sub_pml=8,
                                        nrhs=3),
    "3d-const-2x2x2": lambda: W.small_3d(),
    "3d-layered-3x2x2": lambda: W.small_3d(n=(27, 18, 16), nb=(3, 2, 2), nrhs=1, medium="layered"),
}


def _nonuniform():
    wl = W.small_2d(nx=64, ny=50, nbx=3, nby=3, nrhs=3)
    cuts = (np.array([0, 17, 40, 64]), np.array([0, 21, 33, 50]))
    return dataclasses.replace(wl, cuts=cuts)


CASES["2d-nonuniform-3x3"] = _nonuniform


def _face():
    """Sources half a cell inside and one cell past the internal face between
    boxes 1 and 2 along x: the result is dominated by what crosses that face
    (the transfer strips and the corner transfers of the neighbouring boxes)."""
    wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=2)
    h, c = wl.h, wl.cuts
    y = 0.5 * (c[1][1] + c[1][2]) * h
    f = W.gaussian_sources(wl.n, wl.pml, h, [((c[0][2] - 1.5) * h, y), ((c[0][2] + 0.5) * h, y)], h)
    return dataclasses.replace(wl, f=f)


CASES["2d-face-4x3"] = _face


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_apply_ddm_matches_algorithm(H, case, prec):
    """helm_apply_ddm equals the oracle's Algorithm 3.1 / 4.1 (same windows,
    cutoffs, routing) element by element."""
    wl = CASES[case]()
    ctx = _ctx(H, wl, prec)
    u = H.helm_apply_ddm(ctx, wl.f)
    ref = OD.ddm_solution(wl)
    assert_close(u, ref, TOL[prec], TOL[prec], (case, prec))
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1, 5])
@pytest.mark.parametrize("case", ["2d-layered-4x3-5rhs", "2d-nonuniform-3x3", "3d-layered-3x2x2"])
def test_additive_ddm_matches_algorithm(H, case, prec):
    """helm_config.algorithm = 1: the additive DDM of Section 2.2 (Algorithm
    2.1 in 2D, 2.2 in 3D), every subdomain solving at every step, equals the
    oracle's additive() element by element; it differs from the sweeps'
    result, so the option is in effect."""
    wl = CASES[case]()
    ctx = _ctx(H, wl, prec, algorithm=1)
    u = H.helm_apply_ddm(ctx, wl.f)
    ctx.close()
    _, J = OH.global_operator(wl)
    part = OD.Partition(wl)
    ref = OD.additive(part, wl.f * J.reshape((1,) + wl.f.shape[1:]))
    assert_close(u, ref, TOL[prec], TOL[prec], ("additive", case, prec))
    if prec == 0:
        assert rel(u, OD.ddm_solution(wl)) > 1e-6
    with pytest.raises(H.HelmError):
        H.helm_setup_workload(wl, algorithm=2)


@pytest.mark.parametrize("prec", [0, 5])
def test_alternative_3d_sweep_order_matches_algorithm(H, prec):
    """helm_config.sweep_order = 1 (the second 3D order of Section 4.1) equals
    the oracle's Algorithm 4.1 in that order; the plain FP64 path also differs
    from the first order's result, so the option is in effect."""
    wl = CASES["3d-layered-3x2x2"]()
    ctx = _ctx(H, wl, prec, sweep_order=1)
    u = H.helm_apply_ddm(ctx, wl.f)
    ctx.close()
    ref = OD.ddm_solution(wl, order=1)
    assert_close(u, ref, TOL[prec], TOL[prec], ("order 1", prec))
    if prec == 0:
        assert rel(u, OD.ddm_solution(wl, order=0)) > 1e-6
    with pytest.raises(H.HelmError):
        H.helm_setup_workload(wl, sweep_order=2)


@pytest.mark.parametrize("prec", PRECS)
def test_subdomain_solve_matches_local_direct_solve(H, prec):
    wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=3)
    ctx = _ctx(H, wl, prec)
    part = OD.Partition(wl)
    rng = np.random.default_rng(1)
    for s in (0, 5, 11):
        I = (s % 4, s // 4)
        sub = part.subs[I]
        lo, hi = H.helm_window_info(ctx, s)
        assert lo == sub.lo and hi == sub.hi
        R = rng.standard_normal((3,) + sub.shape) + 1j * rng.standard_normal((3,) + sub.shape)
        u = H.helm_subdomain_solve(ctx, s, R)
        ref = part.local_solve(sub, R)
        tol = {0: 1e-12, 1: 1e-5}.get(prec, 3e-3)  # measured <= 4.4e-15, 2.5e-6, 8.3e-4
        assert_close(u, ref, tol, tol, (s, prec))
    ctx.close()


def test_config1_ddm_fp64(H):
    """Config 1 (160^2, 2x2, one Gaussian): the plain complex128 GPU DDM equals
    the oracle's Algorithm 3.1, and both are within PML truncation of the
    global solution."""
    wl = W.config(1)
    ctx = _ctx(H, wl, 0)
    u = H.helm_apply_ddm(ctx, wl.f)
    ref = OD.ddm_solution(wl)
    assert_close(u, ref, 1e-12, 1e-12, "config 1")
    assert rel(u, OH.solve_global(wl)) < 5e-4
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_gmres_reaches_global_solution(H, prec):
    wl = W.small_2d(nx=64, ny=56, nbx=3, nby=3, pml=10, overlap=4, sub_pml=10, nrhs=3)
    ctx = _ctx(H, wl, prec)
    x, st = H.helm_solve(ctx, wl.f, rtol=1e-10, maxit=60)
    ref = OH.solve_global(wl)
    assert_close(x, ref, 1e-6, 1e-6, ("gmres", prec))
    assert st["resid"] <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", [0, 5])
def test_gmres_long_cycle(H, prec):
    """A GMRES cycle longer than eight iterations: the Gram-Schmidt dots then
    take the basis in a group of eight and a remainder, and the combinations
    run unfused.  A deliberately weak preconditioner (2-cell subdomain PML,
    overlap 2) for which the oracle's FP64 GMRES needs more than eight
    iterations at a relative residual of 1e-10: the FP64 GPU path must need
    that count (one more or fewer for rounding), the FP16 one more than eight
    as well, and both must reach the direct solution."""
    from oracle import krylov as OK
    wl = W.small_2d(nx=64, ny=56, nbx=3, nby=3, pml=10, overlap=2, sub_pml=2, nrhs=2)
    A, J = OH.global_operator(wl, "literal")
    b = wl.f * J.reshape((1,) + wl.f.shape[1:])
    Ax = lambda x: (A @ x.reshape(x.shape[0], -1).T).T.reshape(x.shape)
    _, info = OK.gmres(Ax, b, OD.DDMPreconditioner(wl), rtol=1e-10, restart=30, maxit=30)
    it_ref = int(np.max(info["iters"]))
    assert it_ref >= 9, it_ref
    ctx = _ctx(H, wl, prec)
    x, st = H.helm_solve(ctx, wl.f, rtol=1e-10, maxit=30)
    ctx.close()
    if prec == 0:
        assert abs(st["iters"] - it_ref) <= 1, (st["iters"], it_ref)
    else:
        assert st["iters"] >= 9, (st["iters"], it_ref)
    assert st["resid"] <= 1e-10
    assert_close(x, OH.solve_global(wl), 1e-6, 1e-6, ("long gmres cycle", prec))


def test_stationary_iteration_matches_algorithm(H):
    """helm_iterate, the DDM as an iterative solver (Section 5.2.2): after three
    steps the FP64 iterate equals the oracle's u_3 and its residual; with FP16
    subdomain solves the iteration converges to the global solution."""
    wl = W.small_2d(nx=64, ny=56, nbx=3, nby=3, pml=10, overlap=4, sub_pml=10, nrhs=3)
    A, J = OH.global_operator(wl)
    b = wl.f * J.reshape((1,) + wl.f.shape[1:])
    us, res = OD.stationary(OD.Partition(wl), A, b, 3)
    ctx = _ctx(H, wl, 0)
    u, st = H.helm_iterate(ctx, wl.f, rtol=1e-30, maxit=3, allow_noconv=True)
    ctx.close()
    assert st["applications"] == 3
    assert_close(u, us[-1], 1e-12, 1e-12, "u_3")
    assert abs(st["resid"] - res[-1]) <= 1e-3 * res[-1], (st["resid"], res[-1])
    ctx = _ctx(H, wl, 5)
    u, st = H.helm_iterate(ctx, wl.f, rtol=1e-10, maxit=60)
    ctx.close()
    assert_close(u, OH.solve_global(wl), 1e-6, 1e-6, "stationary fp16")
    assert st["resid"] <= 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_residual_matches_operator(H, dim):
    if dim == 3:
        wl = W.small_3d(n=(12, 10, 9), nb=(2, 2, 1), pml=4, overlap=2, sub_pml=3, nrhs=2,
                        medium="layered")
    else:
        wl = W.small_2d(nx=40, ny=36, nbx=2, nby=2, pml=8, overlap=4, sub_pml=8, nrhs=3)
    ctx = _ctx(H, wl, 0)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(wl.f.shape) + 1j * rng.standard_normal(wl.f.shape)
    r = H.helm_residual(ctx, wl.f, u)
    A, J = OH.global_operator(wl)
    nr = wl.f.shape[0]
    ref = (wl.f.reshape(nr, -1) * J[None] - (A @ u.reshape(nr, -1).T).T).reshape(u.shape)
    assert_close(r, ref, 1e-13, 1e-13, "residual")
    ctx.close()


def test_adjoint_and_gradient(H):
    wl = W.small_2d(nx=40, ny=34, nbx=2, nby=2, pml=8, overlap=4, sub_pml=8, nrhs=2)
    rec = np.array([(wl.pml + k, wl.pml + 2) for k in range(2, 38, 4)])
    ctx = _ctx(H, wl, 1)
    u, _ = H.helm_solve(ctx, wl.f, rtol=1e-11, maxit=80)
    m_true = wl.m * 1.02
    d = OA.receiver_values(OH.solve_global(dataclasses.replace(wl, m=m_true)), rec)
    g_src = OA.adjoint_source(u, rec, d)
    lam, _ = H.helm_adjoint(ctx, g_src, rtol=1e-11, maxit=80)
    # the adjoint solve against the direct A^{-H}
    A, _ = OH.global_operator(wl)
    import scipy.sparse.linalg as spla
    lu = spla.splu(A.tocsc())

    def solve(b):
        return lu.solve(np.ascontiguousarray(b.reshape(b.shape[0], -1).T)).T.reshape(b.shape)

    lam_ref = OA.adjoint_solve(solve, g_src)
    assert_close(lam, lam_ref, 1e-6, 1e-6, "adjoint")
    g = H.helm_gradient(ctx, u, lam)
    g_ref = OA.gradient(wl, u, lam)
    assert_close(g[None], g_ref[None], 1e-12, 1e-12, "gradient")
    ctx.close()


def test_release_and_refactor_give_the_same_gradient(H):
    """HelmSolve with keep_bytes=0 releases the context's factors and buffers
    after the forward solve (helm_release) and recomputes them in backward:
    the device memory between the passes drops to the setup's, and the
    gradient is bitwise the one computed with the factors kept."""
    import torch
    wl = W.small_2d(nx=40, ny=34, nbx=2, nby=2, pml=8, overlap=4, sub_pml=8, nrhs=2)
    rec = np.array([(wl.pml + k, wl.pml + 2) for k in range(2, 38, 4)])
    spec = dict(ndim=wl.ndim, n=wl.n, h=wl.h, omega=wl.omega, pml_width=wl.pml, sigma0=wl.sigma0,
                nb=wl.nb, overlap=wl.overlap, power=wl.power, cuts=wl.cuts, sub_pml=wl.sub_pml,
                precision=H.HELM_PREC_F16)
    F = torch.from_numpy(wl.f).cuda()
    ry, rx = torch.from_numpy(rec[:, 1]).cuda(), torch.from_numpy(rec[:, 0]).cuda()
    grads = []
    for keep in (None, 0):
        m = torch.tensor(wl.m, dtype=torch.float64, device="cuda", requires_grad=True)
        U = H.HelmSolve.apply(m, F, spec, 1e-10, 80, keep)
        loss = (U[:, ry, rx].abs() ** 2).sum()
        loss.backward()
        grads.append(m.grad.cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
    ctx = H.helm_setup_workload(wl, precision=H.HELM_PREC_F16)
    setup_bytes = H.helm_device_bytes(ctx)
    H.helm_factor(ctx)
    u1 = H.helm_apply_ddm(ctx, wl.f)
    assert H.helm_device_bytes(ctx) > setup_bytes
    H.helm_release(ctx)
    assert H.helm_device_bytes(ctx) == setup_bytes
    with pytest.raises(H.HelmError) as e:
        H.helm_apply_ddm(ctx, wl.f)
    assert e.value.code == H.HELM_ERR_NOT_FACTORED
    H.helm_factor(ctx)
    assert np.array_equal(H.helm_apply_ddm(ctx, wl.f), u1)
    ctx.close()


def test_chunked_solve_with_host_buffers(H):
    """helm_solve with host buffers and a device-memory cap that forces the
    batch into chunks: the chunks' uploads and downloads run on a copy stream
    beside the other chunks' solves.  Every right-hand side must still match
    the global direct solve, and the device-pointer call the same way."""
    import torch
    wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=8)
    ref = OH.solve_global(wl)
    base = _ctx(H, wl, 1)  # complex64: the factor holds no transient array beyond its own
    factored = H.helm_device_bytes(base)
    H.helm_solve(base, wl.f, rtol=1e-10, maxit=80)
    need = H.helm_device_bytes(base) - factored  # staging, sources, window buffers, Krylov vectors
    base.close()
    chunked = None
    for frac in (0.7, 0.55, 0.4, 0.3):
        ctx = _ctx(H, wl, 1, max_device_bytes=factored + int(need * frac))
        try:
            u, st = H.helm_solve(ctx, wl.f, rtol=1e-10, maxit=80)
        except H.HelmError as e:
            assert e.code == H.HELM_ERR_OOM
            ctx.close()
            continue
        if st["applications"] > st["iters"] + 1:  # more than one GMRES run
            chunked = (ctx, u, st)
            break
        ctx.close()
    assert chunked is not None, "no cap gave a chunked solve"
    ctx, u, st = chunked
    assert_close(u, ref, 1e-6, 1e-6, ("chunked, host buffers", st))
    ud, _ = H.helm_solve(ctx, torch.from_numpy(wl.f).cuda(), rtol=1e-10, maxit=80)
    assert_close(ud.cpu().numpy(), ref, 1e-6, 1e-6, "chunked, device buffers")
    ctx.close()


def test_errors_are_reported(H):
    wl = W.small_2d()
    with pytest.raises(H.HelmError) as e:
        H.helm_setup(2, wl.n, wl.h, wl.omega, wl.m, wl.pml, wl.sigma0, (40, 1), 4)
    assert e.value.code == H.HELM_ERR_ARG
    ctx = H.helm_setup_workload(wl, precision=1)
    with pytest.raises(H.HelmError) as e:
        H.helm_apply_ddm(ctx, wl.f)
    assert e.value.code == H.HELM_ERR_NOT_FACTORED
    H.helm_factor(ctx)
    with pytest.raises(H.HelmError) as e:
        H.helm_solve(ctx, wl.f, rtol=1e-14, maxit=1)
    assert e.value.code == H.HELM_ERR_NO_CONVERGENCE
    ctx.close()


def test_device_memory_cap_refuses_the_factors(H):
    """helm_config.max_device_bytes set just above what setup holds: helm_factor
    is refused with HELM_ERR_OOM before it allocates, the context holds no more
    than the cap, and it can still be destroyed."""
    wl = W.small_2d()
    probe = H.helm_setup_workload(wl, precision=1)
    setup_bytes = H.helm_device_bytes(probe)
    probe.close()
    cap = setup_bytes + 1024
    ctx = H.helm_setup_workload(wl, precision=1, max_device_bytes=cap)
    with pytest.raises(H.HelmError) as e:
        H.helm_factor(ctx)
    assert e.value.code == H.HELM_ERR_OOM
    assert H.helm_device_bytes(ctx) <= cap
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_expired_wait_is_reported_and_context_stays_usable(H, prec):
    """wait_limit=-1 makes every ordinary bounded wait inside the subdomain-solve
    kernels give up at its first check, so each kernel takes its abort path:
    raise the device error word, stop issuing work, drain the copies and MMAs
    it started, free TMEM, exit.  Every entry point that runs a solve must
    report HELM_ERR_TIMEOUT (the error word is cleared after each report), and
    a fresh context on the same device must still give the right answer.
    The wide case runs the tcgen05 kernel as 2-CTA clusters."""
    wl = CASES["2d-wide-2x2"]()
    bad = _ctx(H, wl, prec, wait_limit=-1)
    for _ in range(2):
        with pytest.raises(H.HelmError) as e:
            H.helm_apply_ddm(bad, wl.f)
        assert e.value.code == H.HELM_ERR_TIMEOUT
    with pytest.raises(H.HelmError) as e:
        H.helm_solve(bad, wl.f, rtol=1e-8, maxit=5)
    assert e.value.code == H.HELM_ERR_TIMEOUT
    lo, hi = H.helm_window_info(bad, 0)
    shape = tuple(reversed([b - a for a, b in zip(lo, hi)]))
    with pytest.raises(H.HelmError) as e:
        H.helm_subdomain_solve(bad, 0, np.ones((1,) + shape, dtype=np.complex128))
    assert e.value.code == H.HELM_ERR_TIMEOUT
    bad.close()
    good = _ctx(H, wl, prec)
    u = H.helm_apply_ddm(good, wl.f)
    assert_close(u, OD.ddm_solution(wl), TOL[prec], TOL[prec], ("after timeout", prec))
    good.close()


def test_deterministic_and_device_pointers(H):
    import torch
    wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=5)
    ctx = _ctx(H, wl, 1)
    u1 = H.helm_apply_ddm(ctx, wl.f)
    u2 = H.helm_apply_ddm(ctx, wl.f)
    assert np.array_equal(u1, u2)
    ud = H.helm_apply_ddm(ctx, torch.from_numpy(wl.f).cuda())
    assert np.array_equal(ud.cpu().numpy(), u1)
    ctx.close()


@pytest.mark.parametrize("case,prec", [("2d-wide-2x2", 2), ("2d-wide-2x2", 4), ("2d-wide-2x2", 5),
                                       ("2d-300row-2x2", 5)])
def test_cluster_tensor_core_path_is_deterministic(H, case, prec):
    """The tcgen05 solves run as 2-CTA clusters: the twisted form (prec 2, 5)
    hands the middle line's vectors between its two halves, the one-ended
    form (prec 4, blocks of more than 128 rows) exchanges the B operand every
    line step.  Repeated applications must be bitwise identical (a handshake
    race would show as run-to-run changes)."""
    wl = CASES[case]()
    ctx = _ctx(H, wl, prec)
    u1 = H.helm_apply_ddm(ctx, wl.f)
    for _ in range(3):
        assert np.array_equal(H.helm_apply_ddm(ctx, wl.f), u1)
    ctx.close()
