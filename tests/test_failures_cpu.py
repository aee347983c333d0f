"""Failure detection that is decided on the host, before any device work, so it
is checked here without a GPU: a non-finite squared slowness returns
HELM_ERR_NUMERIC, a device-memory cap smaller than the grid arrays returns
HELM_ERR_OOM (helm_config.max_device_bytes), and a bad partition returns
HELM_ERR_ARG.  None leaves anything behind: the context is not created.  (On a GPU, tests/test_gpu_parity.py checks the cap
against the factors' allocation, and the bounded waits' HELM_ERR_TIMEOUT.)"""
import dataclasses

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def H():
    import paper_2002_05327_gb300 as H
    from paper_2002_05327_gb300.build import build
    build()
    return H


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_medium_is_a_numeric_error(H, bad):
    wl = W.small_2d()
    m = wl.m.copy()
    m[m.shape[0] // 2, 3] = bad
    with pytest.raises(H.HelmError) as e:
        H.helm_setup(2, wl.n, wl.h, wl.omega, m, wl.pml, wl.sigma0, wl.nb, wl.overlap,
                     sub_pml=wl.sub_pml)
    assert e.value.code == H.HELM_ERR_NUMERIC
    assert "non-finite" in str(e.value)


def test_device_memory_cap_below_the_grid_arrays_is_oom(H):
    wl = W.small_2d()
    with pytest.raises(H.HelmError) as e:
        H.helm_setup_workload(wl, max_device_bytes=4096)
    assert e.value.code == H.HELM_ERR_OOM
    assert "cap" in str(e.value)


def test_negative_cap_is_an_argument_error(H):
    wl = W.small_2d()
    with pytest.raises(H.HelmError) as e:
        H.helm_setup_workload(wl, max_device_bytes=-1)
    assert e.value.code == H.HELM_ERR_ARG


# ---- the partition, checked on the host before any device work
def _setup_error(H, wl):
    with pytest.raises(H.HelmError) as e:
        H.helm_setup_workload(wl)
    return e.value


@pytest.mark.parametrize("what", ["not increasing", "not spanning", "narrow box", "narrow 3D inner box"])
def test_bad_partition_is_an_argument_error(H, what):
    """Cuts that do not increase or do not span 0..n, a box narrower than
    overlap + 2, and in 3D an inner box narrower than twice the overlap (the
    cutoffs of both neighbours along an axis would then reach one node):
    HELM_ERR_ARG, decided before any device work."""
    if what == "narrow 3D inner box":
        # overlap 3: an inner box of 5 cells passes overlap + 2 but not 2 overlap
        wl = W.small_3d(n=(24, 18, 16), nb=(3, 2, 2), pml=5, overlap=3, sub_pml=4, nrhs=1)
        wl = dataclasses.replace(wl, cuts=(np.array([0, 10, 15, 24]), wl.cuts[1], wl.cuts[2]))
        message = "twice the overlap"
    else:
        wl = W.small_2d(nx=60, ny=52, nbx=4, nby=3, nrhs=1)  # overlap 4
        x = {"not increasing": [0, 20, 20, 40, 60], "not spanning": [0, 15, 30, 45, 59],
             "narrow box": [0, 20, 25, 40, 60]}[what]
        wl = dataclasses.replace(wl, cuts=(np.array(x), wl.cuts[1]))
        message = {"not increasing": "increase", "not spanning": "span",
                   "narrow box": "overlap + 2"}[what]
    e = _setup_error(H, wl)
    assert e.code == H.HELM_ERR_ARG, str(e)
    assert message in str(e)


def test_every_gpu_test_partition_passes_the_host_checks(H):
    """The partitions the GPU tests, smoke() and the bench set up get past
    every host-side check of helm_setup: without a device the first error is
    the CUDA runtime's, not HELM_ERR_ARG."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present: the GPU tests set these partitions up")
    import test_gpu_parity as GP
    wls = [mk() for mk in GP.CASES.values()]
    wls += [W.config(k, with_sources=False) for k in (1, 2, 3, 4, 5)]
    wls += [W.iter_const_2d(600, 2, 55), W.iter_const_2d(1200, 4, 105), W.iter_r3_3d(2),
            W.small_2d(nx=64, ny=56, nbx=3, nby=3, pml=10, overlap=2, sub_pml=2, nrhs=1),
            W.small_2d(nx=40, ny=36, nbx=2, nby=2, pml=8, overlap=4, sub_pml=8, nrhs=1),
            W.small_2d(nx=40, ny=36, nbx=3, nby=2, pml=8, overlap=4, sub_pml=8, nrhs=1),
            W.small_3d(n=(12, 10, 9), nb=(2, 2, 1), pml=4, overlap=2, sub_pml=3, nrhs=1)]
    for wl in wls:
        e = _setup_error(H, wl)
        assert e.code == H.HELM_ERR_CUDA, (wl.name, str(e))
