"""Failure detection that is decided on the host, before any device work, so it
is checked here without a GPU: a non-finite squared slowness returns
HELM_ERR_NUMERIC, and a device-memory cap smaller than the grid arrays returns
HELM_ERR_OOM (helm_config.max_device_bytes).  Both leave nothing behind: the
context is not created.  (On a GPU, tests/test_gpu_parity.py checks the cap
against the factors' allocation, and the bounded waits' HELM_ERR_TIMEOUT.)"""
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
