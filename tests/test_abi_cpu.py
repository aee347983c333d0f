"""CPU-side checks of the C ABI: the library loads, exports every entry point
declared in include/helm.h, and the ctypes structures match the C layout.
No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helm.h")


@pytest.fixture(scope="module")
def H():
    import paper_2002_05327_gb300 as H
    from paper_2002_05327_gb300.build import build
    build()
    return H


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("helm_setup", "helm_factor", "helm_solve", "helm_apply_ddm", "helm_adjoint",
                 "helm_destroy", "helm_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(H):
    L = H.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert L.helm_strerror(-4).decode() == "GMRES did not converge"


def test_struct_layout_matches_c(H):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "helm.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("helm_pml %zu\nhelm_partition %zu\nhelm_config %zu\nhelm_stats %zu\n",
         sizeof(helm_pml), sizeof(helm_partition), sizeof(helm_config), sizeof(helm_stats));
  P(helm_pml, sigma0) P(helm_pml, form) P(helm_partition, cuts) P(helm_partition, overlap)
  P(helm_partition, sub_pml) P(helm_config, stream) P(helm_stats, resid)
  P(helm_stats, t_solve_ms) P(helm_stats, levels) P(helm_stats, solves)
  P(helm_config, profile) P(helm_config, tc_kernel) P(helm_config, wait_limit) P(helm_config, sweep_order) P(helm_config, max_device_bytes) P(helm_config, algorithm) P(helm_profile, ms) P(helm_profile, bytes) P(helm_profile, flops)
  printf("helm_profile %zu\n", sizeof(helm_profile));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split("\n")
    c = dict(line.rsplit(" ", 1) for line in out if line.strip())
    c = {k: int(v) for k, v in c.items()}
    assert c["helm_pml"] == ctypes.sizeof(H.helm_pml)
    assert c["helm_partition"] == ctypes.sizeof(H.helm_partition)
    assert c["helm_config"] == ctypes.sizeof(H.helm_config)
    assert c["helm_stats"] == ctypes.sizeof(H.helm_stats)
    assert c["helm_profile"] == ctypes.sizeof(H.helm_profile)
    for key, v in c.items():
        if "." in key:
            s, f = key.split(".")
            assert getattr(getattr(H, s), f).offset == v, key


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2002_05327_gb300 as H
    monkeypatch.setattr(H, "_lib", None)
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        H.lib()


def test_product_path_does_not_import_the_oracle():
    """The package and the CUDA sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2002_05327_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
