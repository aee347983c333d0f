"""Write oracle_gmres_iters.txt: the iterations the oracle's own DDM-preconditioned
FGMRES (oracle.krylov.gmres with one Algorithm 3.1 application as the
preconditioner, restart 30) needs on the first source of the 1064^2 layered
workload and of the 2088x1576 nonuniform workload, to the relative residual
the benchmark solves to (1e-8), with the time of its local factorisations and
of one iteration.  Calls only oracle/ and the input generators; the benchmark's
CPU baseline uses these counts instead of the GPU solve's.

    python tests/golden/make_oracle_gmres_iters.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ddm as OD  # noqa: E402
from oracle import helmholtz as OH  # noqa: E402
from oracle import krylov as OK  # noqa: E402

RTOL = 1e-8


def main():
    lines = ["# workload rtol iterations true_resid factor_s gmres_s  (oracle FGMRES, source 0, restart 30)"]
    for k in (2, 4):
        wl = W.config(k, src=[0])
        A, J = OH.global_operator(wl)
        t0 = time.time()
        part = OD.Partition(wl)
        t_fac = time.time() - t0
        b = wl.f * J.reshape((1,) + wl.f.shape[1:])

        def apply_A(x):
            return (A @ x.reshape(x.shape[0], -1).T).T.reshape(x.shape)

        t1 = time.time()
        x, info = OK.gmres(apply_A, b, lambda v: OD.diagonal_sweep(part, v), rtol=RTOL, restart=30, maxit=60)
        t_gm = time.time() - t1
        lines.append(f"{wl.name} {RTOL:g} {int(info['iters'][0])} {float(info['resid'][0]):.3e} "
                     f"{t_fac:.1f} {t_gm:.1f}")
        print(lines[-1], flush=True)
    open(os.path.join(HERE, "oracle_gmres_iters.txt"), "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
