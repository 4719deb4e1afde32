#!/usr/bin/env python
"""Writes tests/golden/rsw-N512-S256-M64_k01.npz: the FP64 oracle's coarse
predictor U^0 and first parareal iterate U^1 (Eq. 3.1, Algorithm 4) on every
one of the 256 slices of the single large workload (N = 512, eps = 1e-3,
nu = 1e-4, T = 10, fine dt = 1e-4, M = 64, seeded initial spectrum).

Only the oracle and the seeded input generator are used.  The arrays hold the
kept wavenumbers k = 0 .. K (K = 170); every bin above K is zero by the 2/3
rule and is not stored.  The run takes about a minute of one host core.

Usage: python tests/golden/make_large_golden.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import rsw_inputs as ri  # noqa: E402
from oracle import rsw as o  # noqa: E402

WORKLOAD = ri.LARGE_N512
PATH = os.path.join(HERE, "rsw-N512-S256-M64_k01.npz")


def main() -> None:
    w = WORKLOAD
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    t0 = time.perf_counter()
    res = o.parareal(w.initial_state(), p, w.slices, 1)
    K = o.kept_modes(w.n_grid)
    for U in res.iterates:
        assert not np.any(U[..., K + 1:])
    np.savez_compressed(PATH, workload=np.array(w.name), kept=np.array(K),
                        U0=res.iterates[0][..., :K + 1], U1=res.iterates[1][..., :K + 1],
                        change1=np.array(res.changes[0]))
    print(f"wrote {PATH} in {time.perf_counter() - t0:.1f} s")


if __name__ == "__main__":
    main()
