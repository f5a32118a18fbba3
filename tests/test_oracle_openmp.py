"""The oracle built with OpenMP gives the plain build's results bit for bit.

The per-iteration loops of the oracle that write one element per index carry
OpenMP pragmas (norms and other reductions stay serial), so each element's
arithmetic is the same whichever thread runs it.  This is what lets the CPU
baseline time the same oracle on every host core.  Checked on 2D and 3D boxes
with a ±30 % cohesion field through plastic increments (Jaumann term on), on
4 threads against the plain build: every history field and every iteration
count equal.
"""
import numpy as np
import pytest

import oracle as O

FIELDS = {2: ["vx", "vy", "txx", "tyy", "txy", "p", "epl"],
          3: ["vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl"]}


def _run(nd, n, incs, lib_path):
    rng = np.random.default_rng(11)
    nc = int(np.prod(n))
    coh = 1.5e-3 * (1.0 + 0.3 * (2.0 * rng.random(nc) - 1.0))
    coh[nc // 2] *= 0.5
    o = O.Oracle(nd, n, (1.0, 1.0, 1.0), lib_path=lib_path)
    o.set_material(2.0, 1.0, float("inf"), 30.0, 0.0, coh)
    o.set_solver(tol=1e-9, n_chk=20, max_iter=400000)
    rates = [1.0, -1.0] if nd == 2 else [1.0, 0.0, -1.0]
    iters, plastic = [], []
    for _ in range(incs):
        o.apply_increment(rates, 3e-4)
        info = o.solve_increment()
        iters.append(info["iters"])
        plastic.append(info["n_plastic"])
    return iters, plastic, {f: o.get(f).copy() for f in FIELDS[nd]}


@pytest.mark.parametrize("nd,n,incs", [(2, (24, 17), 6), (3, (9, 7, 6), 5)])
def test_openmp_build_equals_plain_build(nd, n, incs):
    path = O.build_omp()
    if path is None:
        pytest.skip("the C compiler has no OpenMP")
    assert O.threads(4, path) == 4
    assert O.threads() == 1
    it0, pl0, f0 = _run(nd, n, incs, None)
    it1, pl1, f1 = _run(nd, n, incs, path)
    assert max(pl0) > 0, "the case must reach plastic increments"
    assert it0 == it1 and pl0 == pl1
    for k in f0:
        assert np.array_equal(f0[k], f1[k]), k
