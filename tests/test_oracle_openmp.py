"""The OpenMP build of the oracle (the multi-core CPU baseline) computes the same
bits as the plain build: its finite-volume loops over blocks write each cell
once from its own inputs, so the thread count cannot change a result."""
import numpy as np

import mrfv_inputs as mi
import oracle


def test_openmp_oracle_is_bit_identical_to_the_plain_oracle():
    out = []
    for omp in (False, True):
        o = oracle.Oracle(2, 3, (2, 3, 1), openmp=omp)
        o.init(mi.IC_QUADRANTS, mi.quadrant_params(4))
        o.adapt(oracle.CRIT_MR, 1e-3)
        for _ in range(4):
            dt = o.dt(0.5)
            o.step(dt)
            o.adapt(oracle.CRIT_MR, 1e-3)
        out.append([o.get_level(l) for l in range(3)])
    for a, b in zip(*out):
        assert np.array_equal(np.isnan(a), np.isnan(b))
        m = ~np.isnan(a)
        assert np.array_equal(a[m], b[m])
    assert oracle.threads(True) >= 1
