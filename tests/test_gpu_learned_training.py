"""End to end: training pairs made by the solver, GPU training, and the gain
of the trained network at half resolution.

Six seeded blast variants (centre offset, inner pressure, field direction)
give coarse/fine pairs; the network trains on the GPU; on the held-out blast
(centre 0, p_in 10, B along (1,1,0)) the coarse run with the network must be
closer to the fine run (restricted) than the coarse run without it, and the
untrained network (zero output layer) must be exactly the plain scheme.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_network_reduces_the_half_resolution_error():
    from paper_2501_06717_gb300 import bats as B
    from paper_2501_06717_gb300 import learn

    X, Y = learn.make_pairs(variants=[101, 102, 103, 104, 105, 106], snapshots=(4, 12), keep=0.3)
    assert X.shape[0] > 100000 and np.isfinite(X).all() and np.isfinite(Y).all()
    P, hist = learn.train(X, Y, epochs=6, lr=1e-3)
    assert hist[-1] < 0.7 * hist[0]
    e_plain, e_learn = learn.evaluate(P, nsteps=16)
    print("half-resolution error vs restricted full-resolution run: plain %.4f, learned %.4f" % (e_plain, e_learn))
    assert e_learn < 0.85 * e_plain
    m = B.Mlp(seed=0)   # untrained: output layer zero
    P0 = m.get_params()
    m.close()
    e_plain0, e_init = learn.evaluate(P0, nsteps=16)
    assert e_init == e_plain0 == e_plain
