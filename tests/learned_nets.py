"""Hand-built networks and checks shared by the learned-form tests."""
import numpy as np


def double_dissipation_net(K=1e3, M=1e3):
    """A network whose density and energy corrections are -M sign(right - left)
    of the stencil's two central cells: clipped, that doubles the Rusanov
    dissipation of rho and e1 at every face, which drives the pressure negative
    next to the blast's jump within a few steps."""
    W1 = np.zeros((64, 40))
    W2 = np.zeros((64, 64))
    W3 = np.zeros((8, 64))
    for n, (o, v) in enumerate(((0, 0), (7, 7))):
        a, b = 4 * n, 4 * n + 1
        W1[a, 16 + v], W1[a, 8 + v] = K, -K
        W1[b, 16 + v], W1[b, 8 + v] = -K, K
        W2[a, a], W2[a, b], W2[b, a], W2[b, b] = 1, -1, -1, 1
        W3[o, a], W3[o, b] = -M, M
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(8)])


def physical_per_block(gamma, U):
    """Per block: every cell finite with rho > 0 and p > 0, p from Eq. 5 in numpy."""
    rho = U[0]
    m2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
    b2 = U[4] ** 2 + U[5] ** 2 + U[6] ** 2
    with np.errstate(all="ignore"):
        p = (gamma - 1) * (U[7] - 0.5 * m2 / rho - 0.5 * b2)
        ok = np.isfinite(U).all(axis=0) & (rho > 0) & (p > 0)
    return ok.reshape(U.shape[1], -1).all(axis=1)
