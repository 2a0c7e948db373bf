"""Volume averages of the TGV diagnostics of Sec. 6.2 for an oracle state --
test infrastructure only: E_k = (1/(rho0 |Omega|)) sum (1/2)|m|^2/rho |cell|
and eps^S = (1/(rho0 |Omega|)) sum mu |curl U|^2 |cell|, rho0 the mean
density, the velocity gradient from the averages and cell-averaged gradients
(d_k U_i = (d_k m_i - U_i d_k rho)/rho)."""
import numpy as np


def tgv_diagnostics(state, dim, vol, mu):
    s = np.asarray(state, dtype=np.float64)
    vol = np.asarray(vol, dtype=np.float64).reshape(s.shape[2:])
    rho = s[0, 0]
    U = s[0, 1:1 + dim] / rho
    ke = 0.5 * rho * (U * U).sum(axis=0)
    # G[i][k] = d_k U_i
    G = [[(s[1 + k, 1 + i] - U[i] * s[1 + k, 0]) / rho for k in range(dim)] for i in range(dim)]
    if dim == 3:
        w2 = (G[2][1] - G[1][2]) ** 2 + (G[0][2] - G[2][0]) ** 2 + (G[1][0] - G[0][1]) ** 2
    else:
        w2 = (G[1][0] - G[0][1]) ** 2
    V = vol.sum()
    rho0 = (rho * vol).sum() / V
    return float((ke * vol).sum() / (rho0 * V)), float((mu * w2 * vol).sum() / (rho0 * V))
