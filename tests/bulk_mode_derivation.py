"""Symbolic linear stability of the well-balanced update about a uniform
rest state (Sec. III equilibrium and forcing, BGK, pull streaming), used by
tests/test_stability.py.  Independent of the oracle and of the CUDA path.

Linearised about rho = rho_b, u = 0, a perturbation df_i(x) = e_i exp(i k.x)
gives delta rho = 1, delta j = c_j, delta F = -i g(k) S with the gradient
symbol g(k) = (sin k_x (2 + cos k_y), sin k_y (2 + cos k_x)) / 3 and
S = rho_b (psi_0''(rho_b) - kappa ell(k)), ell the Laplacian symbol;
delta f_0^eq = delta rho, delta f_i^eq = 3 w_i c_i.(delta j + delta F / 2)
(i != 0), delta F_i = 3 w_i c_i.delta F, and the post-collision value is
streamed with exp(-i k.c_i).  At k_x = pi: g_x = 0 and ell = -4, so S is a
constant; the eigenvalue 1 of the matrix at k = (pi, 0) is followed to
second order in k_y = q."""
import sympy as sp
from sympy.polys.matrices import DomainMatrix

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
WT = [sp.Rational(4, 9)] + [sp.Rational(1, 9)] * 4 + [sp.Rational(1, 36)] * 4


def amplification(q, om, S):
    """9 x 9 amplification matrix at k = (pi, q)."""
    kf = 1 - om / 2
    gy = sp.sin(q) / 3                        # (2 + cos pi) sin q / 3
    M = sp.zeros(9, 9)
    for j in range(9):
        dFy = -sp.I * gy * S
        for i in range(9):
            if i == 0:
                feq = 1
            else:
                feq = 3 * WT[i] * (CX[i] * CX[j] + CY[i] * (CY[j] + dFy / 2))
            Fi = 3 * WT[i] * CY[i] * dFy
            post = (1 - om) * (1 if i == j else 0) + om * feq + kf * Fi
            M[i, j] = (-1) ** abs(CX[i]) * sp.exp(-sp.I * q * CY[i]) * post
    return M


def second_order(lam0):
    """lambda(q) = lam0 + lam1 q + lam2 q^2 + ...; returns (lam1, lam2) and
    the q^2 coefficient of |lambda|^2."""
    q = sp.Symbol("q", real=True)
    om, S = sp.symbols("omega S", positive=True)
    M = amplification(q, om, S)
    M0 = M.subs(q, 0)
    M1 = M.diff(q).subs(q, 0)
    M2 = (M.diff(q, 2) / 2).subs(q, 0)
    A = M0 - lam0 * sp.eye(9)

    def kernel(B):                           # one-dimensional null space, as a column
        rows = DomainMatrix.from_Matrix(B).to_field().nullspace().to_Matrix()
        assert rows.shape[0] == 1            # the eigenvalue is simple
        return rows.T

    v0 = kernel(A)
    u0 = kernel(A.T)
    n0 = (u0.T * v0)[0]
    lam1 = sp.cancel(sp.expand((u0.T * M1 * v0)[0] / n0))
    sol, params = A.gauss_jordan_solve((lam1 * sp.eye(9) - M1) * v0)
    w1 = sol.subs({p: 0 for p in params})
    lam2 = sp.cancel(sp.expand((u0.T * (M2 * v0 + M1 * w1 - lam1 * w1))[0] / n0))
    a2 = sp.cancel(sp.expand(lam1 * sp.conjugate(lam1) + 2 * sp.re(lam0 * lam2)))
    return om, S, lam1, lam2, a2


if __name__ == "__main__":
    for lam0 in (1, -1):
        om, S, lam1, lam2, a2 = second_order(lam0)
        print(lam0, lam1, sp.factor(lam2), sp.factor(a2))
