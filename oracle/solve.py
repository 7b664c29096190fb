"""Linear solvers for the assembled SPD systems (oracle, test infrastructure only).

The method needs the discrete state and adjoint solutions S_l[xi](u) and
q_l (Sec. 2.2); the paper solves them with a multigrid-preconditioned CG
(Sec. 5).  The oracle only needs the discrete solution itself, so it offers

* ``direct``: sparse LU (SuperLU) - exact up to rounding, used for parity at
  small sizes;
* ``pcg``: textbook preconditioned CG stopped at ||b - A x||_2 <= rtol ||b||_2
  (true residual recomputed at the end), preconditioned either by the
  diagonal or by a Galerkin V-cycle built from sparse matrices
  (A_c = P^T A P, trilinear P, damped-Jacobi smoothing).  The preconditioner
  changes only the iteration count, not the converged answer.

If ||b|| = 0 the solution is 0 with 0 iterations.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def direct(A, b):
    if not np.any(b):
        return np.zeros_like(b), 0
    return spla.splu(A.tocsc()).solve(b), 1


def _prolongation_1d(Nc):
    """1D linear interpolation from Nc cells to 2 Nc cells, interior nodes only."""
    nf, nc = 2 * Nc - 1, Nc - 1
    P = sp.lil_matrix((nf, nc))
    for j in range(nc):  # coarse interior node j+1 sits at fine node 2(j+1)
        f = 2 * (j + 1) - 1  # fine interior index
        P[f, j] = 1.0
        P[f - 1, j] = 0.5
        P[f + 1, j] = 0.5
    return P.tocsr()


class GalerkinMG:
    """V(2,2)-cycle with damped Jacobi on Galerkin coarse operators, interior dofs,
    on a hierarchy N, N/2, ..., 2 (N a power of two times the coarsest)."""

    def __init__(self, A, N, omega=0.6):
        self.omega = omega
        self.A = [A]
        self.P = []
        n = N
        while n > 2 and n % 2 == 0:
            P1 = _prolongation_1d(n // 2)
            P = sp.kron(sp.kron(P1, P1), P1).tocsr()  # z slowest, x fastest
            self.P.append(P)
            self.A.append((P.T @ self.A[-1] @ P).tocsr())
            n //= 2
        self.D = [Ai.diagonal() for Ai in self.A]
        self.coarse = spla.splu(self.A[-1].tocsc())

    def _vcycle(self, lev, r):
        if lev == len(self.A) - 1:
            return self.coarse.solve(r)
        A, D, w = self.A[lev], self.D[lev], self.omega
        x = w * r / D
        x = x + w * (r - A @ x) / D
        rc = self.P[lev].T @ (r - A @ x)
        x = x + self.P[lev] @ self._vcycle(lev + 1, rc)
        x = x + w * (r - A @ x) / D
        x = x + w * (r - A @ x) / D
        return x

    def __call__(self, r):
        return self._vcycle(0, r)


def pcg(A, b, rtol, max_iter=100000, precond=None, max_restarts=50):
    """Preconditioned CG; returns (x, iterations).  Raises if not converged, or when
    the true residual stalls above rtol ||b|| (more than max_restarts restarts from the
    true residual: rtol is below the residual FP64 can attain for this system)."""
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    if precond is None:
        d = A.diagonal()
        precond = lambda r: r / d
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    restarts = 0
    for it in range(1, max_iter + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= rtol * bn:
            if np.linalg.norm(b - A @ x) <= rtol * bn:
                return x, it
            # the recursive residual drifted below the true one: restart CG from the
            # true residual (a fresh search direction; the old one belongs to the
            # drifted recursion)
            restarts += 1
            if restarts > max_restarts:
                raise RuntimeError("oracle PCG: true residual stalls at %.3g ||b|| above rtol %.3g" %
                                   (np.linalg.norm(b - A @ x) / bn, rtol))
            r = b - A @ x
            z = precond(r)
            p = z.copy()
            rz = r @ z
            continue
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise RuntimeError("oracle PCG did not converge")


def solve(A, b, N, rtol=1e-13, method="auto"):
    """Solve A x = b on the interior dofs of an N^3-cell level."""
    if method == "auto":
        method = "direct" if N <= 16 else "mg"
    if method == "direct":
        return direct(A, b)
    if method == "jacobi":
        return pcg(A, b, rtol)
    if method == "mg":
        return pcg(A, b, rtol, precond=GalerkinMG(A, N))
    raise ValueError(method)
