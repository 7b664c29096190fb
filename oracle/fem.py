"""Assembled Q1 finite elements on the unit cube (oracle, test infrastructure only).

The state problem is a(xi; y, v) = <B u, v> for all v in V (eq:sys) with
a(xi; y, v) = int exp(a~(x, xi)) grad y . grad v dx and <B u, v> = int u v dx
(Sec. 5, definition of A(xi) and B), homogeneous Dirichlet data
(V = H^1_0).  The FE space on level l is the Q1 (trilinear) space on the
uniform mesh of N = n0 * 2^l cells per side (the paper names its discrete
spaces V_l in Sec. 2.2; element type and coefficient per cell, evaluated at the
cell centre, are this workload's reading).

Matrices are ASSEMBLED from element integrals computed by 2x2x2 Gauss
quadrature of the reference shape functions (not from a closed-form stencil),
so that the closed-form stencil and the discrete eigenpairs are independent
pins of this code (tests/test_oracle_fem.py).

Index conventions: node (i, j, k) at (i h, j h, k h), flat index
i + (N+1) * (j + (N+1) * k); cell (i, j, k) flat index i + N * (j + N * k).
Interior nodes are those with 1 <= i, j, k <= N-1.

Control (Sec. 5: U = L2(D)): z is piecewise constant on the cells of a
control grid with N_c = N * 2^r cells per side.  (B z)_n = int z phi_n
= sum_c z_c h_c^3 phi_n(x_c) (midpoint rule, exact for the multilinear
phi_n on each control cell); the adjoint with respect to
<z, w>_U = h_c^3 sum_c z_c w_c is (B* q)_c = q(x_c), the FE function q
evaluated at the control-cell centres.
"""
import numpy as np
import scipy.sparse as sp

_GP = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])  # 2-pt Gauss on [0, 1]
_GW = np.array([0.5, 0.5])


def _ref_shape(xi, eta, zeta):
    """Trilinear shape functions and reference gradients at one point of [0,1]^3.

    Local node a = dx + 2 dy + 4 dz."""
    N = np.empty(8)
    G = np.empty((8, 3))
    for a in range(8):
        dx, dy, dz = a & 1, (a >> 1) & 1, (a >> 2) & 1
        fx = xi if dx else 1 - xi
        fy = eta if dy else 1 - eta
        fz = zeta if dz else 1 - zeta
        gx = 1.0 if dx else -1.0
        gy = 1.0 if dy else -1.0
        gz = 1.0 if dz else -1.0
        N[a] = fx * fy * fz
        G[a] = (gx * fy * fz, fx * gy * fz, fx * fy * gz)
    return N, G


def element_matrices(h):
    """Element stiffness (coefficient 1) and mass matrices of a cube of side h,
    integrated by the 2x2x2 Gauss rule."""
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    for i, xi in enumerate(_GP):
        for j, eta in enumerate(_GP):
            for k, zeta in enumerate(_GP):
                w = _GW[i] * _GW[j] * _GW[k] * h ** 3
                N, G = _ref_shape(xi, eta, zeta)
                G = G / h  # physical gradients
                Ke += w * G @ G.T
                Me += w * np.outer(N, N)
    return Ke, Me


class Level:
    """One FE level: N cells per side."""

    def __init__(self, N):
        self.N = N
        self.h = 1.0 / N
        self.nn = (N + 1) ** 3
        self.nc = N ** 3
        n1 = N + 1
        ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
        inner = (ii > 0) & (ii < N) & (jj > 0) & (jj < N) & (kk > 0) & (kk < N)
        flat = ii + n1 * (jj + n1 * kk)
        self.interior = np.sort(flat[inner])
        ci, cj, ck = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        cflat = (ci + N * (cj + N * ck)).ravel()
        order = np.argsort(cflat)
        base = (ci + n1 * (cj + n1 * ck)).ravel()[order]
        # connectivity [cell, local node]
        self.conn = np.stack([base + (a & 1) + n1 * ((a >> 1) & 1) + n1 * n1 * ((a >> 2) & 1)
                              for a in range(8)], axis=1)
        self.Ke, self.Me = element_matrices(self.h)
        self._mass = None

    def _assemble(self, cell_weights, Eloc):
        rows = np.repeat(self.conn, 8, axis=1).ravel()
        cols = np.tile(self.conn, (1, 8)).ravel()
        vals = (cell_weights[:, None] * Eloc.ravel()[None, :]).ravel()
        return sp.coo_matrix((vals, (rows, cols)), shape=(self.nn, self.nn)).tocsr()

    def stiffness(self, a_cells):
        """Full (all-node) stiffness matrix for cellwise coefficient a (length N^3)."""
        return self._assemble(np.asarray(a_cells, dtype=np.float64), self.Ke)

    def mass(self):
        if self._mass is None:
            self._mass = self._assemble(np.ones(self.nc), self.Me)
        return self._mass

    def restrict(self, Afull):
        """Dirichlet restriction to interior rows/columns."""
        I = self.interior
        return Afull[I][:, I].tocsr()

    def node_coords(self):
        n1 = self.N + 1
        idx = np.arange(self.nn)
        i, j, k = idx % n1, (idx // n1) % n1, idx // (n1 * n1)
        return i * self.h, j * self.h, k * self.h

    def nodal_target(self, freq=1):
        """Nodal interpolant of g = sin(f pi x) sin(f pi y) sin(f pi z) (f = 1 for the workload,
        f = 2 for the paper's Sec. 5 target); exactly 0 on the boundary."""
        x, y, z = self.node_coords()
        w = freq * np.pi
        g = np.sin(w * x) * np.sin(w * y) * np.sin(w * z)
        g[~np.isin(np.arange(self.nn), self.interior)] = 0.0
        return g

    def interpolation(self, Nc):
        """Matrix I [Nc^3, nodes] with I[c, n] = (1/|c|) int_c phi_n dx, the average of the
        hat function phi_n over control cell c.  Then B z = h_c^3 I^T z is exactly
        int z phi_n dx for a cellwise-constant control z (<Bu, v> = int u v, Sec. 5)
        and B* q = I q is the cell average of q.

        Control grid at least as fine as the level (Nc = r N): phi_n is trilinear on
        each control cell, so its average is its value at the cell centre.
        Control grid coarser (N = r Nc): per axis the average of a 1D hat over a
        control interval of r fine cells is 1/r at the r - 1 inner nodes and 1/(2r)
        at the two end nodes (each end node's hat lies half inside)."""
        rows, cols, vals = [], [], []
        n1 = self.N + 1
        c = np.arange(Nc ** 3)
        ci, cj, ck = c % Nc, (c // Nc) % Nc, c // (Nc * Nc)
        if Nc % self.N == 0:
            r = Nc // self.N
            # position of the centre inside its level cell
            ex, ey, ez = ci // r, cj // r, ck // r
            tx = ((ci % r) + 0.5) / r
            ty = ((cj % r) + 0.5) / r
            tz = ((ck % r) + 0.5) / r
            for a in range(8):
                dx, dy, dz = a & 1, (a >> 1) & 1, (a >> 2) & 1
                w = (tx if dx else 1 - tx) * (ty if dy else 1 - ty) * (tz if dz else 1 - tz)
                node = (ex + dx) + n1 * ((ey + dy) + n1 * (ez + dz))
                rows.append(c)
                cols.append(node)
                vals.append(w)
        else:
            assert self.N % Nc == 0, "one grid must refine the other"
            r = self.N // Nc
            w1 = np.full(r + 1, 1.0 / r)
            w1[0] = w1[-1] = 0.5 / r
            for a in range(r + 1):
                for b in range(r + 1):
                    for d in range(r + 1):
                        node = (r * ci + a) + n1 * ((r * cj + b) + n1 * (r * ck + d))
                        rows.append(c)
                        cols.append(node)
                        vals.append(np.full(c.shape, w1[a] * w1[b] * w1[d]))
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(Nc ** 3, self.nn)).tocsr()
