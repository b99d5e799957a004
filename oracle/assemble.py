"""O1: discretisation of the PML-stretched Helmholtz operator (Section 2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Grid: p_{i,j} = (i h, j h), 1 <= i, j <= n, h = 1/(n+1); unknowns ordered row by
row (x1 fastest).  0-based arrays: node (i, j) -> index [j-1, i-1].

PML (Eq. sigma): sigma(t) = (C/eta) ((t - eta)/eta)^2 on [0, eta], 0 in the
middle, mirrored on [1 - eta, 1]; s(t) = 1 / (1 + i sigma(t)/omega).  eta is
`pml_width` grid cells, eta = pml_width * h.  With pml_form="literal" the 1/eta
prefactor is dropped (sigma = C ((t-eta)/eta)^2), the other printed reading.

5-point stencil (Eq. helmd), after dividing by s1 s2 so that A is symmetric:
  coefficient to the x1-neighbours:  (s1/s2)_{i +- 1/2, j} / h^2
  coefficient to the x2-neighbours:  (s2/s1)_{i, j +- 1/2} / h^2
  diagonal:  omega^2 / ((s1 s2)_{i,j} c_{i,j}^2) - (sum of the four coefficients)
The four-term sum includes the coefficients toward boundary neighbours (where
u = 0), as Eq. helmd is written for every interior point.

Other boundary conditions (Section 2.5; Section 3.2): `pml_sides` is a bit mask of the
sides that carry a PML (1: x1 = 0, 2: x1 = 1, 4: x2 = 0, 8: x2 = 1; default all four).
A side without PML has sigma = 0 near it and is a plain Dirichlet boundary; non-zero
Dirichlet data b on a side enters as a forcing term on the adjacent layer of unknowns
(`boundary_rhs`), the only change the method needs.
"""
import numpy as np
import scipy.sparse as sp


def pml_sigma(t, eta, C, pml_form="paper", lo=True, hi=True):
    """sigma(t) of Eq. sigma, vectorised over t in [0, 1]; lo / hi: the layer at t = 0 /
    t = 1 is present."""
    t = np.asarray(t, dtype=np.float64)
    s = np.zeros_like(t)
    if eta <= 0.0:
        return s
    pref = C / eta if pml_form == "paper" else C
    left = (t < eta) & bool(lo)
    right = (t > 1.0 - eta) & bool(hi)
    s[left] = pref * ((t[left] - eta) / eta) ** 2
    s[right] = pref * ((t[right] - 1.0 + eta) / eta) ** 2
    return s


def stretch(t, eta, C, omega, pml_form="paper", lo=True, hi=True):
    """s(t) = (1 + i sigma(t)/omega)^(-1)  (Section 2.1)."""
    return 1.0 / (1.0 + 1j * pml_sigma(t, eta, C, pml_form, lo, hi) / omega)


class Discretization:
    """Coefficients of A for velocity c (n x n, x1 fastest) at angular frequency omega.

    Attributes (complex128):
      east[j, k]  for k = 0..n : coefficient on the x1-edge between node k-1 and
                  node k of row j, i.e. (s1/s2)_{k+1/2, j+1}/h^2 in 1-based
                  half-point notation; k = 0 and k = n touch the boundary.
      north[k, i] for k = 0..n : coefficient on the x2-edge between rows k-1 and k.
      diag[j, i]  : the diagonal of Eq. helmd.
      s1s2[j, i]  : (s1 s2) at the node.
    """

    def __init__(self, c, omega, pml_width, C=2 * np.pi, pml_form="paper", pml_sides=15):
        c = np.asarray(c, dtype=np.float64)
        n = c.shape[0]
        assert c.shape == (n, n)
        self.n, self.N = n, n * n
        self.omega = float(omega)
        self.c = c
        h = 1.0 / (n + 1)
        self.h = h
        eta = pml_width * h
        self.eta = eta
        xn = (np.arange(n) + 1.0) * h          # nodes
        xh = (np.arange(n + 1) + 0.5) * h      # half points between nodes k-1 and k
        self.pml_sides = int(pml_sides)
        b = [bool(self.pml_sides >> k & 1) for k in range(4)]
        s1n = stretch(xn, eta, C, omega, pml_form, b[0], b[1])   # s1 along x1
        s1h = stretch(xh, eta, C, omega, pml_form, b[0], b[1])
        s2n = stretch(xn, eta, C, omega, pml_form, b[2], b[3])   # s2 along x2
        s2h = stretch(xh, eta, C, omega, pml_form, b[2], b[3])
        self.s_node = s1n
        self.s_half = s1h
        # east[j, k] = s1(xh_k) / s2(xn_j) / h^2
        self.east = s1h[None, :] / s2n[:, None] / (h * h)
        # north[k, i] = s2(xh_k) / s1(xn_i) / h^2
        self.north = s2h[:, None] / s1n[None, :] / (h * h)
        self.s1s2 = s1n[None, :] * s2n[:, None]
        offsum = self.east[:, :-1] + self.east[:, 1:] + self.north[:-1, :] + self.north[1:, :]
        self.diag = omega * omega / (self.s1s2 * c * c) - offsum

    def matrix(self):
        """Sparse A (N x N, CSR).  Each edge coefficient is used for both of its
        endpoints, so A^t = A holds exactly."""
        n, N = self.n, self.N
        idx = np.arange(N).reshape(n, n)
        rows, cols, vals = [idx.ravel()], [idx.ravel()], [self.diag.ravel()]
        # x1-edges inside each row: (i, j) <-> (i+1, j), coefficient east[j, i+1]
        a, b = idx[:, :-1].ravel(), idx[:, 1:].ravel()
        v = self.east[:, 1:-1].ravel()
        rows += [a, b]; cols += [b, a]; vals += [v, v]
        # x2-edges: (i, j) <-> (i, j+1), coefficient north[j+1, i]
        a, b = idx[:-1, :].ravel(), idx[1:, :].ravel()
        v = self.north[1:-1, :].ravel()
        rows += [a, b]; cols += [b, a]; vals += [v, v]
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N))
        return A.tocsr()

    # --- block tridiagonal view (Section 2.1) ---------------------------------
    def A_mm(self, m):
        """Dense tridiagonal diagonal block A_{m,m} for 0-based row m."""
        n = self.n
        T = np.diag(self.diag[m]).astype(np.complex128)
        e = self.east[m, 1:-1]
        T[np.arange(n - 1), np.arange(1, n)] = e
        T[np.arange(1, n), np.arange(n - 1)] = e
        return T

    def A_off(self, m):
        """Diagonal of A_{m, m-1} = A_{m-1, m} (0-based m >= 1), as a vector."""
        return self.north[m].copy()

    def boundary_rhs(self, side, b):
        """The forcing term of Dirichlet data u = b on one side (0: x1 = 0, 1: x1 = 1,
        2: x2 = 0, 3: x2 = 1; b has n values along the side): -(edge coefficient) * b on
        the adjacent nodes, as an (n, n) array to add to f (Section 2.5)."""
        n = self.n
        b = np.asarray(b, dtype=np.complex128)
        g = np.zeros((n, n), dtype=np.complex128)
        if side == 0:
            g[:, 0] = -self.east[:, 0] * b
        elif side == 1:
            g[:, n - 1] = -self.east[:, n] * b
        elif side == 2:
            g[0, :] = -self.north[0, :] * b
        elif side == 3:
            g[n - 1, :] = -self.north[n, :] * b
        else:
            raise ValueError(side)
        return g

    def d_diag_dc(self):
        """Derivative of the diagonal entry A_ii with respect to c_i:
        -2 omega^2 / ((s1 s2)_i c_i^3); the off-diagonal entries do not depend on c."""
        return -2.0 * self.omega ** 2 / (self.s1s2 * self.c ** 3)
