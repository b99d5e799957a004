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
"""
import numpy as np
import scipy.sparse as sp


def pml_sigma(t, eta, C, pml_form="paper"):
    """sigma(t) of Eq. sigma, vectorised over t in [0, 1]."""
    t = np.asarray(t, dtype=np.float64)
    s = np.zeros_like(t)
    if eta <= 0.0:
        return s
    pref = C / eta if pml_form == "paper" else C
    left = t < eta
    right = t > 1.0 - eta
    s[left] = pref * ((t[left] - eta) / eta) ** 2
    s[right] = pref * ((t[right] - 1.0 + eta) / eta) ** 2
    return s


def stretch(t, eta, C, omega, pml_form="paper"):
    """s(t) = (1 + i sigma(t)/omega)^(-1)  (Section 2.1)."""
    return 1.0 / (1.0 + 1j * pml_sigma(t, eta, C, pml_form) / omega)


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

    def __init__(self, c, omega, pml_width, C=2 * np.pi, pml_form="paper"):
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
        s_n = stretch(xn, eta, C, omega, pml_form)
        s_h = stretch(xh, eta, C, omega, pml_form)
        self.s_node = s_n
        self.s_half = s_h
        # east[j, k] = s1(xh_k) / s2(xn_j) / h^2
        self.east = s_h[None, :] / s_n[:, None] / (h * h)
        # north[k, i] = s2(xh_k) / s1(xn_i) / h^2
        self.north = s_h[:, None] / s_n[None, :] / (h * h)
        self.s1s2 = s_n[None, :] * s_n[:, None]
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

    def d_diag_dc(self):
        """Derivative of the diagonal entry A_ii with respect to c_i:
        -2 omega^2 / ((s1 s2)_i c_i^3); the off-diagonal entries do not depend on c."""
        return -2.0 * self.omega ** 2 / (self.s1s2 * self.c ** 3)
