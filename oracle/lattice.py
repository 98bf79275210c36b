"""Square lattice with open boundaries, the PEPS parameter layout and the bonds of Eq. 12.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

Sites: N = nrow * ncol (Eq. 4 uses N = L1 x L2), site i = r * ncol + c.
Local index (Eq. 4, |S_i> = |s_i>|s'_i>): S = 2*s + s', with s (system) and s'
(ancilla) in {0 = up (S^z = +1/2), 1 = down (S^z = -1/2)}; physical dimension d^2 = 4.

Site tensor T_i^{S}[l, r, u, d]: legs to the left/right/up/down neighbours.  With open
boundaries a leg that leaves the lattice has dimension 1 ("trimmed" OBC), every other
leg has dimension D.  The parameter vector theta is the concatenation over sites of
T_i with shape (4, dl, dr, du, dd) in row-major order; N_p = 4 * sum_i dl*dr*du*dd.

O layout (Eq. 8 is non-zero only in the slice S_i of each T_i): one sample's O row
holds, per site, the dl*dr*du*dd entries of that slice; entry k of site i is the
derivative with respect to theta[off_i + S_i * sz_i + k].
"""
import numpy as np


class Lattice:
    def __init__(self, nrow, ncol, D, J1=1.0, J2=0.0):
        self.nrow, self.ncol, self.D = int(nrow), int(ncol), int(D)
        self.J1, self.J2 = float(J1), float(J2)
        self.N = self.nrow * self.ncol
        self.dims = [self.site_dims(i) for i in range(self.N)]
        self.sz = [int(np.prod(d)) for d in self.dims]
        self.theta_off = np.concatenate([[0], np.cumsum([4 * s for s in self.sz])]).astype(np.int64)
        self.o_off = np.concatenate([[0], np.cumsum(self.sz)]).astype(np.int64)
        self.Np = int(self.theta_off[-1])
        self.No = int(self.o_off[-1])

    def site(self, r, c):
        return r * self.ncol + c

    def site_dims(self, i):
        r, c = divmod(i, self.ncol)
        D = self.D
        return (1 if c == 0 else D, 1 if c == self.ncol - 1 else D,
                1 if r == 0 else D, 1 if r == self.nrow - 1 else D)

    def bonds(self):
        """Bonds of Eq. 12 as (i, j, J, kind): nearest neighbours (kind 'h' horizontal,
        'v' vertical) with J1, next-nearest neighbours across each plaquette ('d' for
        (r,c)-(r+1,c+1), 'a' for (r,c+1)-(r+1,c)) with J2 (omitted when J2 == 0)."""
        out = []
        for r in range(self.nrow):
            for c in range(self.ncol - 1):
                out.append((self.site(r, c), self.site(r, c + 1), self.J1, 'h'))
        for r in range(self.nrow - 1):
            for c in range(self.ncol):
                out.append((self.site(r, c), self.site(r + 1, c), self.J1, 'v'))
        if self.J2 != 0.0:
            for r in range(self.nrow - 1):
                for c in range(self.ncol - 1):
                    out.append((self.site(r, c), self.site(r + 1, c + 1), self.J2, 'd'))
                    out.append((self.site(r, c + 1), self.site(r + 1, c), self.J2, 'a'))
        return out

    def tensors(self, theta):
        """Split theta into the site tensors T_i of shape (4, dl, dr, du, dd) (views)."""
        theta = np.asarray(theta, dtype=np.float64)
        return [theta[self.theta_off[i]:self.theta_off[i + 1]].reshape((4,) + self.dims[i])
                for i in range(self.N)]


def spin_sys(S):
    """System spin s of local index S = 2 s + s'."""
    return np.asarray(S) // 2


def spin_anc(S):
    """Ancilla spin s' of local index S = 2 s + s'."""
    return np.asarray(S) % 2


def sz_of(s):
    """S^z eigenvalue of spin bit s: +1/2 for 0 (up), -1/2 for 1 (down)."""
    return 0.5 - np.asarray(s, dtype=np.float64)
