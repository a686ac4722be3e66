"""FP64 oracle: the Kohn-Sham Hamiltonian on a periodic real-space grid.

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.

Follows Eq. (1) and Sec. 2.2 of the paper: H = -1/2 nabla^2 + V, applied on a
Fourier grid where FFT pairs switch between the position representation (the
potential is diagonal) and the momentum representation (the kinetic energy is
diagonal).  The ionic pseudopotential is split into a local part (folded into
the given local potential together with V_H[rho0] + V_xc) and Kleinman-Bylander
nonlocal projectors on atom-centred spheres (Sec. 3, where atomic spheres of
neighbouring atoms overlap).  The optional kinetic-energy cutoff of Sec. 2.2 and
Table 2 is read as T(k) = min(|k|^2/2, E_cut).

Conventions: arrays are indexed [z, y, x] (x fastest); the inner product is
<a|b> = dV sum_r conj(a) b with dV = h^3.
"""
import numpy as np


class Grid:
    """Cubic periodic grid of n^3 points with spacing h (bohr)."""

    def __init__(self, n, h, ecut=None):
        self.n = int(n)
        self.h = float(h)
        self.L = self.n * self.h
        self.dV = self.h ** 3
        self.ng = self.n ** 3
        m = np.fft.fftfreq(self.n) * self.n          # integer frequencies in FFT order
        k1 = 2.0 * np.pi * m / self.L
        kz, ky, kx = np.meshgrid(k1, k1, k1, indexing='ij')
        self.k2 = kx ** 2 + ky ** 2 + kz ** 2
        t = 0.5 * self.k2
        if ecut is not None and ecut > 0:
            t = np.minimum(t, ecut)
        self.T = t                                   # kinetic energy in k space
        vc = np.zeros_like(self.k2)
        nz = self.k2 > 0
        vc[nz] = 4.0 * np.pi / self.k2[nz]
        self.vcoul = vc                              # periodic Coulomb kernel, k=0 dropped

    def shape(self):
        return (self.n, self.n, self.n)

    def dot(self, a, b):
        """<a|b> = dV sum conj(a) b over the last three axes."""
        return self.dV * np.sum(np.conj(a) * b, axis=(-3, -2, -1))


class KB:
    """Kleinman-Bylander nonlocal part: V_NL = sum_{a,p} |beta_ap> E_ap <beta_ap|.

    atoms: list of (support, beta, e) where support is an int array of flat grid
    indices, beta is [n_proj, len(support)] (real) and e is [n_proj].
    """

    def __init__(self, atoms):
        self.atoms = [(np.asarray(s, dtype=np.int64), np.asarray(b, dtype=np.float64),
                       np.asarray(e, dtype=np.float64)) for (s, b, e) in atoms]

    def apply(self, psi, grid):
        """V_NL psi for psi of shape [..., n, n, n]."""
        lead = psi.shape[:-3]
        flat = psi.reshape(lead + (grid.ng,))
        out = np.zeros_like(flat)
        for sup, beta, e in self.atoms:
            vals = flat[..., sup]                                   # [..., nsup]
            c = grid.dV * np.einsum('ps,...s->...p', beta, vals)    # <beta_p|psi>
            out[..., sup] += np.einsum('ps,...p->...s', beta, c * e)
        return out.reshape(psi.shape)


def kinetic(psi, grid):
    """T psi = IFFT( T(k) FFT(psi) ) over the last three axes."""
    return np.fft.ifftn(grid.T * np.fft.fftn(psi, axes=(-3, -2, -1)), axes=(-3, -2, -1))


def apply_h(psi, grid, vloc, kb=None, vext=None):
    """H psi with H = T + V_loc (+ V_NL) (+ an extra local potential vext).

    psi: complex [..., n, n, n]; vloc: real [n, n, n]; vext broadcastable to psi.
    """
    out = kinetic(psi, grid) + vloc * psi
    if kb is not None:
        out = out + kb.apply(psi, grid)
    if vext is not None:
        out = out + vext * psi
    return out


def poisson(rho, grid):
    """Hartree potential of a periodic charge density: v = IFFT(4 pi/|k|^2 FFT(rho)), k=0 dropped.

    Linear and real-symmetric, so it may be applied to complex inputs (real and
    imaginary parts are solved independently).
    """
    return np.fft.ifftn(grid.vcoul * np.fft.fftn(rho, axes=(-3, -2, -1)), axes=(-3, -2, -1))


def dense_h(grid, vloc, kb=None):
    """Dense matrix of H in the grid basis, assembled column by column from unit vectors.

    Only for tiny grids (used to pin the oracle against LAPACK eigh).
    """
    ng = grid.ng
    H = np.zeros((ng, ng), dtype=np.complex128)
    e = np.zeros(grid.shape(), dtype=np.complex128)
    ef = e.reshape(-1)
    for j in range(ng):
        ef[:] = 0
        ef[j] = 1.0
        H[:, j] = apply_h(e, grid, vloc, kb).reshape(-1)
    return H
