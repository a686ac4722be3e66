"""Deterministic references used to pin the oracle's TDH and Sigma(t) (test helper).

* Casida RPA (time-dependent Hartree, closed shell, real orbitals): with pair densities
  P_ia = phi_i phi_a, Delta_ia = e_a - e_i and the Coulomb matrix V_{ia,jb} = (ia|jb),
  Omega_s^2 are the eigenvalues of C = D^2 + 4 D^{1/2} V D^{1/2} (D = diag Delta) and the
  retarded density response is chi(r, r', t) = -2 theta(t) sum_s sin(Omega_s t) rho_s(r) rho_s(r'),
  rho_s = sqrt(2 / Omega_s) sum_ia sqrt(Delta_ia) F_{ia,s} P_ia.
* G0W0 in the time domain from those poles and the KS eigenstates.
"""
import numpy as np

from oracle import hamiltonian as ham


def eigenstates(g, vloc, kb=None):
    """Real eigenpairs of the dense grid Hamiltonian, orbitals normalised to dV sum phi^2 = 1."""
    H = ham.dense_h(g, vloc, kb).real
    H = 0.5 * (H + H.T)
    w, V = np.linalg.eigh(H)
    return w, V.T.reshape((-1,) + g.shape()) / np.sqrt(g.dV)


def casida(g, eps, phis, n_occ):
    """RPA excitation energies Omega_s and response densities rho_s (on the grid)."""
    occ = range(n_occ)
    vir = range(n_occ, len(eps))
    pairs = [(i, a) for i in occ for a in vir]
    P = np.array([phis[i] * phis[a] for i, a in pairs])           # [npair, n, n, n]
    D = np.array([eps[a] - eps[i] for i, a in pairs])
    vP = ham.poisson(P, g).real
    Vm = g.dV * np.einsum('pxyz,qxyz->pq', P, vP)
    Vm = 0.5 * (Vm + Vm.T)
    sd = np.sqrt(D)
    C = np.diag(D * D) + 4.0 * sd[:, None] * Vm * sd[None, :]
    om2, F = np.linalg.eigh(C)
    om = np.sqrt(om2)
    rho = np.einsum('ps,pxyz->sxyz', (sd[:, None] * F) * np.sqrt(2.0 / om)[None, :], P)
    return om, rho


def induced_potential_modes(g, rho):
    """w_s = v_C * rho_s."""
    return ham.poisson(rho, g).real
