"""Shared fixtures for the GPU parity tests: seeded synthetic systems, their oracle-side
eigen data, and helpers to move arrays between numpy (oracle, FP64) and torch (CUDA path)."""
import numpy as np
import scipy.sparse.linalg as sla

from oracle import hamiltonian as ham
from oracle import chebyshev as cheb
from oracle import sgw as osgw
from paper_2601_21005_gb300 import synth


def oracle_eigs(sysd, k):
    """Lowest k eigenpairs of H0 by ARPACK on the oracle's H (orbitals normalised, sign fixed)."""
    g = ham.Grid(sysd['n'], sysd['h'])
    kb = ham.KB(sysd['kb_atoms']) if sysd['kb_atoms'] else None
    n = g.n

    def mv(x):
        return ham.apply_h(x.reshape(n, n, n).astype(np.complex128), g, sysd['vloc'], kb).real.reshape(-1)

    op = sla.LinearOperator((g.ng, g.ng), matvec=mv, dtype=np.float64)
    w, v = sla.eigsh(op, k=k, which='SA', tol=1e-10, v0=np.ones(g.ng))
    order = np.argsort(w)
    w, v = w[order], v[:, order]
    phis = v.T.reshape((k, n, n, n)) / np.sqrt(g.dV)
    for i in range(k):
        if phis[i].sum() < 0:
            phis[i] = -phis[i]
    return g, kb, w, phis


def small_cluster(n=32, h=0.5):
    """Si5H12 on a 32^3 grid with s/p KB projectors on Si (and s on H, to exercise 1-projector atoms)."""
    hp = dict(synth.H_PARAMS)
    hp['Es'] = 0.3
    return synth.si_cluster(n=n, h=h, radius=4.5, hp=hp)


def to_dev(a, torch, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device='cuda', dtype=dtype)


def rel_err(a, b):
    """max |a - b| / max |b| (elementwise, scaled by the reference's largest magnitude)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
