"""FP64 oracle: the split-operator propagator (the paper's own time stepper, Sec. 3).

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.

One step of length dt is the symmetric (palindromic, hence second-order and time-reversible)
product

    S(dt) = K_desc(dt/2) e^{-i V dt/2} e^{-i T dt} e^{-i V dt/2} K_asc(dt/2),

applied right to left: the Kleinman-Bylander factors first, then the local potential V, the
kinetic operator T (exact in k space), V again and the KB factors in reverse order.  The KB part
V_NL = sum_a V_a is split atom by atom: V_a = C_a E_a C_a^T with C_a = sqrt(dV) [beta_a0 ..],
and with the thin QR factorisation C_a = Q_a R_a (orthonormal columns) one gets exactly

    e^{-i tau V_a} = 1 + Q_a (e^{-i tau M_a} - 1) Q_a^T,   M_a = R_a E_a R_a^T.

Atoms whose supports overlap do not commute; the atoms are grouped into colours (greedy, in atom
order: the lowest colour not used by an earlier overlapping atom), atoms of one colour have
disjoint supports and commute, and K_asc applies the colours 0, 1, .., C-1, K_desc the reverse.
"""
import numpy as np

from . import hamiltonian as ham


class KBSplit:
    """Per-atom factors of the split KB part: supports, Q_a and M_a, and the colours."""

    def __init__(self, atoms, grid):
        self.sup, self.q, self.m = [], [], []
        for s, beta, e in atoms:
            s = np.asarray(s, dtype=np.int64)
            c = np.sqrt(grid.dV) * np.asarray(beta, dtype=np.float64).T      # [n_sup, n_proj]
            q, r = np.linalg.qr(c)
            self.sup.append(s)
            self.q.append(q)
            self.m.append(r @ np.diag(np.asarray(e, dtype=np.float64)) @ r.T)
        self.colour = colours(self.sup, grid.ng)
        self.n_colours = (max(self.colour) + 1) if self.colour else 0

    def factor(self, a, tau):
        """The small matrix e^{-i tau M_a} - 1 (via the eigenvectors of the symmetric M_a)."""
        lam, w = np.linalg.eigh(self.m[a])
        return (w * (np.exp(-1j * tau * lam) - 1.0)) @ w.T

    def apply(self, psi, tau, descending):
        """The product of e^{-i tau V_a} over all atoms, colours ascending or descending."""
        flat = psi.reshape(-1).copy()
        order = range(self.n_colours - 1, -1, -1) if descending else range(self.n_colours)
        for c in order:
            for a in range(len(self.sup)):
                if self.colour[a] != c:
                    continue
                s, q = self.sup[a], self.q[a]
                flat[s] += q @ (self.factor(a, tau) @ (q.T @ flat[s]))
        return flat.reshape(psi.shape)


def colours(supports, ng):
    """Greedy colouring of the atoms: atom a gets the lowest colour not used by an earlier atom
    whose support shares a grid point with its own."""
    used_at = {}
    col = []
    for a, s in enumerate(supports):
        taken = set()
        for g in s:
            for b in used_at.get(int(g), ()):
                taken.add(col[b])
        c = 0
        while c in taken:
            c += 1
        col.append(c)
        for g in s:
            used_at.setdefault(int(g), []).append(a)
    return col


def split_step(psi, grid, vloc, kbs, dt):
    """One step S(dt) of the symmetric split-operator scheme (dt < 0 propagates backwards)."""
    x = psi.astype(np.complex128)
    if kbs is not None:
        x = kbs.apply(x, 0.5 * dt, descending=False)
    half = np.exp(-0.5j * dt * vloc)
    x = half * x
    x = np.fft.ifftn(np.exp(-1j * dt * grid.T) * np.fft.fftn(x))
    x = half * x
    if kbs is not None:
        x = kbs.apply(x, 0.5 * dt, descending=True)
    return x


def split_propagate(psi, grid, vloc, kbs, dt, n_steps):
    x = psi.astype(np.complex128)
    for _ in range(n_steps):
        x = split_step(x, grid, vloc, kbs, dt)
    return x


def split_step_tangent(psi, dpsi, grid, v, dv, kbs, dt):
    """One split step of psi under the local potential v and its derivative along v -> v + lam dv:

        a = K_asc psi,             da = K_asc dpsi
        b = e^{-i v dt/2} a,       db = e^{-i v dt/2} (da - i (dt/2) dv a)
        c = e^{-i T dt} b,         dc = e^{-i T dt} db
        d = e^{-i v dt/2} c,       dd = e^{-i v dt/2} (dc - i (dt/2) dv c)
        psi' = K_desc d,           dpsi' = K_desc dd
    (v and dv are diagonal and commute, so d/dlam e^{-i (v + lam dv) dt/2} = -i (dt/2) dv e^{-i v dt/2})."""
    x, dx = psi.astype(np.complex128), dpsi.astype(np.complex128)
    if kbs is not None:
        x = kbs.apply(x, 0.5 * dt, descending=False)
        dx = kbs.apply(dx, 0.5 * dt, descending=False)
    half = np.exp(-0.5j * dt * v)
    x, dx = half * x, half * (dx - 0.5j * dt * dv * x)
    kin = np.exp(-1j * dt * grid.T)
    x = np.fft.ifftn(kin * np.fft.fftn(x))
    dx = np.fft.ifftn(kin * np.fft.fftn(dx))
    x, dx = half * x, half * (dx - 0.5j * dt * dv * x)
    if kbs is not None:
        x = kbs.apply(x, 0.5 * dt, descending=True)
        dx = kbs.apply(dx, 0.5 * dt, descending=True)
    return x, dx
