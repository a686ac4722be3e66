"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

The paper takes its inputs (atomic coordinates, pseudopotentials, the ground-state
density, E_HOMO / E_LUMO and the target orbital; Sec. 2.1) from a preliminary DFT
calculation on relaxed Si_xH_y clusters (Sec. 3, Table 1).  None of those is
available here, so this module builds synthetic stand-ins of the same shape:

* `wells`: a periodic box with Gaussian local wells placed from a seed (the tiny
  16^3 case);
* `si_cluster`: an H-capped Si cluster cut from the diamond lattice (a = 10.26 bohr,
  Sec. 3) to a sphere around an atom, with H at 2.8 bohr along each missing bond,
  Gaussian local pseudopotentials and s/p Gaussian Kleinman-Bylander projectors.

It produces only input arrays (a local potential on the grid, projector supports
and values, atom lists).  It holds none of the method's arithmetic: no Hamiltonian
application, filtering, propagation or self-energy.
"""
import numpy as np

SI_A = 10.26          # diamond lattice constant of Si, bohr (Sec. 3)
SI_H_BOND = 2.8       # Si-H cap distance, bohr

# Synthetic pseudopotential parameters (Hartree, bohr).  Local part: -D exp(-r^2 / 2 s^2);
# KB projectors: s ~ exp(-r^2 / 2 sk^2), p_m ~ (x_m / sk) exp(-r^2 / 2 sk^2), cut at 4 sk,
# each normalised to <beta|beta> = 1 on the grid, with energy E_l.
SI_PARAMS = dict(D=2.2, s=1.15, sk=0.9, Es=1.2, Ep=-0.25)
H_PARAMS = dict(D=1.6, s=0.75, sk=0.6, Es=0.0)


def grid_coords(n, h):
    """Cartesian coordinates (z, y, x order of axes) of the grid points of the periodic box."""
    c = h * np.arange(n)
    return np.meshgrid(c, c, c, indexing='ij')   # Z, Y, X


def min_image(d, L):
    return d - L * np.round(d / L)


def gaussian_wells_potential(n, h, centers, depths, widths):
    """V(r) = -sum_a D_a exp(-|r - R_a|^2 / (2 w_a^2)) with minimum-image distances.

    Each Gaussian is evaluated where it exceeds exp(-37) of its depth (|r - R_a| <= sqrt(74) w_a),
    on a periodic box around R_a when that box is shorter than the cell, else on the whole grid."""
    L = n * h
    v = np.zeros((n, n, n))
    Z = Y = X = None
    for (cx, cy, cz), d, w in zip(centers, depths, widths):
        rc = np.sqrt(74.0) * w
        if 2.0 * rc + 2.0 * h < L:
            c = np.array([cx, cy, cz])
            lo = np.floor((c - rc) / h).astype(int)
            hi = np.ceil((c + rc) / h).astype(int)
            ix, iy, iz = (np.arange(lo[k], hi[k] + 1) for k in range(3))
            dx = ix * h - cx
            dy = iy * h - cy
            dz = iz * h - cz
            g = np.exp(-(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) / (2.0 * w * w))
            v[np.ix_(iz % n, iy % n, ix % n)] -= d * g
        else:
            if Z is None:
                Z, Y, X = grid_coords(n, h)
            dx = min_image(X - cx, L)
            dy = min_image(Y - cy, L)
            dz = min_image(Z - cz, L)
            v -= d * np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * w * w))
    return v


def wells(n=16, h=0.6, n_sites=6, seed=1000, width=1.2, depth=(1.0, 3.0), min_sep=2.0, n_elec=8):
    """The tiny periodic case: n_sites Gaussian wells (depth U[1,3] Ha, width 1.2 bohr)."""
    rng = np.random.default_rng(seed)
    L = n * h
    centers = []
    while len(centers) < n_sites:
        c = rng.uniform(0.0, L, size=3)
        ok = all(np.linalg.norm(min_image(c - np.array(o), L)) >= min_sep for o in centers)
        if ok:
            centers.append(tuple(c))
    depths = rng.uniform(depth[0], depth[1], size=n_sites)
    v = gaussian_wells_potential(n, h, centers, depths, [width] * n_sites)
    return dict(name='wells%d' % n, n=n, h=h, vloc=v, kb_atoms=[], n_occ=n_elec // 2,
                centers=np.array(centers), depths=depths)


def diamond_cluster(radius, a=SI_A):
    """Si positions of the diamond lattice within `radius` of an atom at the origin,
    and H caps along the missing tetrahedral bonds.  Returns (si [N,3], h [M,3])."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    basis = np.vstack([fcc, fcc + 0.25])
    m = int(np.ceil(radius / a)) + 1
    pts = []
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                for b in basis:
                    pts.append((np.array([i, j, k]) + b) * a)
    pts = np.array(pts)
    si = pts[np.linalg.norm(pts, axis=1) <= radius + 1e-9]
    bond = a / 4.0 * np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    key = lambda p: tuple(np.round(p / (a / 4.0)).astype(int))
    have = {key(p) for p in si}
    hs = []
    for p in si:
        # sublattice A (integer quarter-coordinates summing to 0 mod 4) bonds along +bond, B along -bond
        q = np.round(p / (a / 4.0)).astype(int)
        sgn = 1.0 if (q.sum() % 4) == 0 else -1.0
        for d in bond:
            nb = p + sgn * d
            if key(nb) not in have:
                hs.append(p + sgn * d / np.linalg.norm(d) * SI_H_BOND)
    return si, np.array(hs)


def kb_projectors(n, h, center, sk, energies, lmax):
    """Support and values of the s (and p) Gaussian KB projectors of one atom.

    Returns (support flat indices, beta [n_proj, n_sup], e [n_proj]) with every
    projector normalised to dV sum beta^2 = 1 on the grid.
    """
    L = n * h
    rc = 4.0 * sk
    # integer box around the centre, wrapped periodically
    lo = np.floor((np.array(center) - rc) / h).astype(int)
    hi = np.ceil((np.array(center) + rc) / h).astype(int)
    ix = np.arange(lo[0], hi[0] + 1)
    iy = np.arange(lo[1], hi[1] + 1)
    iz = np.arange(lo[2], hi[2] + 1)
    IZ, IY, IX = np.meshgrid(iz, iy, ix, indexing='ij')
    dx = IX * h - center[0]
    dy = IY * h - center[1]
    dz = IZ * h - center[2]
    r2 = dx * dx + dy * dy + dz * dz
    inside = r2 <= rc * rc
    dx, dy, dz, r2 = dx[inside], dy[inside], dz[inside], r2[inside]
    flat = ((IZ[inside] % n) * n + (IY[inside] % n)) * n + (IX[inside] % n)
    g = np.exp(-r2 / (2.0 * sk * sk))
    rows = [g]
    es = [energies[0]]
    if lmax >= 1:
        rows += [dx / sk * g, dy / sk * g, dz / sk * g]
        es += [energies[1]] * 3
    beta = np.array(rows)
    dV = h ** 3
    beta /= np.sqrt(dV * np.sum(beta * beta, axis=1, keepdims=True))
    order = np.argsort(flat)
    assert len(np.unique(flat)) == len(flat), 'projector sphere wraps onto itself'
    return flat[order].astype(np.int64), beta[:, order], np.array(es, dtype=np.float64)


def si_cluster(n=64, h=0.5, radius=10.5, si=SI_PARAMS, hp=H_PARAMS, with_kb=True):
    """H-capped Si cluster centred in the periodic box (35 Si + 36 H at radius 10.5 bohr)."""
    si_pos, h_pos = diamond_cluster(radius)
    L = n * h
    shift = np.full(3, 0.5 * L)
    si_pos = si_pos + shift
    h_pos = h_pos + shift
    centers = list(map(tuple, si_pos)) + list(map(tuple, h_pos))
    depths = [si['D']] * len(si_pos) + [hp['D']] * len(h_pos)
    widths = [si['s']] * len(si_pos) + [hp['s']] * len(h_pos)
    v = gaussian_wells_potential(n, h, centers, depths, widths)
    kb_atoms = []
    if with_kb:
        for p in si_pos:
            kb_atoms.append(kb_projectors(n, h, p, si['sk'], (si['Es'], si['Ep']), 1))
        if hp.get('Es', 0.0) != 0.0:
            for p in h_pos:
                kb_atoms.append(kb_projectors(n, h, p, hp['sk'], (hp['Es'],), 0))
    n_elec = 4 * len(si_pos) + len(h_pos)
    return dict(name='Si%dH%d' % (len(si_pos), len(h_pos)), n=n, h=h, vloc=v, kb_atoms=kb_atoms,
                n_occ=n_elec // 2, si=si_pos, hpos=h_pos)


def smooth_orbital(n, h, center, width=2.0):
    """A normalised Gaussian orbital (a stand-in target state for parity-only checks)."""
    Z, Y, X = grid_coords(n, h)
    L = n * h
    dx = min_image(X - center[0], L)
    dy = min_image(Y - center[1], L)
    dz = min_image(Z - center[2], L)
    f = np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * width * width))
    return f / np.sqrt(h ** 3 * np.sum(f * f))
