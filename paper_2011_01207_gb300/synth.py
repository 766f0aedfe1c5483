"""Seeded synthetic inputs for the polarization solve.

Rigid-water boxes, a random-walk chain solvated in water, and small rigid-body moves
that stand in for MD steps. The paper's benchmark systems (water boxes from 648 atoms
up, DHFR at 23,558 atoms, STMV at ~1.07 M atoms; Sec. 2.2 error study, Sec. 3 tables)
are represented here only by their sizes and densities.

This module places atoms and assigns parameters. It holds none of the method's
arithmetic: no local frame is evaluated, no field, no solve. The CUDA library and the
FP64 oracle both take its arrays as inputs, and neither is imported here.

Multipole values are synthetic (AMOEBA-like magnitudes with the symmetry each frame
allows); they are conventions, not fitted parameters.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FRAME_NONE = 0        # multipoles given in the global frame
FRAME_Z_THEN_X = 1    # z toward the z-atom, x from the x-atom orthogonalised
FRAME_BISECTOR = 2    # z along the bisector of the two frame bonds, x from the x-atom

# rigid water geometry
R_OH = 0.9572
THETA_HOH = np.deg2rad(104.52)

# synthetic water multipoles in each atom's local frame (e, e*A, e*A^2; traceless)
WATER_Q = (-0.51966, 0.25983)
WATER_DIP = (np.array([0.0, 0.0, 0.076]), np.array([-0.020, 0.0, -0.031]))
# xx, xy, xz, yy, yz, zz
WATER_QUAD = (np.array([0.200, 0.0, 0.0, -0.220, 0.0, 0.020]),
              np.array([-0.019, 0.0, -0.029, -0.054, 0.0, 0.073]))
WATER_ALPHA = (0.837, 0.496)
CHAIN_ALPHAS = (1.334, 1.073, 0.837, 0.496)


@dataclass
class System:
    """Atom arrays in the caller's order. Lengths in A, charges in e."""
    xyz: np.ndarray          # [N,3] float64 (any periodic image)
    box: np.ndarray          # [3] float64 orthorhombic edge lengths
    q: np.ndarray            # [N]
    dip: np.ndarray          # [N,3] local-frame dipole, e*A
    quad: np.ndarray         # [N,6] local-frame traceless quadrupole xx,xy,xz,yy,yz,zz, e*A^2
    alpha: np.ndarray        # [N] isotropic polarizability, A^3
    frame: np.ndarray        # [N,3] int32: frame type, z-atom, x-atom (-1 if unused)
    excl: np.ndarray         # [M,2] int32 pairs i<j with permanent->induced scale 0
    mol: np.ndarray          # [N] int32 molecule index
    rigid: np.ndarray = field(default=None)   # [N] int32: 1 for rigid-water atoms

    @property
    def n(self) -> int:
        return self.xyz.shape[0]

    def copy(self) -> "System":
        return System(*(np.array(getattr(self, k)) for k in
                        ("xyz", "box", "q", "dip", "quad", "alpha", "frame", "excl", "mol", "rigid")))

    def excl_csr(self):
        """Exclusions as CSR over atoms (both directions): offsets [N+1], atoms [2M]."""
        n = self.n
        a = np.concatenate([self.excl[:, 0], self.excl[:, 1]])
        b = np.concatenate([self.excl[:, 1], self.excl[:, 0]])
        order = np.lexsort((b, a))
        a, b = a[order], b[order]
        offs = np.zeros(n + 1, np.int32)
        np.add.at(offs, a + 1, 1)
        return np.cumsum(offs).astype(np.int32), b.astype(np.int32)


def _random_rotations(rng, n):
    """Uniform random rotation matrices from normalised Gaussian quaternions."""
    qt = rng.normal(size=(n, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    w, x, y, z = qt.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _water_template():
    """O, H1, H2 in a molecule-fixed frame with the bisector along +z."""
    s, c = np.sin(THETA_HOH / 2), np.cos(THETA_HOH / 2)
    return np.array([[0.0, 0.0, 0.0], [R_OH * s, 0.0, R_OH * c], [-R_OH * s, 0.0, R_OH * c]])


def _close_molecules(xyz, box, mol, dmin):
    """Molecule ids owning an atom closer than dmin to an atom of another molecule."""
    from scipy.spatial import cKDTree
    wrapped = np.mod(xyz, box)
    wrapped[wrapped >= box] = 0.0
    tree = cKDTree(wrapped, boxsize=box)
    pairs = tree.query_pairs(dmin, output_type="ndarray")
    if len(pairs) == 0:
        return np.zeros(0, np.int64)
    inter = mol[pairs[:, 0]] != mol[pairs[:, 1]]
    return np.unique(mol[pairs[inter].ravel()])


def _orient_waters(rng, o_sites, box, dmin_inter, fixed_xyz=None, dmin_fixed=None,
                   max_rounds=400):
    """Random orientations for waters whose O sits at o_sites; redraw clashing ones."""
    m = len(o_sites)
    tmpl = _water_template()
    rot = _random_rotations(rng, m)
    for _ in range(max_rounds):
        xyz = (o_sites[:, None, :] + np.einsum("mab,kb->mka", rot, tmpl)).reshape(-1, 3)
        mol = np.repeat(np.arange(m), 3)
        bad = _close_molecules(xyz, box, mol, dmin_inter)
        if fixed_xyz is not None:
            from scipy.spatial import cKDTree
            t = cKDTree(np.mod(fixed_xyz, box) % box, boxsize=box)
            hits = t.query_ball_point(np.mod(xyz, box) % box, dmin_fixed, return_length=True)
            bad = np.union1d(bad, np.unique(mol[hits > 0]))
        if len(bad) == 0:
            return xyz
        rot[bad] = _random_rotations(rng, len(bad))
    raise RuntimeError("could not place waters without clashes")


def _water_arrays(xyz_w, offset):
    """Parameters, frames and exclusions for consecutive O,H,H waters."""
    m = xyz_w.shape[0] // 3
    n = 3 * m
    q = np.tile([WATER_Q[0], WATER_Q[1], WATER_Q[1]], m)
    dip = np.tile(np.stack([WATER_DIP[0], WATER_DIP[1], WATER_DIP[1]]), (m, 1))
    quad = np.tile(np.stack([WATER_QUAD[0], WATER_QUAD[1], WATER_QUAD[1]]), (m, 1))
    alpha = np.tile([WATER_ALPHA[0], WATER_ALPHA[1], WATER_ALPHA[1]], m)
    base = offset + 3 * np.arange(m)
    frame = np.empty((n, 3), np.int32)
    frame[0::3] = np.stack([np.full(m, FRAME_BISECTOR), base + 1, base + 2], 1)
    frame[1::3] = np.stack([np.full(m, FRAME_Z_THEN_X), base, base + 2], 1)
    frame[2::3] = np.stack([np.full(m, FRAME_Z_THEN_X), base, base + 1], 1)
    excl = np.concatenate([np.stack([base, base + 1], 1), np.stack([base, base + 2], 1),
                           np.stack([base + 1, base + 2], 1)]).astype(np.int32)
    return q, dip, quad, alpha, frame, excl


def water_box(n_mol: int, box_len: float, seed: int, jitter: float = 0.12,
              dmin_inter: float = 1.7) -> System:
    """n_mol rigid waters, O on a jittered cubic lattice, uniform random orientations.

    O-H 0.9572 A, H-O-H 104.52 deg. Orientations are redrawn until no atom pair of two
    different molecules is closer than dmin_inter.
    """
    rng = np.random.default_rng(seed)
    box = np.full(3, float(box_len))
    nl = int(np.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    g = (np.arange(nl) + 0.5) * (box_len / nl)
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if len(sites) > n_mol:
        sites = sites[np.sort(rng.choice(len(sites), n_mol, replace=False))]
    sites = sites + rng.uniform(-jitter, jitter, size=sites.shape)
    xyz = _orient_waters(rng, sites, box, dmin_inter)
    q, dip, quad, alpha, frame, excl = _water_arrays(xyz, 0)
    mol = np.repeat(np.arange(n_mol), 3).astype(np.int32)
    return System(xyz, box, q, dip, quad, alpha, frame, excl, mol, np.ones(3 * n_mol, np.int32))


def _random_walk_chain(rng, n, box, radius, bond=1.53, angle_deg=111.0, dmin=2.2):
    """Self-avoiding walk with fixed bond length and angle, confined to a sphere.

    Non-bonded atoms (|i - j| >= 3) stay at least dmin apart (periodic); earlier atoms
    are looked up in a cell hash of edge >= dmin."""
    center = box / 2
    ang = np.deg2rad(angle_deg)
    ncell = np.maximum(1, np.floor(box / dmin).astype(int))
    csize = box / ncell
    cells = {}
    keys = [None] * n

    def key(p):
        return tuple((np.floor(np.mod(p, box) / csize).astype(int)) % ncell)

    def add(i, p):
        k = key(p)
        keys[i] = k
        cells.setdefault(k, []).append(i)

    def remove_from(i0):
        for j in range(i0, n):
            if keys[j] is None:
                break
            cells[keys[j]].remove(j)
            keys[j] = None

    def clear(p, i):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((k[0] + dx) % ncell[0], (k[1] + dy) % ncell[1], (k[2] + dz) % ncell[2])
                    for j in cells.get(kk, ()):
                        if j <= i - 3:
                            d = pts[j] - p
                            d -= box * np.round(d / box)
                            if d.dot(d) < dmin * dmin:
                                return False
        return True

    pts = np.zeros((n, 3))
    # a walk trapped in a dense globule can backtrack for a very long time: after 40 n
    # placement rounds it restarts from a new first bond, and gives up after 5 restarts
    for restart in range(6):
        if restart:
            cells.clear()
            for j in range(n):
                keys[j] = None
        pts[0] = center + rng.normal(size=3)
        add(0, pts[0])
        if n > 1:
            d = rng.normal(size=3)
            pts[1] = pts[0] + bond * d / np.linalg.norm(d)
            add(1, pts[1])
        i = 2
        fails = 0
        rounds = 0
        while i < n and rounds < 40 * n:
            rounds += 1
            b1 = pts[i - 1] - pts[i - 2]
            b1 /= np.linalg.norm(b1)
            ok = False
            for _ in range(60):
                perp = rng.normal(size=3)
                perp -= perp.dot(b1) * b1
                perp /= np.linalg.norm(perp)
                cand = pts[i - 1] + bond * (np.cos(np.pi - ang) * b1 + np.sin(np.pi - ang) * perp)
                if np.linalg.norm(cand - center) > radius:
                    continue
                if clear(cand, i):
                    ok = True
                    break
            if ok:
                pts[i] = cand
                add(i, cand)
                i += 1
                fails = 0
            else:
                fails += 1
                i = max(2, i - 1 - min(fails, 20))   # backtrack
                remove_from(i)
        if i >= n:
            return pts
    raise RuntimeError(f"self-avoiding walk of {n} atoms did not finish; lower globule_density or dmin")


def solvated_chain(n_chain: int, n_water: int, box_len: float, seed: int,
                   dmin_chain: float = 2.2, dmin_solv: float = 2.2,
                   dmin_inter: float = 1.6, globule_density: float = 0.055) -> System:
    """Random-walk chain (globule) with random multipoles, surrounded by rigid waters.

    Chain: bonds 1.53 A, angle 111 deg, non-bonded atoms >= dmin_chain apart, inside a
    sphere sized for a loose globule. Charges ~N(0,0.3) made neutral, dipoles ~N(0,0.1)
    per component, quadrupoles sym(N(0,0.1)) with the trace removed, polarizabilities
    drawn from {1.334, 1.073, 0.837, 0.496}; multipoles are in the global frame; 1-2 and
    1-3 pairs have permanent->induced scale 0. The walk is confined to a sphere holding
    the chain at globule_density atoms/A^3. Waters fill lattice sites at least dmin_solv
    (+ the O-H reach) away from every chain atom.
    """
    rng = np.random.default_rng(seed)
    box = np.full(3, float(box_len))
    radius = (3.0 * n_chain / (4.0 * np.pi * globule_density)) ** (1.0 / 3.0) + 1.0
    chain = _random_walk_chain(rng, n_chain, box, radius, dmin=dmin_chain) if n_chain else np.zeros((0, 3))
    qc = rng.normal(0.0, 0.3, n_chain)
    qc -= qc.mean() if n_chain else 0.0
    dc = rng.normal(0.0, 0.1, (n_chain, 3))
    g = rng.normal(0.0, 0.1, (n_chain, 3, 3))
    g = 0.5 * (g + g.transpose(0, 2, 1))
    g -= np.eye(3)[None] * (np.trace(g, axis1=1, axis2=2) / 3.0)[:, None, None]
    quadc = np.stack([g[:, 0, 0], g[:, 0, 1], g[:, 0, 2], g[:, 1, 1], g[:, 1, 2], g[:, 2, 2]], 1)
    alc = rng.choice(CHAIN_ALPHAS, n_chain)
    framec = np.tile(np.array([FRAME_NONE, -1, -1], np.int32), (n_chain, 1))
    exc = [np.stack([np.arange(n_chain - k), np.arange(k, n_chain)], 1) for k in (1, 2) if n_chain > k]
    exclc = np.concatenate(exc).astype(np.int32) if exc else np.zeros((0, 2), np.int32)

    # candidate O sites on a lattice finer than the water spacing, away from the chain;
    # refined (down to 2.55 A, above the 2.5 A O-O floor) until there are enough of them
    nl = int(np.floor(box_len / 2.9))
    while True:
        gg = (np.arange(nl) + 0.5) * (box_len / nl)
        sites = np.stack(np.meshgrid(gg, gg, gg, indexing="ij"), -1).reshape(-1, 3)
        if n_chain:
            from scipy.spatial import cKDTree
            t = cKDTree(np.mod(chain, box) % box, boxsize=box)
            near = t.query_ball_point(sites, dmin_solv + R_OH, return_length=True)
            sites = sites[near == 0]
        if len(sites) >= 1.05 * n_water or box_len / (nl + 1) < 2.55:
            break
        nl += 1
    if len(sites) < n_water:
        raise RuntimeError(f"only {len(sites)} free water sites for {n_water} waters")
    sites = sites[np.sort(rng.choice(len(sites), n_water, replace=False))]
    sites = sites + rng.uniform(-0.1, 0.1, sites.shape)
    xyz_w = _orient_waters(rng, sites, box, dmin_inter,
                           fixed_xyz=chain if n_chain else None, dmin_fixed=dmin_solv)
    q, dip, quad, alpha, frame, excl = _water_arrays(xyz_w, n_chain)
    mol = np.concatenate([np.zeros(n_chain, np.int32), 1 + np.repeat(np.arange(n_water), 3)]).astype(np.int32)
    return System(
        np.concatenate([chain, xyz_w]), box,
        np.concatenate([qc, q]), np.concatenate([dc, dip]), np.concatenate([quadc, quad]),
        np.concatenate([alc, alpha]), np.concatenate([framec, frame]).astype(np.int32),
        np.concatenate([exclc, excl]).astype(np.int32), mol,
        np.concatenate([np.zeros(n_chain, np.int32), np.ones(3 * n_water, np.int32)]))


def perturb(sys: System, seed: int, sigma_t: float = 0.005, sigma_r: float = 0.01) -> System:
    """One synthetic 'MD step': rigid waters translate ~N(0, sigma_t) per axis and rotate
    about their O by an angle vector ~N(0, sigma_r); other atoms move ~N(0, sigma_t)."""
    rng = np.random.default_rng(seed)
    out = sys.copy()
    n = sys.n
    rigid = sys.rigid if sys.rigid is not None else np.zeros(n, np.int32)
    free = np.nonzero(rigid == 0)[0]
    out.xyz[free] += rng.normal(0.0, sigma_t, (len(free), 3))
    o_idx = np.nonzero((rigid == 1) & (sys.frame[:, 0] == FRAME_BISECTOR))[0]
    if len(o_idx):
        h1 = sys.frame[o_idx, 1]
        h2 = sys.frame[o_idx, 2]
        w = rng.normal(0.0, sigma_r, (len(o_idx), 3))
        th = np.linalg.norm(w, axis=1, keepdims=True)
        k = w / np.maximum(th, 1e-300)
        t = rng.normal(0.0, sigma_t, (len(o_idx), 3))
        for h in (h1, h2):
            v = sys.xyz[h] - sys.xyz[o_idx]
            v = v * np.cos(th) + np.cross(k, v) * np.sin(th) + k * np.einsum("ij,ij->i", k, v)[:, None] * (1 - np.cos(th))
            out.xyz[h] = sys.xyz[o_idx] + t + v
        out.xyz[o_idx] = sys.xyz[o_idx] + t
    return out


def water_velocities(sys: System, temperature: float, seed: int) -> np.ndarray:
    """Seeded initial velocities (A/fs) for an MD run of a water-only system: every atom
    ~N(0, kB T / m) per axis (O 15.999, H 1.008 amu; kB = 0.0019872041 kcal/mol/K and
    1 kcal/mol/amu = 4.184e-4 A^2/fs^2), the total momentum removed. The integrator projects
    them onto the rigid-water constraints itself."""
    rng = np.random.default_rng(seed)
    m = np.full(sys.n, 1.008)
    m[0::3] = 15.999
    sd = np.sqrt(0.0019872041 * temperature * 4.184e-4 / m)
    v = rng.normal(size=(sys.n, 3)) * sd[:, None]
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return v


def water_cfg(n_mol: int) -> float:
    """Cubic edge (A) for n_mol waters at 0.0333 molecules/A^3 (the configs' density)."""
    return (n_mol / 0.03334) ** (1.0 / 3.0)


def replica_sizes(n_rep: int, lo: int, hi: int, seed: int):
    """Seeded replica sizes (atoms, rounded down to whole waters) uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return (rng.integers(lo, hi + 1, n_rep) // 3 * 3).astype(np.int64)


# AMOEBA's scale factors of the two induced-dipole sets (force-field inputs, not part of
# the method's arithmetic): the direct field (d) is scaled by 0 between atoms of the same
# polarization group; the polarization field (p) by 0 for 1-2 and 1-3 pairs and by 1/2 for
# 1-4 pairs inside one group; every other pair, and the mutual field, by 1.
D_SCALE_SAME_GROUP = 0.0
P_SCALE_12_13 = 0.0
P_SCALE_14_SAME_GROUP = 0.5


def polarization_groups(sys: System, seed: int, lo: int = 3, hi: int = 6) -> np.ndarray:
    """Group index per atom: every water is one group; the chain (consecutive atoms of
    molecule 0 that are not rigid) is cut into consecutive runs of U[lo, hi] atoms."""
    rng = np.random.default_rng(seed)
    rigid = sys.rigid if sys.rigid is not None else np.zeros(sys.n, np.int32)
    chain = np.nonzero(rigid == 0)[0]
    grp = np.empty(sys.n, np.int64)
    g, k = 0, 0
    while k < len(chain):
        m = int(rng.integers(lo, hi + 1))
        grp[chain[k:k + m]] = g
        g += 1
        k += m
    water = np.nonzero(rigid == 1)[0]
    if len(water):
        grp[water] = g + (sys.mol[water] - sys.mol[water].min())
    return grp


def dp_scales(sys: System, groups: np.ndarray):
    """Pairs whose d or p scale differs from 1, with (d, p) scales: (pairs [M,2] int32 with
    i < j, scales [M,2] float64). Bonds: chain atoms k, k+1 and water O-H; 1-3 and 1-4
    pairs follow along the chain, and H-H inside a water."""
    rigid = sys.rigid if sys.rigid is not None else np.zeros(sys.n, np.int32)
    chain = np.nonzero(rigid == 0)[0]
    table = {}

    def put(i, j, d, p):
        a, b = (int(i), int(j)) if i < j else (int(j), int(i))
        table[(a, b)] = (d, p)

    for sep in (1, 2, 3):
        for a, b in zip(chain[:-sep], chain[sep:]):
            same = groups[a] == groups[b]
            d = D_SCALE_SAME_GROUP if same else 1.0
            p = P_SCALE_12_13 if sep < 3 else (P_SCALE_14_SAME_GROUP if same else 1.0)
            if (d, p) != (1.0, 1.0):
                put(a, b, d, p)
    # same-group chain pairs beyond 1-4: d scaled only
    for g in np.unique(groups[chain]) if len(chain) else ():
        mem = chain[groups[chain] == g]
        for x in range(len(mem)):
            for y in range(x + 1, len(mem)):
                if (min(mem[x], mem[y]), max(mem[x], mem[y])) not in table:
                    put(mem[x], mem[y], D_SCALE_SAME_GROUP, 1.0)
    # waters: O-H (1-2) and H-H (1-3), one group each
    for a, b in sys.excl:
        if rigid[a] == 1 and rigid[b] == 1:
            put(a, b, D_SCALE_SAME_GROUP, P_SCALE_12_13)
    keys = sorted(table)
    pairs = np.array(keys, np.int32).reshape(-1, 2)
    scales = np.array([table[k] for k in keys], np.float64).reshape(-1, 2)
    return pairs, scales


def dp_system(sys: System, seed: int, lo: int = 3, hi: int = 6):
    """(system, pairs, scales) for the two-dipole-set path: a copy of `sys` whose exclusion
    list is the set of scaled pairs (the pairs the pair kernels leave to the scaled-pair
    corrections), and the d/p scale table from dp_scales."""
    pairs, scales = dp_scales(sys, polarization_groups(sys, seed, lo, hi))
    out = sys.copy()
    out.excl = pairs.copy()
    return out, pairs, scales
