"""Pair enumeration for the real-space sums (oracle, FP64).

Real-space Ewald terms run over every ordered pair (i, j, image n) with
|x_i - x_j + n L| < r_c, excluding i = j at n = 0 (Sec. 1.2.1 "Real space scheme":
pairs within a cutoff). Three enumerations are provided; each returns ordered pairs
(I, J, R) with R = x_I - x_J + n L, the vector from source J to target I.
"""
import numpy as np


def _ordered(i, j, rij):
    return (np.concatenate([i, j]), np.concatenate([j, i]), np.concatenate([rij, -rij]))


def pairs_min_image(xyz, box, rc):
    """Minimum-image pairs within rc; requires rc < min(box)/2 so that at most one image
    of each atom is inside the cutoff. Brute force for small N, a periodic k-d tree
    (SciPy) for large N; both give the same set."""
    xyz = np.asarray(xyz, np.float64)
    box = np.asarray(box, np.float64)
    assert rc < 0.5 * box.min(), "minimum-image enumeration needs rc < L/2"
    n = xyz.shape[0]
    if n <= 2500:
        i, j = np.triu_indices(n, 1)
        d = xyz[i] - xyz[j]
        d -= box * np.round(d / box)
        keep = np.einsum("ij,ij->i", d, d) < rc * rc
        return _ordered(i[keep], j[keep], d[keep])
    from scipy.spatial import cKDTree
    w = np.mod(xyz, box)
    w[w >= box] = 0.0
    pr = cKDTree(w, boxsize=box).query_pairs(rc, output_type="ndarray")
    i, j = pr[:, 0], pr[:, 1]
    d = xyz[i] - xyz[j]
    d -= box * np.round(d / box)
    keep = np.einsum("ij,ij->i", d, d) < rc * rc
    return _ordered(i[keep], j[keep], d[keep])


def pairs_images(xyz, box, rc):
    """All ordered (i, j, n) within rc over enough periodic images; includes an atom's own
    images (i = j, n != 0). For small systems and large cutoffs (convergence tests)."""
    xyz = np.asarray(xyz, np.float64)
    box = np.asarray(box, np.float64)
    n = xyz.shape[0]
    nimg = np.ceil(rc / box).astype(int) + 1
    shifts = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in nimg], indexing="ij"), -1).reshape(-1, 3)
    shifts = shifts * box
    I, J, R = [], [], []
    base = xyz[:, None, :] - xyz[None, :, :]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for s in shifts:
        d = base + s
        r2 = np.einsum("ijk,ijk->ij", d, d)
        keep = (r2 < rc * rc) & ~((ii == jj) & (np.abs(s).sum() == 0))
        I.append(ii[keep])
        J.append(jj[keep])
        R.append(d[keep])
    return np.concatenate(I), np.concatenate(J), np.concatenate(R)


def pairs_open(xyz):
    """All ordered pairs i != j without periodicity (isolated clusters)."""
    n = xyz.shape[0]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = ii != jj
    return ii[keep], jj[keep], (xyz[:, None, :] - xyz[None, :, :])[keep]


def scale_of_pairs(I, J, excl, n, R=None, box=None):
    """sigma = 0 for pairs listed in excl (either order), 1 otherwise. With R and box
    given, only the minimum image of an excluded pair gets sigma = 0 (the bonded
    partner itself, not its periodic copies)."""
    if len(excl) == 0:
        return np.ones(len(I))
    a = np.minimum(excl[:, 0], excl[:, 1]).astype(np.int64)
    b = np.maximum(excl[:, 0], excl[:, 1]).astype(np.int64)
    keys = np.unique(a * n + b)
    lo = np.minimum(I, J).astype(np.int64)
    hi = np.maximum(I, J).astype(np.int64)
    hit = np.isin(lo * n + hi, keys)
    if R is not None:
        mi = R - box * np.round(R / box)
        hit &= np.all(np.abs(mi - R) < 1e-9, axis=1)
    return np.where(hit, 0.0, 1.0)


def scales_from_table(I, J, table_pairs, table_values, n, R=None, box=None):
    """Per-pair scale factor looked up in a table of unordered pairs (i, j) with values;
    pairs not in the table get 1. With R and box given, only the minimum image of a listed
    pair takes the table value (as in scale_of_pairs)."""
    out = np.ones(len(I))
    if len(table_pairs) == 0:
        return out
    a = np.minimum(table_pairs[:, 0], table_pairs[:, 1]).astype(np.int64)
    b = np.maximum(table_pairs[:, 0], table_pairs[:, 1]).astype(np.int64)
    keys = a * n + b
    order = np.argsort(keys)
    keys, vals = keys[order], np.asarray(table_values, np.float64)[order]
    lo = np.minimum(I, J).astype(np.int64)
    hi = np.maximum(I, J).astype(np.int64)
    k = lo * n + hi
    pos = np.clip(np.searchsorted(keys, k), 0, len(keys) - 1)
    hit = keys[pos] == k
    if R is not None:
        mi = R - box * np.round(R / box)
        hit &= np.all(np.abs(mi - R) < 1e-9, axis=1)
    out[hit] = vals[pos[hit]]
    return out
