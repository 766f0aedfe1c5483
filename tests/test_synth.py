"""The seeded input generators follow their recipe: rigid-water geometry, distance floors,
neutral charges, the frame and exclusion conventions, rigid moves that keep each water's
shape, replica sizes and polarization groups, and the same arrays from the same seed."""
import numpy as np

from paper_2011_01207_gb300 import synth


def _min_image(v, box):
    return v - box * np.round(v / box)


def test_water_box_geometry_floors_and_conventions():
    s = synth.water_box(64, 12.4, 5)
    assert s.n == 192 and np.allclose(s.box, 12.4)
    o, h1, h2 = s.xyz[0::3], s.xyz[1::3], s.xyz[2::3]
    for h in (h1, h2):
        np.testing.assert_allclose(np.linalg.norm(h - o, axis=1), synth.R_OH, atol=1e-12)
    cosang = np.einsum("ia,ia->i", h1 - o, h2 - o) / synth.R_OH ** 2
    np.testing.assert_allclose(np.arccos(np.clip(cosang, -1, 1)), synth.THETA_HOH, atol=1e-9)
    d = _min_image(s.xyz[:, None, :] - s.xyz[None, :, :], s.box)
    r = np.linalg.norm(d, axis=-1)
    other = s.mol[:, None] != s.mol[None, :]
    assert r[other].min() >= 1.7 - 1e-12
    assert abs(s.q.sum()) < 1e-12
    # oxygen: bisector frame on its two hydrogens; hydrogens: z toward O, x toward the other H
    np.testing.assert_array_equal(s.frame[0::3], np.stack([np.full(64, synth.FRAME_BISECTOR),
                                                            np.arange(64) * 3 + 1, np.arange(64) * 3 + 2], 1))
    np.testing.assert_array_equal(s.frame[1::3, :2], np.stack([np.full(64, synth.FRAME_Z_THEN_X), np.arange(64) * 3], 1))
    assert {tuple(p) for p in s.excl} == {(3 * m + a, 3 * m + b) for m in range(64) for a, b in ((0, 1), (0, 2), (1, 2))}
    # traceless quadrupoles
    np.testing.assert_allclose(s.quad[:, 0] + s.quad[:, 3] + s.quad[:, 5], 0.0, atol=1e-12)


def test_solvated_chain_recipe():
    s = synth.solvated_chain(40, 60, 18.0, 9)
    chain = np.nonzero(s.rigid == 0)[0]
    assert len(chain) == 40 and s.n == 40 + 180
    bonds = np.linalg.norm(np.diff(s.xyz[chain], axis=0), axis=1)
    np.testing.assert_allclose(bonds, 1.53, atol=1e-9)
    d = np.linalg.norm(s.xyz[chain][:, None] - s.xyz[chain][None], axis=-1)
    far = np.abs(np.arange(40)[:, None] - np.arange(40)[None]) >= 3
    assert d[far].min() >= 2.2 - 1e-9
    assert abs(s.q[chain].sum()) < 1e-12 and abs(s.q.sum()) < 1e-12
    assert np.all(s.frame[chain, 0] == synth.FRAME_NONE)
    np.testing.assert_allclose(s.quad[chain, 0] + s.quad[chain, 3] + s.quad[chain, 5], 0.0, atol=1e-12)
    assert set(np.round(s.alpha[chain], 3)) <= set(synth.CHAIN_ALPHAS)
    ex = {tuple(p) for p in s.excl}
    assert all((i, i + 1) in ex and (i, i + 2) in ex for i in range(38)) and (38, 39) in ex
    w = np.nonzero(s.rigid == 1)[0]
    dw = _min_image(s.xyz[w][:, None] - s.xyz[chain][None], s.box)
    assert np.linalg.norm(dw, axis=-1).min() >= 2.2 - 1e-9


def test_perturb_moves_waters_rigidly():
    s = synth.water_box(27, 9.3, 11)
    p = synth.perturb(s, 3, sigma_t=0.05, sigma_r=0.1)
    for a in (s, p):
        o, h1, h2 = a.xyz[0::3], a.xyz[1::3], a.xyz[2::3]
        np.testing.assert_allclose(np.linalg.norm(h1 - o, axis=1), synth.R_OH, atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(h2 - h1, axis=1),
                                   np.linalg.norm(s.xyz[2::3] - s.xyz[1::3], axis=1), atol=1e-12)
    step = np.linalg.norm(p.xyz[0::3] - s.xyz[0::3], axis=1)
    assert 0.02 < step.mean() < 0.15                       # ~ sigma_t sqrt(8/pi) for 3-D N(0, 0.05)
    np.testing.assert_array_equal(synth.perturb(s, 3, 0.05, 0.1).xyz, p.xyz)


def test_replicas_and_groups():
    sz = synth.replica_sizes(64, 648, 24000, 1005)
    assert len(sz) == 64 and sz.min() >= 645 and sz.max() <= 24000 and np.all(sz % 3 == 0)
    np.testing.assert_array_equal(sz, synth.replica_sizes(64, 648, 24000, 1005))
    s = synth.solvated_chain(30, 20, 14.0, 21)
    g = synth.polarization_groups(s, 7)
    chain = np.nonzero(s.rigid == 0)[0]
    runs = np.bincount(g[chain])
    assert runs[:-1].min() >= 3 and runs.max() <= 6 and np.all(np.diff(g[chain]) >= 0)
    w = np.nonzero(s.rigid == 1)[0]
    assert np.all(np.bincount(g[w] - g[w].min()) == 3)     # one group per water
    assert set(g[chain]).isdisjoint(set(g[w]))


def test_same_seed_same_arrays():
    a, b = synth.water_box(27, 9.3, 11), synth.water_box(27, 9.3, 11)
    for k in ("xyz", "q", "dip", "quad", "alpha", "frame", "excl"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.xyz, synth.water_box(27, 9.3, 12).xyz)
