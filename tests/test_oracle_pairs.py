"""Pins of the oracle's pair enumeration (real-space sums run over every ordered pair and
periodic image within the cutoff) against counting that does not share its code: a plain
minimum-image double loop, lattice-point counts of an atom's own images, and the rule
that only the bonded partner itself, not its periodic copies, is excluded."""
import numpy as np

from oracle import pairs


def _sorted(I, J, R):
    o = np.lexsort((J, I))
    return I[o], J[o], R[o]


def test_kd_tree_path_equals_a_plain_double_loop():
    rng = np.random.default_rng(3)
    box = np.array([30.0, 27.0, 33.0])
    x = rng.uniform(-5.0, 40.0, size=(3000, 3))          # above the brute-force size; unwrapped
    rc = 4.5
    I, J, R = _sorted(*pairs.pairs_min_image(x, box, rc))
    want_I, want_J, want_R = [], [], []
    for i in range(len(x)):
        d = x[i] - x
        d -= box * np.round(d / box)
        hit = np.nonzero((np.einsum("ja,ja->j", d, d) < rc * rc) & (np.arange(len(x)) != i))[0]
        want_I.append(np.full(len(hit), i))
        want_J.append(hit)
        want_R.append(d[hit])
    wI, wJ, wR = _sorted(np.concatenate(want_I), np.concatenate(want_J), np.concatenate(want_R))
    assert np.array_equal(I, wI) and np.array_equal(J, wJ)
    np.testing.assert_allclose(R, wR, rtol=0, atol=1e-12)
    np.testing.assert_allclose(R, x[I] - x[J] - box * np.round((x[I] - x[J]) / box), atol=1e-12)


def test_image_enumeration_reduces_to_minimum_image_below_half_the_box():
    rng = np.random.default_rng(4)
    box = np.array([12.0, 12.0, 12.0])
    x = rng.uniform(0.0, 12.0, size=(60, 3))
    a = _sorted(*pairs.pairs_min_image(x, box, 5.5))
    b = _sorted(*pairs.pairs_images(x, box, 5.5))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    np.testing.assert_allclose(a[2], b[2], atol=1e-12)


def test_own_images_match_lattice_point_counts():
    """One atom in a cube of side L: its images within rc are the nonzero integer vectors
    with |n| L < rc - 6 at rc = 1.2 L (faces), 18 at 1.5 L (+ edges at sqrt 2), 26 at
    1.8 L (+ corners at sqrt 3), 32 at 2.1 L (+ the six at distance 2)."""
    box = np.array([5.0, 5.0, 5.0])
    for f, want in ((1.2, 6), (1.5, 18), (1.8, 26), (2.1, 32)):
        I, J, R = pairs.pairs_images(np.array([[1.0, 2.0, 3.0]]), box, f * 5.0)
        assert len(I) == want and np.all(I == 0) and np.all(J == 0)


def test_exclusion_applies_to_the_minimum_image_only():
    box = np.array([6.0, 6.0, 6.0])
    x = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0], [4.0, 4.0, 4.0]])
    excl = np.array([[1, 0]])                                # either order
    I, J, R = pairs.pairs_images(x, box, 8.0)                # several images of every pair
    sig = pairs.scale_of_pairs(I, J, excl, 3, R, box)
    zero = np.nonzero(sig == 0.0)[0]
    assert len(zero) == 2                                    # (0, 1) and (1, 0), nearest copy
    assert set(zip(I[zero], J[zero])) == {(0, 1), (1, 0)}
    np.testing.assert_allclose(np.abs(R[zero]).sum(1), 1.0)
    n01 = np.sum(((I == 0) & (J == 1)) | ((I == 1) & (J == 0)))
    assert n01 > 2                                           # the copies keep scale 1


def test_scale_table_lookup_in_either_order():
    I = np.array([0, 1, 2, 3, 2, 0])
    J = np.array([1, 0, 3, 2, 0, 3])
    table = np.array([[1, 0], [2, 3]])
    vals = np.array([0.25, 0.5])
    got = pairs.scales_from_table(I, J, table, vals, 4)
    np.testing.assert_array_equal(got, [0.25, 0.25, 0.5, 0.5, 1.0, 1.0])
    np.testing.assert_array_equal(pairs.scales_from_table(I, J, np.zeros((0, 2), int), [], 4), np.ones(6))
