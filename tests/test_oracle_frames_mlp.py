"""Pins for the oracle's local frames (geometry, and the chain rule checked on a test
function linear in the global multipoles) and for its MLP gradients and Adam step."""
import numpy as np

from oracle import frames, mlp


def test_frames_geometry(water_small):
    s = water_small
    R = frames.frame_matrices(s.xyz, s.box, s.frame)
    np.testing.assert_allclose(np.einsum("nab,nac->nbc", R, R), np.tile(np.eye(3), (s.n, 1, 1)), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)
    o, h1, h2 = 0, 1, 2
    u1 = s.xyz[h1] - s.xyz[o]
    u2 = s.xyz[h2] - s.xyz[o]
    u1 /= np.linalg.norm(u1)
    u2 /= np.linalg.norm(u2)
    np.testing.assert_allclose(R[o][:, 2].dot(u1), R[o][:, 2].dot(u2), atol=1e-14)   # bisector
    np.testing.assert_allclose(R[h1][:, 2], -u1, atol=1e-14)                          # z toward O
    # the dipole of each water O points along its bisector
    d, Q, _ = frames.rotate_multipoles(s.xyz, s.box, s.frame, s.dip, s.quad)
    np.testing.assert_allclose(np.cross(d[o], R[o][:, 2]), 0.0, atol=1e-15)
    np.testing.assert_allclose(np.trace(Q, axis1=1, axis2=2), 0.0, atol=1e-15)


def test_frame_chain_rule_by_finite_differences(water_small):
    s = water_small
    rng = np.random.default_rng(3)
    gd = rng.normal(size=(s.n, 3))
    gq = rng.normal(size=(s.n, 3, 3))
    gq = 0.5 * (gq + gq.transpose(0, 2, 1))

    def U(x):
        d, Q, _ = frames.rotate_multipoles(x, s.box, s.frame, s.dip, s.quad)
        return np.sum(gd * d) + np.sum(gq * Q)
    grad = frames.frame_gradient(s.xyz, s.box, s.frame, s.dip, s.quad, gd, gq)
    h = 1e-6
    fd = np.zeros_like(grad)
    for i in range(s.n):
        for a in range(3):
            xp, xm = s.xyz.copy(), s.xyz.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd[i, a] = (U(xp) - U(xm)) / (2 * h)
    np.testing.assert_allclose(grad, fd, atol=1e-8)


def _params(rng, nin=16, nh=32, nout=3):
    return [rng.normal(size=(nin, nh)) * 0.3, rng.normal(size=nh) * 0.1,
            rng.normal(size=(nh, nh)) * 0.2, rng.normal(size=nh) * 0.1,
            rng.normal(size=(nh, nout)) * 0.2, rng.normal(size=nout) * 0.1]


def test_mlp_gradients_by_finite_differences():
    rng = np.random.default_rng(5)
    P = _params(rng)
    X = rng.normal(size=(7, 16))
    T = rng.normal(size=(7, 3))
    L, G = mlp.loss_and_grads(P, X, T)
    h = 1e-6
    for k in range(6):
        flat = P[k].ravel()
        for idx in rng.choice(flat.size, min(5, flat.size), replace=False):
            Pp = [p.copy() for p in P]
            Pm = [p.copy() for p in P]
            Pp[k].ravel()[idx] += h
            Pm[k].ravel()[idx] -= h
            fd = (mlp.loss_and_grads(Pp, X, T)[0] - mlp.loss_and_grads(Pm, X, T)[0]) / (2 * h)
            assert abs(fd - G[k].ravel()[idx]) < 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_is_signed_lr():
    """With zero moments, Adam's first bias-corrected step is lr * g / (|g| + eps)."""
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    out, m, v = mlp.adam_step(p, g, [np.zeros(3)], [np.zeros(3)], 1, 0.01)
    np.testing.assert_allclose(out[0], p[0] - 0.01 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-12)


def test_features_rotation_invariant(water_small):
    s = water_small
    rng = np.random.default_rng(1)
    E = rng.normal(size=(s.n, 3))
    E1 = rng.normal(size=(s.n, 3))
    X, _ = mlp.features(s.xyz, s.box, s.frame, s.alpha, E, E1)
    x = s.xyz
    rot = lambda v: np.stack([-v[:, 1], v[:, 0], v[:, 2]], 1)
    Xr, _ = mlp.features(rot(x), s.box, s.frame, s.alpha, rot(E), rot(E1))
    np.testing.assert_allclose(Xr, X, atol=1e-12)


def test_bf16_round_ties_to_even():
    # 1 + 2^-8 is halfway between bfloat16 neighbours 1 and 1 + 2^-7: ties go to even (1)
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-3])
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, -2.5, 197 * 2.0 ** -16])   # 3e-3 = 196.6 * 2^-16
    np.testing.assert_array_equal(mlp.bf16_round(vals), want)
