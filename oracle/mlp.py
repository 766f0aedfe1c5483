"""The learned initial-guess network in FP64 (oracle).

Per atom, rotation-invariant features f_i (the permanent field, the short-range
first-order induced field and the fields at its frame atoms, all expressed in the atom's
local frame, plus its polarizability and frame kind)
pass through a two-hidden-layer perceptron
    h1 = relu(f W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 W3 + b3,
and the guess is mu0_i = alpha_i E_i + s_out R_i y_i (R_i the atom's frame). Training
minimises L = (1 / 2B) sum_i |y_i - t_i|^2 over a batch of B atoms, with t_i the
converged dipole's correction to alpha_i E_i in the local frame, divided by s_out.
Adam updates follow Kingma & Ba (2015).
"""
import numpy as np

from . import frames

N_FEAT = 16
E_SCALE = 0.05      # typical permanent-field magnitude, e/A^2
OUT_SCALE = 0.02    # typical correction magnitude, e*A


SHORT_RANGE = 4.0   # A


def short_field(n, I, J, R, alpha, E, beta, thole_a, rs=SHORT_RANGE):
    """E1_i = sum over pairs closer than rs of the real-space dipole field of alpha_j E_j."""
    from .realspace import real_dipole_field
    keep = np.einsum("pa,pa->p", R, R) < rs * rs
    return real_dipole_field(n, I[keep], J[keep], R[keep], alpha[:, None] * E, alpha, beta, thole_a)


def features(xyz, box, frame, alpha, E, E1):
    """Feature matrix [N, 16], fields divided by E_SCALE: E_i and E1_i in the atom's
    frame (3 + 3), E at the z-atom and x-atom in i's frame (3 + 3), |E_i|, |E1_i|,
    alpha_i, frame kind (0 global, 0.5 Z-then-X, 1 bisector)."""
    n = xyz.shape[0]
    rot = frames.frame_matrices(xyz, box, frame)
    e = E / E_SCALE
    loc = np.einsum("nba,nb->na", rot, e)
    loc1 = np.einsum("nba,nb->na", rot, E1 / E_SCALE)
    fz = np.where(frame[:, 1] >= 0, frame[:, 1], np.arange(n))
    fx = np.where(frame[:, 2] >= 0, frame[:, 2], np.arange(n))
    has = (frame[:, 0] != 0)[:, None]
    ez = np.where(has, np.einsum("nba,nb->na", rot, e[fz]), 0.0)
    ex = np.where(has, np.einsum("nba,nb->na", rot, e[fx]), 0.0)
    kind = np.array([0.0, 0.5, 1.0])[frame[:, 0]]
    return np.concatenate([loc, loc1, ez, ex, np.linalg.norm(loc, axis=1, keepdims=True),
                           np.linalg.norm(loc1, axis=1, keepdims=True), alpha[:, None], kind[:, None]],
                          axis=1), rot


def forward(params, X, round_hidden=None):
    """round_hidden (optional) is applied to the hidden activations before they enter the
    next layer, to emulate a reduced-precision storage of them; None keeps FP64."""
    W1, b1, W2, b2, W3, b3 = params
    rh = round_hidden or (lambda a: a)
    Z1 = X @ W1 + b1
    H1 = rh(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2 + b2
    H2 = rh(np.maximum(Z2, 0.0))
    Y = H2 @ W3 + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grads(params, X, T):
    """L = (1/2B) sum |Y - T|^2 and its gradients w.r.t. (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    Y, (X, Z1, H1, Z2, H2) = forward(params, X)
    B = X.shape[0]
    dY = (Y - T) / B
    L = 0.5 * np.sum((Y - T) ** 2) / B
    dW3 = H2.T @ dY
    db3 = dY.sum(0)
    dZ2 = (dY @ W3.T) * (Z2 > 0)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2.T) * (Z1 > 0)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(0)
    return L, (dW1, db1, dW2, db2, dW3, db3)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed, nin=N_FEAT, nh=128, nout=3):
    """He-style seeded initialisation (the random numbers the method draws, as inputs)."""
    rng = np.random.default_rng(seed)
    return [rng.normal(size=(nin, nh)) * np.sqrt(2.0 / nin), np.zeros(nh),
            rng.normal(size=(nh, nh)) * np.sqrt(2.0 / nh), np.zeros(nh),
            rng.normal(size=(nh, nout)) * np.sqrt(1.0 / nh), np.zeros(nout)]


def flatten(params):
    return np.concatenate([p.ravel() for p in params])


def unflatten(v, nin=N_FEAT, nh=128, nout=3):
    shapes = [(nin, nh), (nh,), (nh, nh), (nh,), (nh, nout), (nout,)]
    out, k = [], 0
    for sh in shapes:
        m = int(np.prod(sh))
        out.append(np.asarray(v[k:k + m], np.float64).reshape(sh))
        k += m
    return out


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** t)
        vh = vv / (1 - b2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v


def guess(params, xyz, box, frame, alpha, E, E1, round_input=None, round_hidden=None):
    """mu0 = alpha E + OUT_SCALE * R y."""
    X, rot = features(xyz, box, frame, alpha, E, E1)
    if round_input is not None:
        X = round_input(X)
    Y, _ = forward(params, X, round_hidden)
    return alpha[:, None] * E + OUT_SCALE * np.einsum("nab,nb->na", rot, Y)


def targets(xyz, box, frame, alpha, E, mu):
    """Local-frame correction t = R^T (mu - alpha E) / OUT_SCALE."""
    rot = frames.frame_matrices(xyz, box, frame)
    return np.einsum("nba,nb->na", rot, mu - alpha[:, None] * E) / OUT_SCALE
