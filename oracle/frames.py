"""Local multipole frames (oracle, FP64).

AMOEBA gives each atom's dipole and quadrupole in a local frame fixed by bonded
neighbours; the global multipoles rotate with the molecule, so forces include the
frame-atom terms (torques). Frame vectors use the minimum image.

  Z-then-X: z = unit(v_z), x = unit(v_x - (v_x.z) z), y = z cross x,
            with v_z = x_Zatom - x_i, v_x = x_Xatom - x_i.
  Bisector: u1 = unit(v_z), u2 = unit(v_x), z = unit(u1 + u2),
            x = unit(u2 - (u2.z) z), y = z cross x.
  None:     the global frame.
R has the local axes as columns: d_global = R d_local, Q_global = R Q_local R^T.
"""
import numpy as np

FRAME_NONE, FRAME_Z_THEN_X, FRAME_BISECTOR = 0, 1, 2


def quad6_to_mat(q6):
    """[..., 6] (xx, xy, xz, yy, yz, zz) -> [..., 3, 3] symmetric."""
    xx, xy, xz, yy, yz, zz = np.moveaxis(q6, -1, 0)
    return np.stack([np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1),
                     np.stack([xz, yz, zz], -1)], -2)


def min_image(v, box):
    return v - box * np.round(v / box)


def _unit(v):
    n = np.linalg.norm(v, axis=-1, keepdims=True)
    return v / n, n


def frame_matrices(xyz, box, frame):
    """Rotation matrices R [N,3,3] (columns x, y, z axes) and the intermediate vectors."""
    n = xyz.shape[0]
    rot = np.tile(np.eye(3), (n, 1, 1))
    ftype, fz, fx = frame[:, 0], frame[:, 1], frame[:, 2]
    for t in (FRAME_Z_THEN_X, FRAME_BISECTOR):
        idx = np.nonzero(ftype == t)[0]
        if len(idx) == 0:
            continue
        vz = min_image(xyz[fz[idx]] - xyz[idx], box)
        vx = min_image(xyz[fx[idx]] - xyz[idx], box)
        if t == FRAME_Z_THEN_X:
            z, _ = _unit(vz)
            w = vx - np.einsum("ij,ij->i", vx, z)[:, None] * z
        else:
            u1, _ = _unit(vz)
            u2, _ = _unit(vx)
            z, _ = _unit(u1 + u2)
            w = u2 - np.einsum("ij,ij->i", u2, z)[:, None] * z
        x, _ = _unit(w)
        y = np.cross(z, x)
        rot[idx] = np.stack([x, y, z], -1)
    return rot


def rotate_multipoles(xyz, box, frame, dip_local, quad_local):
    """Global dipoles [N,3] and quadrupole matrices [N,3,3]."""
    rot = frame_matrices(xyz, box, frame)
    dip = np.einsum("nab,nb->na", rot, dip_local)
    ql = quad6_to_mat(quad_local)
    quad = np.einsum("nab,nbc,ndc->nad", rot, ql, rot)
    return dip, quad, rot


def _frame_vector_gradients(xyz, box, frame, dip_local, quad_local, g_dip, g_quad):
    """dU/dv_z and dU/dv_x of every framed atom from dU/d(global dipole) [N,3] and
    dU/d(global quadrupole) [N,3,3] (symmetric), by the chain rule through the frame
    construction. Yields (atoms, z atoms, x atoms, dU/dv_z, dU/dv_x, v_z, v_x) per kind."""
    rot = frame_matrices(xyz, box, frame)
    ql = quad6_to_mat(quad_local)
    g_quad = 0.5 * (g_quad + np.swapaxes(g_quad, 1, 2))
    # dU/dR = G_d d_l^T + 2 G_Q R Q_l
    g_rot = np.einsum("na,nb->nab", g_dip, dip_local) + 2.0 * np.einsum("nab,nbc,ncd->nad", g_quad, rot, ql)
    ftype, fz, fx = frame[:, 0], frame[:, 1], frame[:, 2]

    def dot(a, b):
        return np.einsum("ij,ij->i", a, b)[:, None]

    for t in (FRAME_Z_THEN_X, FRAME_BISECTOR):
        idx = np.nonzero(ftype == t)[0]
        if len(idx) == 0:
            continue
        R = rot[idx]
        xa, za = R[:, :, 0], R[:, :, 2]
        gx, gy, gz = g_rot[idx, :, 0], g_rot[idx, :, 1], g_rot[idx, :, 2]
        # y = z cross x
        gx = gx + np.cross(gy, za)
        gz = gz + np.cross(xa, gy)
        vz = min_image(xyz[fz[idx]] - xyz[idx], box)
        vx = min_image(xyz[fx[idx]] - xyz[idx], box)
        if t == FRAME_Z_THEN_X:
            w = vx - dot(vx, za) * za
            gw = (gx - dot(gx, xa) * xa) / np.linalg.norm(w, axis=1, keepdims=True)
            g_vx = gw - dot(gw, za) * za
            gz = gz - dot(gw, za) * vx - dot(vx, za) * gw
            g_vz = (gz - dot(gz, za) * za) / np.linalg.norm(vz, axis=1, keepdims=True)
        else:
            u1, n1 = _unit(vz)
            u2, n2 = _unit(vx)
            s = u1 + u2
            w = u2 - dot(u2, za) * za
            gw = (gx - dot(gx, xa) * xa) / np.linalg.norm(w, axis=1, keepdims=True)
            g_u2 = gw - dot(gw, za) * za
            gz = gz - dot(gw, za) * u2 - dot(u2, za) * gw
            g_s = (gz - dot(gz, za) * za) / np.linalg.norm(s, axis=1, keepdims=True)
            g_u1 = g_s
            g_u2 = g_u2 + g_s
            g_vz = (g_u1 - dot(g_u1, u1) * u1) / n1
            g_vx = (g_u2 - dot(g_u2, u2) * u2) / n2
        yield idx, fz[idx], fx[idx], g_vz, g_vx, vz, vx


def frame_gradient(xyz, box, frame, dip_local, quad_local, g_dip, g_quad):
    """dU/dx [N,3] from dU/d(global dipole) [N,3] and dU/d(global quadrupole) [N,3,3]
    (symmetric), by the chain rule through the frame construction: v_z = x_Z - x_i and
    v_x = x_X - x_i, so x_Z and x_X receive dU/dv and atom i minus their sum."""
    out = np.zeros((xyz.shape[0], 3))
    for idx, iz, ix, g_vz, g_vx, _, _ in _frame_vector_gradients(xyz, box, frame, dip_local, quad_local,
                                                                   g_dip, g_quad):
        np.add.at(out, iz, g_vz)
        np.add.at(out, ix, g_vx)
        np.add.at(out, idx, -(g_vz + g_vx))
    return out


def frame_virial(xyz, box, frame, dip_local, quad_local, g_dip, g_quad):
    """The frames' share of dU/d(strain) [3,3]: a homogeneous deformation x -> (I + e) x
    maps each frame vector v to (I + e) v, so it contributes sum (dU/dv)_a v_b over the
    frame vectors of every atom (U's dependence on the global multipoles only)."""
    V = np.zeros((3, 3))
    for _, _, _, g_vz, g_vx, vz, vx in _frame_vector_gradients(xyz, box, frame, dip_local, quad_local,
                                                                 g_dip, g_quad):
        V += np.einsum("na,nb->ab", g_vz, vz) + np.einsum("na,nb->ab", g_vx, vx)
    return V
