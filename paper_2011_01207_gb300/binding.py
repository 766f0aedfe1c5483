"""ctypes binding of libamoebapol.so (argument marshalling only).

Every function has the name of the C entry point it calls and takes PyTorch CUDA tensors
(used only as device memory). Nothing here computes any part of the method: a missing
library or GPU raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

AP_OK, AP_NOT_CONVERGED = 0, 1
AP_MIXED, AP_FP64, AP_FIXED = 0, 1, 2
AP_ERR_NONFINITE = -4
_ERRORS = {-1: "AP_ERR_ARG", -2: "AP_ERR_CUDA", -4: "AP_ERR_NONFINITE",
           -5: "AP_ERR_TIMEOUT", -6: "AP_ERR_STATE"}

# every symbol the public header declares
EXPORTS = ("ap_create", "ap_destroy", "ap_last_error", "build_neighbour_blocks", "permanent_field",
           "induced_dipoles_pcg", "polarization_energy_forces", "dipole_field_matvec", "ap_list_stats",
           "ap_stream", "ap_solve_info_last", "ap_time_kernel", "polarization_energy_noalloc",
           "ap_mlp_param_count", "ap_mlp_packed_bytes", "ap_mlp_pack", "ap_mlp_forward", "ap_mlp_status",
           "ap_mlp_features", "ap_learned_guess", "ap_mlp_gradient", "ap_mlp_train_step",
           "ap_batch_create", "ap_batch_capture", "ap_batch_launch", "ap_batch_destroy", "ap_autotune",
           "ap_extrapolate_guess", "induced_dipoles_diis", "set_scaled_pairs", "permanent_field_dp",
           "induced_dipoles_pcg_dp", "polarization_energy_forces_dp", "ap_adaptive_guess", "ap_fp32_peak",
           "ap_eval_erfc", "ap_direct_guess", "ap_md_kick_drift", "ap_md_kick", "ap_lj_forces")
KERNELS = {"real_matvec": 0, "real_field": 1, "spread_dipoles": 2, "convolve": 3, "gather_field": 4,
           "spread_multipoles": 5, "pair_forces": 6,
           "pcg_vectors": 7, "real_matvec2": 8, "fft_roundtrip": 9, "pme_dipoles": 10, "dipole_operator": 11}


class ApParams(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("box", ctypes.c_double * 3), ("cutoff", ctypes.c_double),
                ("buffer", ctypes.c_double), ("ewald_beta", ctypes.c_double), ("grid", ctypes.c_int * 3),
                ("pme_order", ctypes.c_int), ("thole_a", ctypes.c_double), ("precision", ctypes.c_int)]


class ApSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("eps_debye", ctypes.c_double),
                ("eps_initial", ctypes.c_double)]


class ApBatchStep(ctypes.Structure):
    _fields_ = [("d_xyz", ctypes.c_void_p), ("d_mpole", ctypes.c_void_p), ("d_frame", ctypes.c_void_p),
                ("d_alpha", ctypes.c_void_p), ("d_mlp_packed", ctypes.c_void_p), ("d_mu0", ctypes.c_void_p),
                ("tol_debye", ctypes.c_double), ("max_iter", ctypes.c_int), ("d_mu", ctypes.c_void_p),
                ("d_energy", ctypes.c_void_p), ("d_forces", ctypes.c_void_p), ("d_hist", ctypes.c_void_p),
                ("d_hist_lsq", ctypes.c_void_p), ("d_virial", ctypes.c_void_p)]


class ApError(RuntimeError):
    """A failed call; `code` is the library's AP_ERR_* value (0 for a marshalling error)."""

    def __init__(self, msg, code=0):
        super().__init__(msg)
        self.code = code


_lib = None


def load(path: str = LIB) -> ctypes.CDLL:
    """Load the library (built by build.build_library); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ApError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "ap_create": (I, [ctypes.POINTER(P), ctypes.POINTER(ApParams), P]),
        "ap_destroy": (None, [P]),
        "ap_last_error": (ctypes.c_char_p, [P]),
        "build_neighbour_blocks": (I, [P, P, P, P, I]),
        "permanent_field": (I, [P, P, P, P, P, P]),
        "induced_dipoles_pcg": (I, [P, P, D, I, P, ctypes.POINTER(ApSolveInfo)]),
        "induced_dipoles_diis": (I, [P, P, D, I, I, P, ctypes.POINTER(ApSolveInfo)]),
        "ap_adaptive_guess": (I, [I, P, P, P, P, P, P, P, P, P, P]),
        "set_scaled_pairs": (I, [P, I, P, P]),
        "permanent_field_dp": (I, [P, P, P, P, P, P, P]),
        "induced_dipoles_pcg_dp": (I, [P, P, P, D, I, P, P, ctypes.POINTER(ApSolveInfo)]),
        "polarization_energy_forces_dp": (I, [P, P, P, P, P, P]),
        "polarization_energy_forces": (I, [P, P, P, P, P]),
        "dipole_field_matvec": (I, [P, P, P]),
        "ap_list_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "ap_stream": (P, [P]),
        "ap_solve_info_last": (I, [P, ctypes.POINTER(ApSolveInfo)]),
        "ap_time_kernel": (I, [P, I, I, ctypes.POINTER(D)]),
        "polarization_energy_noalloc": (I, [P, P, I, P, P]),
        "ap_extrapolate_guess": (I, [I, P, P, P, P, P, P, P]),
        "ap_mlp_param_count": (I, []),
        "ap_mlp_packed_bytes": (I, []),
        "ap_mlp_pack": (I, [P, P, P]),
        "ap_mlp_forward": (I, [P, P, I, P, P]),
        "ap_mlp_status": (I, []),
        "ap_mlp_features": (I, [P, P, P, P]),
        "ap_learned_guess": (I, [P, P, P]),
        "ap_mlp_gradient": (I, [P, P, P, I, P, P, P]),
        "ap_mlp_train_step": (I, [P, P, P, P, I, ctypes.c_float, P, P, I, P, P, P]),
        "ap_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I]),
        "ap_batch_capture": (I, [P, ctypes.POINTER(ApBatchStep)]),
        "ap_batch_launch": (I, [P, P]),
        "ap_batch_destroy": (None, [P]),
        "ap_autotune": (I, [P, I, ctypes.POINTER(I)]),
        "ap_fp32_peak": (I, [I, ctypes.POINTER(D), ctypes.POINTER(I)]),
        "ap_eval_erfc": (I, [P, I, P, P, P]),
        "ap_direct_guess": (I, [P, P]),
        "ap_md_kick_drift": (I, [I, P, ctypes.POINTER(D), P, D, P, P, P, P, P]),
        "ap_md_kick": (I, [I, P, ctypes.POINTER(D), P, D, P, P, P, D, P, P, P]),
        "ap_lj_forces": (I, [P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t, dtype=None, shape=None, name="tensor", allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ApError(f"{name} is required")
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ApError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ApError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ApError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ApError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, code, what):
    if code < 0:
        msg = load().ap_last_error(ctx).decode(errors="replace")
        raise ApError(f"{what} failed: {_ERRORS.get(code, code)}: {msg}", code)
    return code


def ap_create(params: ApParams, stream: int = 0):
    lib = load()
    ctx = ctypes.c_void_p()
    code = lib.ap_create(ctypes.byref(ctx), ctypes.byref(params), ctypes.c_void_p(stream))
    if code != 0:
        raise ApError(f"ap_create failed: {_ERRORS.get(code, code)}: {lib.ap_last_error(None).decode()}")
    return ctx


def ap_destroy(ctx):
    load().ap_destroy(ctx)


def build_neighbour_blocks(ctx, xyz, excl_offsets, excl_atoms, n_excl: int):
    import torch
    n = xyz.shape[0]
    return _check(ctx, load().build_neighbour_blocks(
        ctx, _ptr(xyz, torch.float64, (n, 3), "xyz"), _ptr(excl_offsets, torch.int32, (n + 1,), "excl_offsets"),
        _ptr(excl_atoms, torch.int32, None, "excl_atoms"), int(n_excl)), "build_neighbour_blocks")


def permanent_field(ctx, xyz, mpole, frame, alpha, field=None):
    import torch
    n = xyz.shape[0]
    return _check(ctx, load().permanent_field(
        ctx, _ptr(xyz, torch.float64, (n, 3), "xyz"), _ptr(mpole, torch.float64, (n, 10), "mpole"),
        _ptr(frame, torch.int32, (n, 3), "frame"), _ptr(alpha, torch.float64, (n,), "alpha"),
        _ptr(field, torch.float64, (n, 3), "field", allow_none=True)), "permanent_field")


def induced_dipoles_pcg(ctx, guess, tol_debye: float, max_iter: int, mu, want_info: bool = True):
    import torch
    n = mu.shape[0]
    info = ApSolveInfo()
    code = load().induced_dipoles_pcg(
        ctx, _ptr(guess, torch.float64, (n, 3), "guess", allow_none=True), float(tol_debye), int(max_iter),
        _ptr(mu, torch.float64, (n, 3), "mu"), ctypes.byref(info) if want_info else None)
    _check(ctx, code, "induced_dipoles_pcg")
    return info if want_info else None


def induced_dipoles_diis(ctx, guess, tol_debye: float, max_iter: int, depth: int, mu, want_info: bool = True):
    import torch
    n = mu.shape[0]
    info = ApSolveInfo()
    code = load().induced_dipoles_diis(
        ctx, _ptr(guess, torch.float64, (n, 3), "guess", allow_none=True), float(tol_debye), int(max_iter),
        int(depth), _ptr(mu, torch.float64, (n, 3), "mu"), ctypes.byref(info) if want_info else None)
    _check(ctx, code, "induced_dipoles_diis")
    return info if want_info else None


def set_scaled_pairs(ctx, pairs, scales):
    """pairs: int32 [m, 2] CUDA tensor (caller atom indices); scales: float64 [m, 2] (d, p)."""
    import torch
    m = int(pairs.shape[0])
    return _check(ctx, load().set_scaled_pairs(
        ctx, m, _ptr(pairs, torch.int32, (m, 2), "pairs", allow_none=m == 0),
        _ptr(scales, torch.float64, (m, 2), "scales", allow_none=m == 0)), "set_scaled_pairs")


def permanent_field_dp(ctx, xyz, mpole, frame, alpha, field_d=None, field_p=None):
    import torch
    n = xyz.shape[0]
    return _check(ctx, load().permanent_field_dp(
        ctx, _ptr(xyz, torch.float64, (n, 3), "xyz"), _ptr(mpole, torch.float64, (n, 10), "mpole"),
        _ptr(frame, torch.int32, (n, 3), "frame"), _ptr(alpha, torch.float64, (n,), "alpha"),
        _ptr(field_d, torch.float64, (n, 3), "field_d", allow_none=True),
        _ptr(field_p, torch.float64, (n, 3), "field_p", allow_none=True)), "permanent_field_dp")


def induced_dipoles_pcg_dp(ctx, guess_d, guess_p, tol_debye: float, max_iter: int, mu_d, mu_p,
                           want_info: bool = True):
    import torch
    n = mu_d.shape[0]
    info = ApSolveInfo()
    code = load().induced_dipoles_pcg_dp(
        ctx, _ptr(guess_d, torch.float64, (n, 3), "guess_d", allow_none=True),
        _ptr(guess_p, torch.float64, (n, 3), "guess_p", allow_none=True), float(tol_debye), int(max_iter),
        _ptr(mu_d, torch.float64, (n, 3), "mu_d"), _ptr(mu_p, torch.float64, (n, 3), "mu_p"),
        ctypes.byref(info) if want_info else None)
    _check(ctx, code, "induced_dipoles_pcg_dp")
    return info if want_info else None


def polarization_energy_forces_dp(ctx, mu_d, mu_p, energy, forces, virial=None):
    import torch
    n = mu_d.shape[0]
    return _check(ctx, load().polarization_energy_forces_dp(
        ctx, _ptr(mu_d, torch.float64, (n, 3), "mu_d"), _ptr(mu_p, torch.float64, (n, 3), "mu_p"),
        _ptr(energy, torch.float64, (1,), "energy"), _ptr(forces, torch.float64, (n, 3), "forces"),
        _ptr(virial, torch.float64, (3, 3), "virial", allow_none=True)), "polarization_energy_forces_dp")


def polarization_energy_forces(ctx, mu, energy, forces, virial=None):
    """virial: optional float64 [3, 3] CUDA tensor receiving V_ab = dE_pol/de_ab."""
    import torch
    n = mu.shape[0]
    return _check(ctx, load().polarization_energy_forces(
        ctx, _ptr(mu, torch.float64, (n, 3), "mu"), _ptr(energy, torch.float64, (1,), "energy"),
        _ptr(forces, torch.float64, (n, 3), "forces"), _ptr(virial, torch.float64, (3, 3), "virial", allow_none=True)),
        "polarization_energy_forces")


def dipole_field_matvec(ctx, v, out):
    import torch
    n = v.shape[0]
    return _check(ctx, load().dipole_field_matvec(
        ctx, _ptr(v, torch.float64, (n, 3), "v"), _ptr(out, torch.float64, (n, 3), "out")), "dipole_field_matvec")


def ap_list_stats(ctx):
    b, t, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    load().ap_list_stats(ctx, ctypes.byref(b), ctypes.byref(t), ctypes.byref(e))
    return b.value, t.value, e.value


def ap_solve_info_last(ctx):
    info = ApSolveInfo()
    _check(ctx, load().ap_solve_info_last(ctx, ctypes.byref(info)), "ap_solve_info_last")
    return info


def ap_time_kernel(ctx, which, reps=20):
    ms = ctypes.c_double()
    k = KERNELS[which] if isinstance(which, str) else int(which)
    _check(ctx, load().ap_time_kernel(ctx, k, int(reps), ctypes.byref(ms)), "ap_time_kernel")
    return ms.value


def polarization_energy_noalloc(mu, field, energy, stream=None):
    """Context-free energy (no device allocation); `stream` is a torch stream or None."""
    import torch
    n = mu.shape[0]
    for t, name in ((field, "field"), (energy, "energy")):
        if isinstance(t, torch.Tensor) and t.device != mu.device:
            raise ApError(f"{name} is on {t.device}, mu on {mu.device}: all three must be on one device")
    # the library launches on the current device with that device's scratch array
    with torch.cuda.device(mu.device):
        sp = ctypes.c_void_p((stream or torch.cuda.current_stream(mu.device)).cuda_stream)
        code = load().polarization_energy_noalloc(
            _ptr(mu, torch.float64, (n, 3), "mu"), _ptr(field, torch.float64, (n, 3), "field"), int(n),
            _ptr(energy, torch.float64, (1,), "energy"), sp)
    return _check(None, code, "polarization_energy_noalloc")


def ap_extrapolate_guess(out, mu1, mu2, base=None, base1=None, base2=None, stream=None):
    """out = base + 2 (mu1 - base1) - (mu2 - base2); None bases are zero (caller-order [n][3])."""
    import torch
    n = out.shape[0]
    opt = lambda t, name: None if t is None else _ptr(t, torch.float64, (n, 3), name)
    return _check(None, load().ap_extrapolate_guess(int(n), opt(base, "base"), _ptr(mu1, torch.float64, (n, 3), "mu1"),
                                                     opt(base1, "base1"), _ptr(mu2, torch.float64, (n, 3), "mu2"),
                                                     opt(base2, "base2"), _ptr(out, torch.float64, (n, 3), "out"),
                                                     _stream_ptr(out, stream)), "ap_extrapolate_guess")


AP_ADAPTIVE_SCRATCH = 520


def ap_adaptive_guess(out, mu1, mu2, mu3, scratch, base=None, base1=None, base2=None, base3=None, stream=None):
    """out = base + e1 + c (e1 - e2), e_k = mu_k - base_k, c the clamped least-squares
    coefficient from the three previous steps; scratch: zeroed float64 CUDA tensor of
    AP_ADAPTIVE_SCRATCH entries (scratch[0] holds c afterwards)."""
    import torch
    n = out.shape[0]
    opt = lambda t, name: None if t is None else _ptr(t, torch.float64, (n, 3), name)
    return _check(None, load().ap_adaptive_guess(
        int(n), opt(base, "base"), _ptr(mu1, torch.float64, (n, 3), "mu1"), opt(base1, "base1"),
        _ptr(mu2, torch.float64, (n, 3), "mu2"), opt(base2, "base2"), _ptr(mu3, torch.float64, (n, 3), "mu3"),
        opt(base3, "base3"), _ptr(out, torch.float64, (n, 3), "out"),
        _ptr(scratch, torch.float64, (AP_ADAPTIVE_SCRATCH,), "scratch"), _stream_ptr(out, stream)),
        "ap_adaptive_guess")


def _stream_ptr(t, stream=None):
    import torch
    return ctypes.c_void_p((stream or torch.cuda.current_stream(t.device)).cuda_stream)


def ap_mlp_param_count():
    return load().ap_mlp_param_count()


def ap_mlp_packed_bytes():
    return load().ap_mlp_packed_bytes()


def ap_mlp_pack(params, packed, stream=None):
    import torch
    _check(None, load().ap_mlp_pack(_ptr(params, torch.float32, (ap_mlp_param_count(),), "params"),
                                    _ptr(packed, torch.uint8, (ap_mlp_packed_bytes(),), "packed"),
                                    _stream_ptr(params, stream)), "ap_mlp_pack")


def ap_mlp_forward(packed, feat, y, stream=None):
    import torch
    n = feat.shape[0]
    _check(None, load().ap_mlp_forward(_ptr(packed, torch.uint8, (ap_mlp_packed_bytes(),), "packed"),
                                       _ptr(feat, torch.float32, (n, 16), "feat"), int(n),
                                       _ptr(y, torch.float32, (n, 3), "y"), _stream_ptr(feat, stream)),
           "ap_mlp_forward")


def ap_mlp_gradient(packed, feat, target, grad, loss, stream=None):
    import torch
    n = feat.shape[0]
    _check(None, load().ap_mlp_gradient(_ptr(packed, torch.uint8, (ap_mlp_packed_bytes(),), "packed"),
                                        _ptr(feat, torch.float32, (n, 16), "feat"),
                                        _ptr(target, torch.float32, (n, 3), "target"), int(n),
                                        _ptr(grad, torch.float32, (ap_mlp_param_count(),), "grad"),
                                        _ptr(loss, torch.float64, (1,), "loss"), _stream_ptr(feat, stream)),
           "ap_mlp_gradient")


def ap_mlp_train_step(params, grad, m, v, step, lr, feat, target, loss, packed, stream=None):
    import torch
    n = feat.shape[0]
    P = ap_mlp_param_count()
    _check(None, load().ap_mlp_train_step(
        _ptr(params, torch.float32, (P,), "params"), _ptr(grad, torch.float32, (P,), "grad"),
        _ptr(m, torch.float32, (P,), "m"), _ptr(v, torch.float32, (P,), "v"), int(step), float(lr),
        _ptr(feat, torch.float32, (n, 16), "feat"), _ptr(target, torch.float32, (n, 3), "target"), int(n),
        _ptr(loss, torch.float64, (1,), "loss"), _ptr(packed, torch.uint8, (ap_mlp_packed_bytes(),), "packed"),
        _stream_ptr(feat, stream)), "ap_mlp_train_step")


def ap_mlp_status():
    return _check(None, load().ap_mlp_status(), "ap_mlp_status")


def ap_mlp_features(ctx, feat, mu=None, target=None):
    import torch
    n = feat.shape[0]
    _check(ctx, load().ap_mlp_features(ctx, _ptr(mu, torch.float64, (n, 3), "mu", allow_none=True),
                                       _ptr(feat, torch.float32, (n, 16), "feat"),
                                       _ptr(target, torch.float32, (n, 3), "target", allow_none=True)),
           "ap_mlp_features")


def _lengths(h):
    arr = (ctypes.c_double * 3)(*[float(x) for x in h])
    return arr


def ap_md_kick_drift(mol, lengths, mass, dt, forces, xyz, vel, status=None, stream=None):
    """First half of a rigid-water velocity-Verlet step (positions and velocities in place)."""
    import torch
    n = xyz.shape[0]
    nm = mol.shape[0]
    _check(None, load().ap_md_kick_drift(int(nm), _ptr(mol, torch.int32, (nm, 3), "mol"), _lengths(lengths),
                                         _ptr(mass, torch.float64, (n,), "mass"), float(dt),
                                         _ptr(forces, torch.float64, (n, 3), "forces"),
                                         _ptr(xyz, torch.float64, (n, 3), "xyz"), _ptr(vel, torch.float64, (n, 3), "vel"),
                                         _ptr(status, torch.int32, (1,), "status", allow_none=True),
                                         _stream_ptr(xyz, stream)), "ap_md_kick_drift")


def ap_md_kick(mol, lengths, mass, dt, forces, xyz, vel, kinetic=None, status=None, stream=None, scale=1.0):
    """Second half of the step (velocities in place, then scaled by `scale`); kinetic:
    optional [1] float64 output."""
    import torch
    n = xyz.shape[0]
    nm = mol.shape[0]
    _check(None, load().ap_md_kick(int(nm), _ptr(mol, torch.int32, (nm, 3), "mol"), _lengths(lengths),
                                   _ptr(mass, torch.float64, (n,), "mass"), float(dt),
                                   _ptr(forces, torch.float64, (n, 3), "forces"),
                                   _ptr(xyz, torch.float64, (n, 3), "xyz"), _ptr(vel, torch.float64, (n, 3), "vel"),
                                   float(scale), _ptr(kinetic, torch.float64, (1,), "kinetic", allow_none=True),
                                   _ptr(status, torch.int32, (1,), "status", allow_none=True),
                                   _stream_ptr(xyz, stream)), "ap_md_kick")


def ap_lj_forces(ctx, lj, energy, forces):
    """Force-shifted Lennard-Jones of the current configuration: energy [1] written, forces
    [n][3] added to."""
    import torch
    n = forces.shape[0]
    _check(ctx, load().ap_lj_forces(ctx, _ptr(lj, torch.float64, (n, 2), "lj"), _ptr(energy, torch.float64, (1,), "energy"),
                                    _ptr(forces, torch.float64, (n, 3), "forces")), "ap_lj_forces")


def ap_direct_guess(ctx, mu0):
    """mu0 [n][3] (caller order) = alpha E of the current configuration."""
    import torch
    n = mu0.shape[0]
    _check(ctx, load().ap_direct_guess(ctx, _ptr(mu0, torch.float64, (n, 3), "mu0")), "ap_direct_guess")


def ap_learned_guess(ctx, packed, mu0):
    import torch
    n = mu0.shape[0]
    _check(ctx, load().ap_learned_guess(ctx, _ptr(packed, torch.uint8, (ap_mlp_packed_bytes(),), "packed"),
                                        _ptr(mu0, torch.float64, (n, 3), "mu0")), "ap_learned_guess")


def ap_fp32_peak(reps=10):
    """(TFLOP/s, SM count): the device's FP32 FMA rate measured by the library's microbenchmark."""
    tf, sms = ctypes.c_double(), ctypes.c_int()
    _check(None, load().ap_fp32_peak(int(reps), ctypes.byref(tf), ctypes.byref(sms)), "ap_fp32_peak")
    return tf.value, sms.value


def ap_eval_erfc(x, approx, lib, stream=None):
    """approx = erfc as the FP32 pair kernels form it, lib = CUDA's erfcf, at x (float32 CUDA)."""
    import torch
    n = x.shape[0]
    _check(None, load().ap_eval_erfc(_ptr(x, torch.float32, (n,), "x"), int(n), _ptr(approx, torch.float32, (n,), "approx"),
                                     _ptr(lib, torch.float32, (n,), "lib"), _stream_ptr(x, stream)), "ap_eval_erfc")


def ap_autotune(ctx, reps=5):
    ch = (ctypes.c_int * 2)()
    _check(ctx, load().ap_autotune(ctx, int(reps), ch), "ap_autotune")
    return int(ch[0]), int(ch[1])


class Batch:
    """One CUDA graph advancing several replica Contexts (each on its own stream)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.ctx.value for c in self.contexts])
        self.ptr = ctypes.c_void_p()
        _check(None, load().ap_batch_create(ctypes.byref(self.ptr), arr, len(self.contexts)), "ap_batch_create")
        self._keep = []

    def capture(self, tol=1e-5, max_iter=200, packed=None, forces=True, history=False, virial=False):
        steps = (ApBatchStep * len(self.contexts))()
        self._keep = []
        for k, c in enumerate(self.contexts):
            st = steps[k]
            st.d_xyz, st.d_mpole = c.xyz.data_ptr(), c.mpole.data_ptr()
            st.d_frame, st.d_alpha = c.frame.data_ptr(), c.alpha.data_ptr()
            if packed is not None:
                mu0 = c.torch.zeros((c.n, 3), dtype=c.torch.float64, device=c.device)
                self._keep.append(mu0)
                st.d_mlp_packed, st.d_mu0 = packed.data_ptr(), mu0.data_ptr()
                if history == "adaptive":
                    hist = c.torch.zeros(7 * c.n * 3 + AP_ADAPTIVE_SCRATCH, dtype=c.torch.float64, device=c.device)
                    self._keep.append(hist)
                    st.d_hist_lsq = hist.data_ptr()
                elif history:
                    hist = c.torch.zeros((5, c.n, 3), dtype=c.torch.float64, device=c.device)
                    self._keep.append(hist)
                    st.d_hist = hist.data_ptr()
            st.tol_debye, st.max_iter = float(tol), int(max_iter)
            st.d_mu = c.mu.data_ptr()
            if forces:
                st.d_energy, st.d_forces = c.energy.data_ptr(), c.forces.data_ptr()
                if virial:
                    st.d_virial = c.virial.data_ptr()
        _check(None, load().ap_batch_capture(self.ptr, steps), "ap_batch_capture")

    def launch(self, stream):
        _check(None, load().ap_batch_launch(self.ptr, ctypes.c_void_p(stream.cuda_stream)), "ap_batch_launch")

    def close(self):
        if self.ptr is not None:
            load().ap_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- marshalling helpers ---------------------------------------------------------------
def make_params(n, box, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), thole_a=0.39,
                precision=AP_MIXED) -> ApParams:
    p = ApParams()
    p.n_atoms = int(n)
    for d in range(3):
        p.box[d] = float(box[d])
        p.grid[d] = int(grid[d])
    p.cutoff, p.buffer, p.ewald_beta, p.thole_a = float(cutoff), float(buffer), float(beta), float(thole_a)
    p.pme_order = 5
    p.precision = int(precision)
    return p


class Context:
    """Owns an ap_ctx and the device copies of one system's inputs (torch tensors)."""

    def __init__(self, sysobj, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), thole_a=0.39,
                 precision=AP_MIXED, device="cuda", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise ApError("no CUDA device")
        self.torch = torch
        self.device = torch.device(device)
        self.n = sysobj.n
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = make_params(self.n, sysobj.box, cutoff, buffer, beta, grid, thole_a, precision)
        self.ctx = ap_create(self.params, self.stream.cuda_stream)
        self.upload(sysobj)

    def upload(self, sysobj):
        t = self.torch
        dev = self.device
        self.xyz = t.tensor(np.ascontiguousarray(sysobj.xyz, np.float64), device=dev)
        mp = np.concatenate([sysobj.q[:, None], sysobj.dip, sysobj.quad], axis=1)
        self.mpole = t.tensor(np.ascontiguousarray(mp, np.float64), device=dev)
        self.frame = t.tensor(np.ascontiguousarray(sysobj.frame, np.int32), device=dev)
        self.alpha = t.tensor(np.ascontiguousarray(sysobj.alpha, np.float64), device=dev)
        off, atoms = sysobj.excl_csr()
        self.excl_off = t.tensor(off, device=dev)
        self.excl_atoms = t.tensor(atoms if len(atoms) else np.zeros(1, np.int32), device=dev)
        self.n_excl = int(off[-1])
        self.field = t.zeros((self.n, 3), dtype=t.float64, device=dev)
        self.mu = t.zeros((self.n, 3), dtype=t.float64, device=dev)
        self.forces = t.zeros((self.n, 3), dtype=t.float64, device=dev)
        self.energy = t.zeros(1, dtype=t.float64, device=dev)
        self.virial = t.zeros((3, 3), dtype=t.float64, device=dev)

    def set_positions(self, xyz):
        self.xyz.copy_(self.torch.as_tensor(np.ascontiguousarray(xyz, np.float64)), non_blocking=False)

    def build(self):
        return build_neighbour_blocks(self.ctx, self.xyz, self.excl_off, self.excl_atoms, self.n_excl)

    def permanent_field(self, out=True):
        return permanent_field(self.ctx, self.xyz, self.mpole, self.frame, self.alpha, self.field if out else None)

    def solve(self, tol=1e-5, max_iter=200, guess=None, want_info=True):
        return induced_dipoles_pcg(self.ctx, guess, tol, max_iter, self.mu, want_info)

    def solve_diis(self, tol=1e-5, max_iter=200, depth=6, guess=None, want_info=True):
        return induced_dipoles_diis(self.ctx, guess, tol, max_iter, depth, self.mu, want_info)

    # AMOEBA's two dipole sets: the context's exclusion list must hold every listed pair
    def set_scaled_pairs(self, pairs, scales):
        t = self.torch
        self.dp_pairs = t.tensor(np.ascontiguousarray(pairs, np.int32).reshape(-1, 2), device=self.device)
        self.dp_scales = t.tensor(np.ascontiguousarray(scales, np.float64).reshape(-1, 2), device=self.device)
        z = lambda: t.zeros((self.n, 3), dtype=t.float64, device=self.device)
        self.field_d, self.field_p, self.mu_d, self.mu_p = z(), z(), z(), z()
        return set_scaled_pairs(self.ctx, self.dp_pairs, self.dp_scales)

    def permanent_field_dp(self, out=True):
        return permanent_field_dp(self.ctx, self.xyz, self.mpole, self.frame, self.alpha,
                                  self.field_d if out else None, self.field_p if out else None)

    def solve_dp(self, tol=1e-5, max_iter=200, guess_d=None, guess_p=None, want_info=True):
        return induced_dipoles_pcg_dp(self.ctx, guess_d, guess_p, tol, max_iter, self.mu_d, self.mu_p, want_info)

    def energy_forces_dp(self, mu_d=None, mu_p=None, virial=False):
        polarization_energy_forces_dp(self.ctx, self.mu_d if mu_d is None else mu_d,
                                      self.mu_p if mu_p is None else mu_p, self.energy, self.forces,
                                      self.virial if virial else None)
        return (self.energy, self.forces, self.virial) if virial else (self.energy, self.forces)

    def energy_forces(self, mu=None, virial=False):
        """(energy, forces) or, with virial=True, (energy, forces, virial [3, 3])."""
        polarization_energy_forces(self.ctx, self.mu if mu is None else mu, self.energy, self.forces,
                                   self.virial if virial else None)
        return (self.energy, self.forces, self.virial) if virial else (self.energy, self.forces)

    def matvec(self, v, out):
        return dipole_field_matvec(self.ctx, v, out)

    def stats(self):
        return ap_list_stats(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ap_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
