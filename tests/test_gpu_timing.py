"""The benchmark-support call ap_time_kernel on the GPU, through the C-ABI.

Every kernel id, the composite ones included (the FFT round trip, the reciprocal branch and a
whole operator application, each captured into a CUDA graph and the graph timed), returns a
positive mean duration, and the call leaves the context's stored field, lists and solver state
usable: a solve and an energy/force call after the timings give the same iterations, dipoles,
energy and forces as before them (to FP32 rounding in the mixed mode, whose grid and
accumulator additions run in varying order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("prec", [binding.AP_MIXED, binding.AP_FP64])
def test_time_kernel_ids_leave_state_usable(prec):
    s = synth.water_box(216, 18.64, 1001)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), precision=prec)
    c.build()
    c.permanent_field()
    info0 = c.solve(tol=1e-6, max_iter=100)
    mu0 = c.mu.clone()
    e0, f0 = (t.clone() for t in c.energy_forces())
    for name in ("real_matvec", "real_field", "spread_dipoles", "convolve", "gather_field", "spread_multipoles",
                 "pair_forces", "pcg_vectors", "fft_roundtrip", "pme_dipoles", "dipole_operator"):
        ms = binding.ap_time_kernel(c.ctx, name, 3)
        assert np.isfinite(ms) and ms > 0.0, name
    info1 = c.solve(tol=1e-6, max_iter=100)
    e1, f1 = c.energy_forces()
    assert info1.iterations == info0.iterations
    tol = 1e-12 if prec == binding.AP_FP64 else 1e-5
    assert (c.mu - mu0).abs().max().item() <= tol * mu0.abs().max().item()
    assert abs(e1.item() - e0.item()) <= tol * abs(e0.item())
    assert (f1 - f0).abs().max().item() <= tol * f0.abs().max().item()
    c.close()
