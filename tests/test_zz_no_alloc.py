"""The allocation-free energy entry point, for callers that cannot allocate device memory
(all their memory belongs to another framework's pool, or allocation is forbidden after
set-up, or they hold no library context). Its scratch is a fixed array inside the
library; two calls in a row on different systems must each match the energy that the
context-based entry point polarization_energy_forces() returns, so nothing of the first
call leaks into the second. Collected last on purpose."""
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


def _reference(s, grid):
    c = binding.Context(s, cutoff=5.5, buffer=1.0, beta=0.5446, grid=grid, precision=binding.AP_FP64)
    c.build()
    c.permanent_field()
    c.solve(tol=1e-7, max_iter=200)
    e, _ = c.energy_forces()
    torch.cuda.synchronize()
    out = (c.mu.clone(), c.field.clone(), float(e.cpu()[0]))
    c.close()
    return out


def test_noalloc_energy_matches_entry_point_twice():
    systems = [(synth.water_box(216, 18.64, 1001), (24, 24, 24)),
               (synth.water_box(80, 14.0, 31), (16, 16, 16))]
    refs = [_reference(s, g) for s, g in systems]
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for mu, field, e_ref in refs:                 # two calls in a row, different sizes
        assert binding.polarization_energy_noalloc(mu, field, out) == 0
        torch.cuda.synchronize()
        e = float(out.cpu()[0])
        assert abs(e - e_ref) <= 1e-12 * abs(e_ref), (e, e_ref)


def test_noalloc_rejects_oversize_without_launching():
    lib = binding.load()
    code = lib.polarization_energy_noalloc(None, None, 1, None, None)
    assert code == -1
    mu = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    import ctypes
    code = lib.polarization_energy_noalloc(ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(mu.data_ptr()),
                                           (1 << 24) + 1, ctypes.c_void_p(out.data_ptr()), None)
    assert code == -1
    assert b"16777216" in lib.ap_last_error(None)
