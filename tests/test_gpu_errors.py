"""Failure paths and numerical building blocks on the GPU, through the C-ABI.

A NaN in one multipole value (never in the positions, which feed the cell indexing) makes
the solve's reductions non-finite: the direct call returns AP_ERR_NONFINITE, and so does
ap_solve_info_last() for a solve that ran inside a batch graph, while the other replicas of
the same graph are unaffected. The FP32 erfc of the pair kernels (Abramowitz & Stegun
7.1.26, absolute error <= 1.5e-7, evaluated in FP32) is compared with CUDA's erfcf over the
range the cutoff allows, beta r in [0, 0.5446 * 7]: within 1e-6 absolute."""
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


def _ctx(s, stream=None):
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), precision=binding.AP_MIXED,
                        stream=stream)
    c.build()
    return c


def test_nonfinite_multipole_direct_solve():
    s = synth.water_box(216, 18.64, 1001)
    c = _ctx(s)
    c.mpole[7, 0] = float("nan")                 # the charge of one atom
    c.permanent_field()
    with pytest.raises(binding.ApError) as e:
        c.solve(tol=1e-5, max_iter=50)
    assert e.value.code == binding.AP_ERR_NONFINITE
    with pytest.raises(binding.ApError) as e:
        binding.ap_solve_info_last(c.ctx)
    assert e.value.code == binding.AP_ERR_NONFINITE
    # a finite configuration afterwards solves normally on the same context
    c.upload(s)
    c.build()
    c.permanent_field()
    info = c.solve(tol=1e-5, max_iter=50)
    assert info.status == 0 and info.eps_debye <= 1e-5
    c.close()


def test_nonfinite_multipole_in_batch_graph():
    good = _ctx(synth.water_box(216, 18.64, 1001), stream=torch.cuda.Stream())
    bad = _ctx(synth.water_box(216, 18.64, 1002), stream=torch.cuda.Stream())
    bad.mpole[11, 2] = float("nan")              # one dipole component
    for c in (good, bad):
        with torch.cuda.stream(c.stream):
            c.permanent_field(out=False)
    torch.cuda.synchronize()
    b = binding.Batch([good, bad])
    b.capture(tol=1e-5, max_iter=50, forces=False)
    b.launch(torch.cuda.Stream())
    torch.cuda.synchronize()
    info = binding.ap_solve_info_last(good.ctx)
    assert info.status == 0 and info.eps_debye <= 1e-5
    with pytest.raises(binding.ApError) as e:
        binding.ap_solve_info_last(bad.ctx)
    assert e.value.code == binding.AP_ERR_NONFINITE
    b.close()
    good.close()
    bad.close()


def test_erfc_against_cuda_erfcf():
    x = torch.linspace(0.0, 0.5446 * 7.0, 40001, dtype=torch.float32, device="cuda")
    approx, lib = torch.empty_like(x), torch.empty_like(x)
    binding.ap_eval_erfc(x, approx, lib)
    torch.cuda.synchronize()
    a, l = approx.cpu().numpy().astype(np.float64), lib.cpu().numpy().astype(np.float64)
    err = np.abs(a - l)
    # A&S 7.1.26's 1.5e-7, the FP32 rounding of its polynomial and reciprocal, the fast
    # exponential's few ulp of e^{-x^2} and erfcf's own ulps (measured on GB300: 5.4e-7);
    # relative to the bare Coulomb term (erfc(x) / r against 1 / r) the bound is the same,
    # 10x below the 1e-5 tolerance of the field
    assert err.max() < 1e-6, err.max()
    print(f"max |erfc_pair - erfcf| = {err.max():.2e} over beta r in [0, {0.5446 * 7:.3f}]")
