"""GPU parity of the polarization virial, the third output of polarization_energy_forces()
and polarization_energy_forces_dp(), against the oracle's virial (which is pinned on its own
by finite differences of the re-solved energy under box stretches, the isolated-cluster
identity, independence of the Ewald parameter and symmetry), all nine components, at the
forces' tolerances: FP64 to 1e-8, mixed precision and fixed point to 1e-4 of the largest
component.

The pair kernel forms the pairs' share in two ways, both covered here: per pair side in
small boxes, where every pair takes its own minimum image (the 648-atom and the chain box),
and once per work item from the per-target force sums in larger boxes, where every position
of an item sits in one frame (the 3,000-atom box). The reciprocal share (potential
derivatives times multipoles, and the structure-factor sum over the half spectrum with its
Nyquist planes) and the frame vectors' share enter every case; the chain adds global-frame
atoms and excluded pairs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu
PRECS = [(binding.AP_FP64, 1e-8), (binding.AP_MIXED, 1e-4), (binding.AP_FIXED, 1e-4)]


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


CASES = {
    "water648": (lambda: synth.water_box(216, 18.64, 1001), (24, 24, 24)),
    "water3000": (lambda: synth.water_box(1000, 31.1, 3001), (40, 40, 40)),
    "chain240": (lambda: synth.solvated_chain(60, 180, 26.0, 1103), (32, 32, 32)),
}
_oracle_cache = {}


def _reference(name):
    if name not in _oracle_cache:
        make, grid = CASES[name]
        s = make()
        o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=7.0))
        E = o.permanent_field()
        mu, _ = o.pcg(E, tol=1e-10)
        _oracle_cache[name] = (s, grid, mu, o.virial(mu), o.energy(mu, E))
    return _oracle_cache[name]


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec,tol", PRECS)
def test_virial_matches_oracle(name, prec, tol):
    s, grid, mu, V_o, e_o = _reference(name)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=prec)
    c.build()
    c.permanent_field()
    e, f, V = c.energy_forces(torch.tensor(mu, device="cuda"), virial=True)
    e, f, V = e.clone(), f.clone(), V.cpu().numpy()
    assert abs(float(e.cpu()[0]) - e_o) < max(tol, 1e-9) * abs(e_o)
    assert _rel(V, V_o) < tol, (V, V_o)
    # the call with the virial returns the same energy and forces as the call without it: bit
    # for bit in fixed point; to rounding in FP64 (FP64 atomics in varying order); to the
    # FP32 grid's rounding in the mixed mode (FP32 atomics of the spread in varying order)
    e2, f2 = c.energy_forces(torch.tensor(mu, device="cuda"))
    if prec == binding.AP_FIXED:
        assert torch.equal(f, f2) and torch.equal(e, e2)
    else:
        bound = 1e-12 if prec == binding.AP_FP64 else 1e-5
        assert (f - f2).abs().max().item() < bound * f2.abs().max().item()
    c.close()


def test_fixed_point_virial_is_bitwise_reproducible():
    s, grid, mu, _, _ = _reference("water3000")
    out = []
    for _ in range(2):
        c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=binding.AP_FIXED)
        c.build()
        c.permanent_field()
        _, _, V = c.energy_forces(torch.tensor(mu, device="cuda"), virial=True)
        out.append(V.cpu().numpy().tobytes())
        c.close()
    assert out[0] == out[1]


@pytest.mark.parametrize("prec,tol", PRECS)
def test_two_set_virial_matches_oracle(prec, tol):
    s, pairs, scales = synth.dp_system(synth.solvated_chain(60, 180, 26.0, 1103), 7)
    grid = (24, 24, 24)
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=7.0), dp=(pairs, scales))
    E_d, E_p = o.permanent_field_dp()
    mu_d, mu_p, _ = o.pcg_dp(E_d, E_p, tol=1e-10)
    V_o = o.virial_dp(mu_d, mu_p)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=prec)
    c.build()
    c.set_scaled_pairs(pairs, scales)
    c.permanent_field_dp()
    _, _, V = c.energy_forces_dp(torch.tensor(mu_d, device="cuda"), torch.tensor(mu_p, device="cuda"),
                                 virial=True)
    assert _rel(V.cpu().numpy(), V_o) < tol
    c.close()


def test_batch_step_virial():
    """The batch graph's optional virial output equals the direct call's."""
    s = synth.water_box(216, 18.64, 1001)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), precision=binding.AP_FP64,
                        stream=torch.cuda.Stream())
    c.build()
    with torch.cuda.stream(c.stream):
        c.permanent_field(out=False)
        c.solve(tol=1e-8, max_iter=100)
        _, _, V = c.energy_forces(virial=True)
        V_direct = V.clone()
    torch.cuda.synchronize()
    b = binding.Batch([c])
    b.capture(tol=1e-8, max_iter=100, virial=True)
    c.virial.zero_()
    b.launch(torch.cuda.Stream())
    torch.cuda.synchronize()
    assert _rel(c.virial.cpu().numpy(), V_direct.cpu().numpy()) < 1e-10
    b.close()
    c.close()
