"""GPU parity of AMOEBA's two induced-dipole sets (set_scaled_pairs, permanent_field_dp,
induced_dipoles_pcg_dp, polarization_energy_forces_dp) through the C-ABI against the
oracle's *_dp methods on the same seeded inputs: a solvated chain cut into polarization
groups, so that the d and p fields differ (1-2/1-3 pairs, 1-4 pairs inside a group with
p-scale 1/2, longer pairs inside a group with d-scale 0). FP64 mode agrees to rounding with
the oracle's iterates; the mixed and fixed-point modes within the tolerances of the
single-set path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu
DEBYE = 4.80321
GRID = (24, 24, 24)


def _rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


def _rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.fixture(scope="module")
def chain():
    s = synth.solvated_chain(60, 180, 26.0, 1103)
    return synth.dp_system(s, 7)


@pytest.fixture(scope="module")
def oracle_chain(chain):
    s, pairs, scales = chain
    o = Oracle(s, Params(beta=0.5446, grid=GRID, cutoff=7.0), dp=(pairs, scales))
    E_d, E_p = o.permanent_field_dp()
    return o, E_d, E_p


def _ctx(s, pairs, scales, prec):
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=GRID, precision=prec)
    c.build()
    c.set_scaled_pairs(pairs, scales)
    c.permanent_field_dp()
    return c


@pytest.mark.parametrize("prec,tol", [(binding.AP_FP64, 1e-9), (binding.AP_MIXED, 1e-5), (binding.AP_FIXED, 1e-5)])
def test_fields(chain, oracle_chain, prec, tol):
    s, pairs, scales = chain
    o, E_d, E_p = oracle_chain
    c = _ctx(s, pairs, scales, prec)
    assert _rel_rms(c.field_d.cpu().numpy(), E_d) < tol
    assert _rel_rms(c.field_p.cpu().numpy(), E_p) < tol
    assert _rel_max(E_d, E_p) > 1e-2    # the two sets really differ here
    c.close()


def test_fp64_matches_oracle_iterates(chain, oracle_chain):
    s, pairs, scales = chain
    o, E_d, E_p = oracle_chain
    c = _ctx(s, pairs, scales, binding.AP_FP64)
    info = c.solve_dp(tol=1e-6, max_iter=100)
    mu_d_o, mu_p_o, info_o = o.pcg_dp(E_d, E_p, tol=1e-6)
    assert info.status == 0 and info.iterations == info_o["iters"]
    assert abs(info.eps_debye - info_o["eps"]) < 1e-6 * info_o["eps"]
    assert _rel_max(c.mu_d.cpu().numpy(), mu_d_o) < 1e-8
    assert _rel_max(c.mu_p.cpu().numpy(), mu_p_o) < 1e-8
    assert binding.ap_solve_info_last(c.ctx).iterations == info.iterations
    c.close()


@pytest.mark.parametrize("prec,etol,ftol", [(binding.AP_FP64, 1e-9, 1e-8), (binding.AP_MIXED, 1e-5, 1e-4),
                                             (binding.AP_FIXED, 1e-5, 1e-4)])
def test_energy_forces_at_gpu_dipoles(chain, oracle_chain, prec, etol, ftol):
    s, pairs, scales = chain
    o, E_d, E_p = oracle_chain
    c = _ctx(s, pairs, scales, prec)
    c.solve_dp(tol=1e-6, max_iter=100)
    e, f = c.energy_forces_dp()
    mu_d, mu_p = c.mu_d.cpu().numpy(), c.mu_p.cpu().numpy()
    e_o = o.energy_dp(mu_d, E_p)
    assert abs(float(e.cpu()[0]) - e_o) < etol * abs(e_o)
    F_o = o.forces_dp(mu_d, mu_p)
    assert _rel_rms(f.cpu().numpy(), F_o) < ftol
    c.close()


@pytest.mark.parametrize("prec", [binding.AP_MIXED, binding.AP_FIXED])
def test_reduced_precision_reaches_tolerance(chain, oracle_chain, prec):
    s, pairs, scales = chain
    o, E_d, E_p = oracle_chain
    tol = 1e-5
    c = _ctx(s, pairs, scales, prec)
    info = c.solve_dp(tol=tol, max_iter=100)
    assert info.status == 0 and info.eps_debye <= tol
    for mu, E in ((c.mu_d, E_d), (c.mu_p, E_p)):
        assert o.residual_eps(E - o.apply_A(mu.cpu().numpy())) < 1.5 * tol
    c.close()


def test_fixed_point_is_bitwise_reproducible(chain):
    s, pairs, scales = chain
    out = []
    for _ in range(2):
        c = _ctx(s, pairs, scales, binding.AP_FIXED)
        c.solve_dp(tol=1e-6, max_iter=100)
        e, f = c.energy_forces_dp()
        out.append(b"".join(t.cpu().numpy().tobytes() for t in (c.field_d, c.field_p, c.mu_d, c.mu_p, e, f)))
        c.close()
    assert out[0] == out[1]


def test_equal_tables_reproduce_the_single_set():
    """Water with d and p scales both 0 inside each molecule: both sets equal the single
    set's field and dipoles, and the forces equal the single-set forces."""
    s = synth.water_box(216, 18.64, 1001)
    pairs, scales = s.excl, np.zeros((len(s.excl), 2))
    c = _ctx(s, pairs, scales, binding.AP_FP64)
    c.permanent_field()
    E = c.field.cpu().numpy()
    assert _rel_max(c.field_d.cpu().numpy(), E) < 1e-14
    assert _rel_max(c.field_p.cpu().numpy(), E) < 1e-14
    c.permanent_field_dp()
    info = c.solve_dp(tol=1e-7, max_iter=100)
    info1 = c.solve(tol=1e-7, max_iter=100)
    assert info.iterations == info1.iterations
    mu = c.mu.cpu().numpy()
    assert _rel_max(c.mu_d.cpu().numpy(), mu) < 1e-12
    assert _rel_max(c.mu_p.cpu().numpy(), mu) < 1e-12
    e1, f1 = c.energy_forces(c.mu)
    e1, f1 = float(e1.cpu()[0]), f1.cpu().numpy().copy()
    e2, f2 = c.energy_forces_dp()
    assert abs(float(e2.cpu()[0]) - e1) < 1e-11 * abs(e1)
    assert _rel_max(f2.cpu().numpy(), f1) < 1e-10
    c.close()


def test_state_and_argument_errors(chain):
    s, pairs, scales = chain
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=GRID, precision=binding.AP_MIXED)
    c.build()
    with pytest.raises(binding.ApError):
        binding.permanent_field_dp(c.ctx, c.xyz, c.mpole, c.frame, c.alpha)
    bad = np.array(pairs, copy=True)
    bad[3, 1] = s.n
    with pytest.raises(binding.ApError):
        c.set_scaled_pairs(bad, scales)
    bad[3, 1] = bad[3, 0]
    with pytest.raises(binding.ApError):
        c.set_scaled_pairs(bad, scales)
    c.set_scaled_pairs(pairs, scales)
    with pytest.raises(binding.ApError):
        c.solve_dp(tol=1e-5, max_iter=10)    # before permanent_field_dp
    c.permanent_field_dp()
    info = c.solve_dp(tol=1e-12, max_iter=3)
    assert info.status == binding.AP_NOT_CONVERGED and info.iterations == 3
    c.close()


def test_no_listed_pairs_gives_two_copies_of_the_single_set(chain):
    """With an empty table both fields are the single-set field of the context's exclusion
    list, so the lockstep solve returns that solve twice."""
    s, pairs, scales = chain
    c = _ctx(s, np.zeros((0, 2), np.int32), np.zeros((0, 2)), binding.AP_FP64)
    c.permanent_field()
    E = c.field.cpu().numpy()
    assert _rel_max(c.field_d.cpu().numpy(), E) < 1e-14 and _rel_max(c.field_p.cpu().numpy(), E) < 1e-14
    c.permanent_field_dp()
    info = c.solve_dp(tol=1e-7, max_iter=100)
    info1 = c.solve(tol=1e-7, max_iter=100)
    assert info.iterations == info1.iterations
    mu = c.mu.cpu().numpy()
    assert _rel_max(c.mu_d.cpu().numpy(), mu) < 1e-12 and _rel_max(c.mu_p.cpu().numpy(), mu) < 1e-12
    c.close()


@pytest.mark.parametrize("n_chain,n_water,box,grid", [(7, 4, 12.0, (12, 12, 12)), (13, 8, 14.0, (16, 14, 12))])
def test_small_and_ragged_chains(n_chain, n_water, box, grid):
    """A few dozen atoms (one or two blocks with a ragged tail), non-cubic grid: FP64 fields,
    iterations, dipoles, energy and forces against the oracle."""
    s0 = synth.solvated_chain(n_chain, n_water, box, 300 + n_chain)
    s, pairs, scales = synth.dp_system(s0, 11, 3, 5)
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=5.0), dp=(pairs, scales))
    E_d, E_p = o.permanent_field_dp()
    c = binding.Context(s, cutoff=5.0, buffer=1.0, beta=0.5446, grid=grid, precision=binding.AP_FP64)
    c.build()
    c.set_scaled_pairs(pairs, scales)
    c.permanent_field_dp()
    assert _rel_rms(c.field_d.cpu().numpy(), E_d) < 1e-9 and _rel_rms(c.field_p.cpu().numpy(), E_p) < 1e-9
    info = c.solve_dp(tol=1e-8, max_iter=200)
    mu_d, mu_p, info_o = o.pcg_dp(E_d, E_p, tol=1e-8)
    assert info.iterations == info_o["iters"]
    assert _rel_max(c.mu_d.cpu().numpy(), mu_d) < 1e-7 and _rel_max(c.mu_p.cpu().numpy(), mu_p) < 1e-7
    e, f = c.energy_forces_dp()
    gd, gp = c.mu_d.cpu().numpy(), c.mu_p.cpu().numpy()
    assert abs(float(e.cpu()[0]) - o.energy_dp(gd, E_p)) < 1e-9 * abs(o.energy_dp(gd, E_p))
    assert _rel_rms(f.cpu().numpy(), o.forces_dp(gd, gp)) < 1e-8
    c.close()
