"""The minimal rigid-water integrator (row f3) on the GPU through the C-ABI, against the
oracle's integrator (oracle/md.py, pinned by energy conservation, time reversibility and its
constraint identities): the same initial state gives the same trajectory step by step (FP64
to 1e-8 A, mixed precision to 1e-5 A over ten 1 fs steps), the force-shifted Lennard-Jones term
matches the oracle's (both pair paths: per-pair minimum image in small boxes, per-tile
shifts in larger ones), the library's trajectory conserves the total energy in the mixed
precision, and the Berendsen scale multiplies the kinetic energy by its square."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params, md
from paper_2011_01207_gb300 import binding, dynamics, synth

pytestmark = pytest.mark.gpu
BETA, GRID, RC = 0.6, (16, 16, 16), 6.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _small():
    return synth.water_box(64, 13.0, 43)


def _oracle_force(s, params, rc):
    eps = np.zeros(s.n)
    sig = np.ones(s.n)
    eps[0::3], sig[0::3] = dynamics.LJ_O

    class _At:
        def __init__(self, x):
            for k in ("q", "alpha", "dip", "quad", "frame", "excl", "n", "box"):
                setattr(self, k, getattr(s, k))
            self.xyz = x

    def force(x):
        o = Oracle(_At(x), params)
        E = o.permanent_field()
        mu, _ = o.pcg(E, tol=1e-11, maxiter=500)
        U_lj, F_lj = md.lj_energy_forces(x, s.box, eps, sig, rc)
        return o.energy(mu, E) + U_lj, o.forces(mu) + F_lj
    return force


def _gpu_run(s, prec, steps, dt, tol, v0):
    c = binding.Context(s, cutoff=RC, buffer=0.5, beta=BETA, grid=GRID, precision=prec)
    dyn = dynamics.RigidWaterMD(c, s, dt=dt, rebuild_every=1, tol=tol)
    dyn.start(v0)
    xs, vs, es = [c.xyz.cpu().numpy()], [dyn.vel.cpu().numpy()], [dyn.total_energy()]
    for _ in range(steps):
        dyn.step()
        xs.append(c.xyz.cpu().numpy())
        vs.append(dyn.vel.cpu().numpy())
        es.append(dyn.total_energy())
    dyn.check()
    c.close()
    return np.array(xs), np.array(vs), np.array(es)


@pytest.mark.parametrize("prec,xtol", [(binding.AP_FP64, 1e-8), (binding.AP_MIXED, 1e-5)])
def test_trajectory_matches_oracle(prec, xtol):
    s = _small()
    v0 = synth.water_velocities(s, 300.0, 7)
    m = md.water_masses(s.n)
    mol, lengths = md.water_constraints(s)
    force = _oracle_force(s, Params(beta=BETA, grid=GRID, cutoff=RC), RC)
    xo, vo, eo = md.run(s.xyz.copy(), md.rattle(v0, s.xyz, mol, lengths, 1.0 / m), m, 1.0, 10, force, mol, lengths)
    xg, vg, eg = _gpu_run(s, prec, 10, 1.0, 1e-10, v0)
    assert np.abs(xg - xo).max() < xtol
    assert np.abs(vg - vo).max() < xtol * np.abs(vo).max() * 10
    assert np.abs(eg - eo).max() < max(1e-8, xtol) * np.abs(eo).max() * 10
    for a, b, k in md.PAIRS:
        r = xg[-1][mol[:, a]] - xg[-1][mol[:, b]]
        assert np.abs(np.linalg.norm(r, axis=1) - lengths[k]).max() < 1e-9


@pytest.mark.parametrize("prec,tol,etol", [(binding.AP_FP64, 1e-10, 1e-10), (binding.AP_MIXED, 1e-5, 5e-5)])
@pytest.mark.parametrize("n_mol,box,grid", [(216, 18.64, (24, 24, 24)), (1000, 31.1, (40, 40, 40))])
def test_lj_matches_oracle(n_mol, box, grid, prec, tol, etol):
    """Forces to tol (RMS-relative); the energy to etol: in the mixed mode the pair vectors
    are FP32 (~1e-6 A) and close contacts carry tens of kcal/mol/A, while the total cancels
    to ~10 kcal/mol (repulsion, dispersion and the shift terms), so ~1e-4 kcal/mol remains."""
    s = synth.water_box(n_mol, box, 1001)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=prec)
    c.build()
    c.permanent_field()
    dyn = dynamics.RigidWaterMD(c, s)
    F = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    binding.ap_lj_forces(c.ctx, dyn.lj, e, F)
    eps = np.zeros(s.n)
    sig = np.ones(s.n)
    eps[0::3], sig[0::3] = dynamics.LJ_O
    U_o, F_o = md.lj_energy_forces(s.xyz, s.box, eps, sig, 7.0, excl=s.excl)
    Fg = F.cpu().numpy()
    assert np.sqrt(np.mean((Fg - F_o) ** 2) / np.mean(F_o ** 2)) < tol
    assert abs(float(e.item()) - U_o) < etol * abs(U_o)
    c.close()


def test_energy_conserved_mixed_precision():
    s = synth.water_box(216, 18.64, 1001)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), precision=binding.AP_MIXED)
    dyn = dynamics.RigidWaterMD(c, s, dt=1.0, rebuild_every=10, tol=1e-7)
    dyn.start(synth.water_velocities(s, 300.0, 9))
    e0, k0 = dyn.total_energy(), float(dyn.kinetic.item())
    es = [e0]
    for _ in range(100):
        dyn.step()
        es.append(dyn.total_energy())
    dyn.check()
    assert np.abs(np.array(es) - e0).max() < 1e-2 * k0
    c.close()


def test_berendsen_scale():
    s = _small()
    c = binding.Context(s, cutoff=RC, buffer=0.5, beta=BETA, grid=GRID, precision=binding.AP_FP64)
    dyn = dynamics.RigidWaterMD(c, s, dt=1.0)
    dyn.start(synth.water_velocities(s, 300.0, 7))
    k0 = float(dyn.kinetic.item())
    binding.ap_md_kick(dyn.mol, dyn.lengths, dyn.mass, 1.0, dyn.zero, c.xyz, dyn.vel, dyn.kinetic, dyn.status,
                       scale=0.9)
    assert abs(float(dyn.kinetic.item()) - 0.81 * k0) < 1e-12 * k0
    with pytest.raises(binding.ApError):
        binding.ap_md_kick(dyn.mol, dyn.lengths, dyn.mass, 1.0, dyn.zero, c.xyz, dyn.vel, scale=0.0)
    c.close()
