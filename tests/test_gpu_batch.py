"""Batched replicas in one CUDA graph: every replica's step (field, solve with its WHILE
loop, energy, forces and virial) as a parallel branch. Each replica's results are checked
against the FP64 oracle (a water box, a solvated chain with global frames and exclusions,
and a larger water box); they also equal the standalone calls, and a relaunch picks up new
positions written into the captured buffers.

Mixed precision accumulates the PME grid with FP32 atomics, whose order varies from run
to run, so "equal" means: same iteration count, dipoles within a tenth of the solve
tolerance (in Debye), energy to 1e-7 and forces to 1e-5 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _replicas():
    systems = [(synth.water_box(216, 18.64, 1001), (24, 24, 24)),
               (synth.solvated_chain(60, 180, 26.0, 1103), (32, 32, 32)),
               (synth.water_box(1000, 31.1, 3001), (40, 40, 40))]
    out = []
    for s, g in systems:
        c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=g, precision=binding.AP_MIXED,
                            stream=torch.cuda.Stream())
        c.build()
        out.append((s, c))
    return out


def _standalone(c):
    with torch.cuda.stream(c.stream):
        c.permanent_field(out=False)
        info = c.solve(tol=1e-5, max_iter=200)
        e, f = c.energy_forces()
    torch.cuda.synchronize()
    return info.iterations, c.mu.clone(), e.clone(), f.clone()


def test_batch_graph_matches_standalone_and_relaunches():
    reps = _replicas()
    for s, c in reps:
        with torch.cuda.stream(c.stream):
            c.permanent_field(out=False)
            binding.ap_autotune(c.ctx, 3)
    ref = [_standalone(c) for _, c in reps]
    for _, c in reps:
        c.mu.zero_()
        c.forces.zero_()
    b = binding.Batch([c for _, c in reps])
    b.capture(tol=1e-5, max_iter=200)
    main = torch.cuda.Stream()
    b.launch(main)
    torch.cuda.synchronize()
    for (s, c), (it, mu, e, f) in zip(reps, ref):
        assert binding.ap_solve_info_last(c.ctx).iterations == it
        assert 4.80321 * (c.mu - mu).abs().max().item() < 0.1 * 1e-5
        assert abs(c.energy.item() - e.item()) < 1e-7 * abs(e.item())
        assert (c.forces - f).abs().max().item() < 1e-5 * f.abs().max().item()
    # new positions into the captured buffers, relaunch, compare with standalone again
    for k, (s, c) in enumerate(reps):
        c.set_positions(synth.perturb(s, 50 + k).xyz)
    torch.cuda.synchronize()
    b.launch(main)
    torch.cuda.synchronize()
    got = [(c.mu.clone(), c.energy.clone()) for _, c in reps]
    ref2 = [_standalone(c) for _, c in reps]
    for (mu_b, e_b), (it, mu, e, f) in zip(got, ref2):
        assert 4.80321 * (mu_b - mu).abs().max().item() < 0.1 * 1e-5
        assert abs(e_b.item() - e.item()) < 1e-7 * abs(e.item())
    b.close()
    for _, c in reps:
        c.close()


def test_batch_history_guess():
    """With d_hist, each launch starts from the learned guess plus the linear extrapolation
    of its error over the two previous launches (the learned guess alone before that), and
    still converges to the standalone solution."""
    from paper_2011_01207_gb300 import learned
    reps = _replicas()
    tr = learned.Trainer(seed=3)            # untrained weights: any guess is a valid start
    for s, c in reps:
        with torch.cuda.stream(c.stream):
            c.permanent_field(out=False)
    torch.cuda.synchronize()
    b = binding.Batch([c for _, c in reps])
    b.capture(tol=1e-6, max_iter=200, packed=tr.packed, history=True)
    g_buf = [t for t in b._keep if t.dim() == 2]     # learned guesses, one per replica
    h_buf = [t for t in b._keep if t.dim() == 3]     # [5][n][3] histories
    main = torch.cuda.Stream()
    cur = [s for s, _ in reps]
    past = [[] for _ in reps]                       # (mu, g) per earlier launch
    for step in range(4):
        for k, (s, c) in enumerate(reps):
            cur[k] = synth.perturb(cur[k], 70 + 10 * step + k)
            c.set_positions(cur[k].xyz)
        torch.cuda.synchronize()
        b.launch(main)
        torch.cuda.synchronize()
        for k, (s, c) in enumerate(reps):
            g, used, mu = g_buf[k].clone(), h_buf[k][4].clone(), c.mu.clone()
            if step < 2:
                assert torch.equal(used, g)
            else:
                (m1, g1), (m2, g2) = past[k][-1], past[k][-2]
                want = g + 2.0 * (m1 - g1) - (m2 - g2)
                assert (used - want).abs().max().item() < 1e-12
            past[k].append((mu, g))
            ref = _standalone(c)                    # same configuration, guess alpha E
            assert 4.80321 * (mu - ref[1]).abs().max().item() < 1e-4
    b.close()
    for _, c in reps:
        c.close()


def test_batch_adaptive_history_guess():
    """With d_hist_lsq, launch 0 starts from the learned guess, launches 1-2 hold its
    previous error, later launches extrapolate it with the least-squares coefficient of the
    three previous launches (ap_adaptive_guess's definition); every launch still converges
    to the standalone solution."""
    from paper_2011_01207_gb300 import learned
    reps = _replicas()
    tr = learned.Trainer(seed=3)
    for s, c in reps:
        with torch.cuda.stream(c.stream):
            c.permanent_field(out=False)
    torch.cuda.synchronize()
    b = binding.Batch([c for _, c in reps])
    b.capture(tol=1e-6, max_iter=200, packed=tr.packed, history="adaptive")
    g_buf = [t for t in b._keep if t.dim() == 2]     # learned guesses, one per replica
    h_buf = [t for t in b._keep if t.dim() == 1]     # flat histories
    main = torch.cuda.Stream()
    cur = [s for s, _ in reps]
    past = [[] for _ in reps]
    for step in range(5):
        for k, (s, c) in enumerate(reps):
            cur[k] = synth.perturb(cur[k], 90 + 10 * step + k)
            c.set_positions(cur[k].xyz)
        torch.cuda.synchronize()
        b.launch(main)
        torch.cuda.synchronize()
        for k, (s, c) in enumerate(reps):
            n3 = 3 * c.n
            g, used, mu = g_buf[k].clone(), h_buf[k][6 * n3:7 * n3].view(c.n, 3).clone(), c.mu.clone()
            if step == 0:
                assert torch.equal(used, g)
            elif step < 3:
                m1, g1 = past[k][-1]
                assert (used - (g + (m1 - g1))).abs().max().item() < 1e-12
            else:
                (m1, g1), (m2, g2), (m3, g3) = past[k][-1], past[k][-2], past[k][-3]
                e1, e2, e3 = m1 - g1, m2 - g2, m3 - g3
                cc = float(((e1 - e2) * (e2 - e3)).sum() / ((e2 - e3) ** 2).sum())
                cc = min(1.0, max(0.0, cc))
                want = g + e1 + cc * (e1 - e2)
                assert (used - want).abs().max().item() < 1e-9
            past[k].append((mu, g))
            ref = _standalone(c)
            assert 4.80321 * (mu - ref[1]).abs().max().item() < 1e-4
    b.close()
    for _, c in reps:
        c.close()


def test_batch_graph_against_oracle():
    """One graph launch over the three replicas in the mixed precision: each replica's
    dipoles reach the tolerance in the oracle's true residual, and its energy, forces and
    virial at those dipoles match the oracle's at the stated tolerances (1e-5, 1e-4, 1e-4)."""
    systems = [(synth.water_box(216, 18.64, 1001), (24, 24, 24)),
               (synth.solvated_chain(60, 180, 26.0, 1103), (32, 32, 32)),
               (synth.water_box(1000, 31.1, 3001), (40, 40, 40))]
    reps = []
    for s, g in systems:
        c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=g, precision=binding.AP_MIXED,
                            stream=torch.cuda.Stream())
        c.build()
        with torch.cuda.stream(c.stream):
            c.permanent_field(out=False)
        reps.append((s, g, c))
    torch.cuda.synchronize()
    tol = 1e-5
    b = binding.Batch([c for _, _, c in reps])
    b.capture(tol=tol, max_iter=200, virial=True)
    b.launch(torch.cuda.Stream())
    torch.cuda.synchronize()
    for s, g, c in reps:
        info = binding.ap_solve_info_last(c.ctx)
        assert info.status == 0 and info.eps_debye <= tol
        o = Oracle(s, Params(beta=0.5446, grid=g, cutoff=7.0))
        E = o.permanent_field()
        mu = c.mu.cpu().numpy()
        assert o.residual_eps(E - o.apply_A(mu)) < 1.5 * tol
        e_o = o.energy(mu, E)
        assert abs(c.energy.item() - e_o) < 1e-5 * abs(e_o)
        F_o = o.forces(mu)
        F = c.forces.cpu().numpy()
        assert np.sqrt(np.mean((F - F_o) ** 2) / np.mean(F_o ** 2)) < 1e-4
        V_o = o.virial(mu)
        assert np.abs(c.virial.cpu().numpy() - V_o).max() < 1e-4 * np.abs(V_o).max()
    b.close()
    for _, _, c in reps:
        c.close()
