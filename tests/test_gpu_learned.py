"""What the trained network gains: PCG iterations to the same tolerance from the learned
guess vs the direct-field guess alpha E, on configurations not used for training; the
converged dipoles are the same either way. Checkpoint round trip."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2011_01207_gb300 import binding, learned, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _traj(s, n, seed):
    out, cur = [], s
    for k in range(n):
        cur = synth.perturb(cur, seed + k, sigma_t=0.08, sigma_r=0.15)   # well-separated samples
        out.append(cur.xyz.copy())
    return out


def test_learned_guess_saves_iterations(tmp_path):
    s = synth.water_box(1000, 31.1, 3001)
    ctx = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(40, 40, 40), precision=binding.AP_MIXED)
    ctx.build()
    train_pos = _traj(s, 24, 100)
    test_pos = _traj(s.copy(), 40, 900)[-6:]
    feat, tgt = learned.collect(ctx, train_pos)
    tr = learned.Trainer(seed=7)
    losses = tr.fit(feat, tgt, steps=1500, batch=4096, lr=3e-3, lr_final=3e-4)
    assert losses[-50:].mean() < 0.5 * losses[:10].mean()
    plain, learn = [], []
    mu0 = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    for xyz in test_pos:
        ctx.set_positions(xyz)
        ctx.permanent_field(out=False)
        info = ctx.solve(tol=1e-5, max_iter=100)
        plain.append(info.iterations)
        mu_plain = ctx.mu.clone()
        binding.ap_learned_guess(ctx.ctx, tr.packed, mu0)
        info = ctx.solve(tol=1e-5, max_iter=100, guess=mu0)
        learn.append(info.iterations)
        assert info.status == 0
        d = (ctx.mu - mu_plain).abs().max().item()
        assert d < 5e-5                      # same solution to the tolerance
    assert np.mean(learn) < np.mean(plain), (plain, learn)
    # checkpoint round trip reproduces the guess bit for bit
    path = str(tmp_path / "mlp.bin")
    tr.save(path)
    tr2 = learned.Trainer.load(path)
    mu1 = torch.zeros_like(mu0)
    binding.ap_learned_guess(ctx.ctx, tr.packed, mu0)
    binding.ap_learned_guess(ctx.ctx, tr2.packed, mu1)
    torch.cuda.synchronize()
    assert torch.equal(mu0, mu1) and tr2.step == tr.step
    print("iterations plain", plain, "learned", learn)
    ctx.close()
