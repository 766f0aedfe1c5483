"""What the trained network gains: PCG iterations to the same tolerance from the learned
guess vs the direct-field guess alpha E on a held-out box (a water box of another seed than
every training box); the converged dipoles are the same either way. Checkpoint round trip.
The learned guess end to end from the oracle's own field: the oracle's field, features and
FP64 network (with the trained BF16 weights) against the library's guess."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from oracle import mlp as omlp
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


def _collect(ctx, positions):
    """Training pairs at each configuration, with the lists rebuilt there (the samples are
    far apart, beyond half the list buffer)."""
    feats, tgts = [], []
    for xyz in positions:
        ctx.set_positions(xyz)
        ctx.build()
        f, t = learned.collect(ctx, [xyz])
        feats.append(f)
        tgts.append(t)
    return torch.cat(feats), torch.cat(tgts)


def _train_on_other_boxes(ctx, seeds, per_box=6):
    """Training pairs from water boxes of the given seeds (same size as ctx's system),
    `per_box` perturbed configurations of each, solved tightly."""
    feats, tgts = [], []
    for sd in seeds:
        f, t = _collect(ctx, _traj(synth.water_box(1000, 31.1, sd), per_box, 100 + sd))
        feats.append(f)
        tgts.append(t)
    return torch.cat(feats), torch.cat(tgts)


def test_learned_guess_saves_iterations(tmp_path):
    s = synth.water_box(1000, 31.1, 3001)           # held out: never seen in training
    ctx = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(40, 40, 40), precision=binding.AP_MIXED)
    feat, tgt = _train_on_other_boxes(ctx, (3002, 3003, 3004, 3005))
    ctx.set_positions(s.xyz)
    ctx.build()
    test_pos = _traj(s.copy(), 40, 900)[-6:]
    tr = learned.Trainer(seed=7)
    losses = tr.fit(feat, tgt, steps=1500, batch=4096, lr=3e-3, lr_final=3e-4)
    assert losses[-50:].mean() < 0.5 * losses[:10].mean()
    plain, learn = [], []
    mu0 = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    for xyz in test_pos:
        ctx.set_positions(xyz)
        ctx.build()
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


def test_learned_guess_from_oracle_field():
    """The whole guess from the oracle's side: its permanent field E, short-range induced
    field E1 and features, and its FP64 network with the library's trained weights (rounded
    to BF16 as the tensor cores take them), give mu0 = alpha E + 0.02 R y; the library's
    guess from its own mixed-precision field must agree."""
    s = synth.water_box(216, 18.64, 1001)
    grid = (24, 24, 24)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=binding.AP_MIXED)
    feat, tgt = _collect(c, _traj(s, 4, 300))
    tr = learned.Trainer(seed=7)
    tr.fit(feat, tgt, steps=200, batch=512, lr=3e-3)
    c.set_positions(s.xyz)
    c.build()
    c.permanent_field(out=False)
    mu0 = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    binding.ap_learned_guess(c.ctx, tr.packed, mu0)
    torch.cuda.synchronize()
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=7.0))
    E = o.permanent_field()
    E1 = omlp.short_field(s.n, o.I, o.J, o.R, s.alpha, E, 0.5446, 0.39)
    W1, b1, W2, b2, W3, b3 = omlp.unflatten(tr.params.cpu().numpy().astype(np.float64))
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    params = [omlp.bf16_round(W1), f32(b1), omlp.bf16_round(W2), f32(b2), omlp.bf16_round(W3), f32(b3)]
    want = omlp.guess(params, s.xyz, s.box, s.frame, s.alpha, E, E1,
                      lambda a: omlp.bf16_round(np.asarray(a, np.float32)), omlp.bf16_round)
    got = mu0.cpu().numpy()
    corr = want - s.alpha[:, None] * E                 # the network's share of the guess
    assert np.sqrt(np.mean(corr ** 2)) > 1e-4          # the trained network is not idle
    # BF16 inputs: a field difference of ~1e-6 can flip a rounding; the network's share
    # agrees to a few BF16 ulps, the whole guess to 1e-3 relative
    assert np.sqrt(np.mean((got - want) ** 2)) < 1e-3 * np.sqrt(np.mean(want ** 2))
    assert np.sqrt(np.mean((got - want) ** 2)) < 5e-2 * np.sqrt(np.mean(corr ** 2))
    c.close()
