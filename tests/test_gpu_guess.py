"""The trajectory-extrapolation guess entry point against its definition, and its use:
extrapolated guesses along a short trajectory reach the same solution in fewer PCG
iterations than alpha E."""
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


def test_extrapolate_guess_definition():
    rng = np.random.default_rng(2)
    n = 1001
    a = {k: rng.normal(size=(n, 3)) for k in ("b", "m1", "b1", "m2", "b2")}
    t = {k: torch.tensor(v, device="cuda") for k, v in a.items()}
    out = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    binding.ap_extrapolate_guess(out, t["m1"], t["m2"], base=t["b"], base1=t["b1"], base2=t["b2"])
    ref = a["b"] + 2 * (a["m1"] - a["b1"]) - (a["m2"] - a["b2"])
    assert np.array_equal(out.cpu().numpy(), ref)
    binding.ap_extrapolate_guess(out, t["m1"], t["m2"])
    assert np.array_equal(out.cpu().numpy(), 2 * a["m1"] - a["m2"])
    binding.ap_extrapolate_guess(t["b"], t["m1"], t["m2"], base=t["b"], base1=t["b1"], base2=t["b2"])   # aliased
    assert np.array_equal(t["b"].cpu().numpy(), ref)


def test_extrapolated_guess_saves_iterations():
    s = synth.water_box(216, 18.64, 1001)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(24, 24, 24), precision=binding.AP_MIXED)
    cur = s
    mus, plain, extrap = [], [], []
    for k in range(5):
        cur = synth.perturb(cur, 50 + k)
        c.set_positions(cur.xyz)
        if k == 0:
            c.build()
        c.permanent_field()
        plain.append(c.solve(tol=1e-6, max_iter=100).iterations)
        mu_plain = c.mu.clone()
        if len(mus) >= 2:
            g = torch.empty_like(c.mu)
            binding.ap_extrapolate_guess(g, mus[-1], mus[-2])
            info = c.solve(tol=1e-6, max_iter=100, guess=g)
            extrap.append(info.iterations)
            assert (c.mu - mu_plain).abs().max().item() < 1e-5   # same solution at the tolerance
        mus.append(mu_plain)
    assert np.mean(extrap) < np.mean(plain[2:])
    c.close()


def test_adaptive_guess_definition():
    """ap_adaptive_guess against its definition written out in NumPy, and its limits: steady
    motion gives c = 1 (linear extrapolation), a reversal clamps c to 0 (hold)."""
    rng = np.random.default_rng(3)
    n = 1003
    a = {k: rng.normal(size=(n, 3)) for k in ("b", "m1", "b1", "m2", "b2", "m3", "b3")}
    t = {k: torch.tensor(v, device="cuda") for k, v in a.items()}
    out = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    scratch = torch.zeros(binding.AP_ADAPTIVE_SCRATCH, dtype=torch.float64, device="cuda")
    binding.ap_adaptive_guess(out, t["m1"], t["m2"], t["m3"], scratch, base=t["b"], base1=t["b1"], base2=t["b2"],
                              base3=t["b3"])
    e1, e2, e3 = a["m1"] - a["b1"], a["m2"] - a["b2"], a["m3"] - a["b3"]
    c = float(np.clip(np.sum((e1 - e2) * (e2 - e3)) / np.sum((e2 - e3) ** 2), 0.0, 1.0))
    assert abs(scratch[0].item() - c) < 1e-13
    np.testing.assert_allclose(out.cpu().numpy(), a["b"] + e1 + c * (e1 - e2), rtol=0, atol=1e-12)
    # steady motion: mu_k = x + (4 - k) v -> c = 1, out = 2 mu1 - mu2
    x, v = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    m = [torch.tensor(x + (4 - k) * v, device="cuda") for k in (1, 2, 3)]
    binding.ap_adaptive_guess(out, m[0], m[1], m[2], scratch)
    assert abs(scratch[0].item() - 1.0) < 1e-12
    np.testing.assert_allclose(out.cpu().numpy(), x + 4 * v, rtol=0, atol=1e-12)
    # reversal: mu3 = mu1 -> (e1 - e2) = -(e2 - e3), c = -1 clamped to 0: hold mu1
    binding.ap_adaptive_guess(out, m[0], m[1], m[0], scratch)
    assert scratch[0].item() == 0.0
    assert np.array_equal(out.cpu().numpy(), m[0].cpu().numpy())
