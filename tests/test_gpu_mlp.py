"""Learned-guess kernels (tcgen05 BF16 MLP) against the FP64 oracle MLP.

The oracle side applies the same BF16 roundings (weights, inputs, hidden activations) so
that only the accumulation order differs (FP32 on the tensor cores vs FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from oracle import mlp as omlp
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _packed(params):
    flat = torch.tensor(omlp.flatten(params), dtype=torch.float32, device="cuda")
    packed = torch.zeros(binding.ap_mlp_packed_bytes(), dtype=torch.uint8, device="cuda")
    binding.ap_mlp_pack(flat, packed)
    return packed


def _bf16_params(params):
    W1, b1, W2, b2, W3, b3 = params
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return [omlp.bf16_round(W1), f32(b1), omlp.bf16_round(W2), f32(b2), omlp.bf16_round(W3), f32(b3)]


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 4099])
def test_forward_matches_oracle(n):
    params = omlp.init_params(11)
    params[1] = np.random.default_rng(3).normal(size=128) * 0.1
    params[5] = np.array([0.1, -0.2, 0.3])
    X = np.random.default_rng(n).normal(size=(n, 16))
    y = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    binding.ap_mlp_forward(_packed(params), torch.tensor(X, dtype=torch.float32, device="cuda"), y)
    torch.cuda.synchronize()
    assert binding.ap_mlp_status() == 0
    Yo, _ = omlp.forward(_bf16_params(params), omlp.bf16_round(X), omlp.bf16_round)
    Yg = y.cpu().numpy()
    assert np.abs(Yg - Yo).max() < 2e-3 * max(1.0, np.abs(Yo).max())


def test_features_and_guess_match_oracle():
    s = synth.solvated_chain(60, 180, 26.0, 1103)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=(32, 32, 32), precision=binding.AP_FP64)
    c.build()
    c.permanent_field()
    feat = torch.zeros((s.n, 16), dtype=torch.float32, device="cuda")
    binding.ap_mlp_features(c.ctx, feat)
    E = c.field.cpu().numpy()
    Xo, _ = omlp.features(s.xyz, s.box, s.frame, s.alpha, E)
    np.testing.assert_allclose(feat.cpu().numpy(), Xo, rtol=2e-6, atol=2e-6)
    params = omlp.init_params(5)
    mu0 = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    binding.ap_learned_guess(c.ctx, _packed(params), mu0)
    torch.cuda.synchronize()
    want = omlp.guess(_bf16_params(params), s.xyz, s.box, s.frame, s.alpha, E,
                      lambda a: omlp.bf16_round(np.asarray(a, np.float32)), omlp.bf16_round)
    got = mu0.cpu().numpy()
    assert np.abs(got - want).max() < 2e-3 * omlp.OUT_SCALE * 10
    # targets invert the guess construction
    mu = torch.tensor(want, device="cuda")
    tgt = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
    binding.ap_mlp_features(c.ctx, feat, mu, tgt)
    t_o = omlp.targets(s.xyz, s.box, s.frame, s.alpha, E, want)
    np.testing.assert_allclose(tgt.cpu().numpy(), t_o, rtol=1e-5, atol=1e-5)
    c.close()
