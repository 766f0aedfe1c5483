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
    o = Oracle(s, Params(beta=0.5446, grid=(32, 32, 32), cutoff=7.0))
    E1 = omlp.short_field(s.n, o.I, o.J, o.R, s.alpha, E, 0.5446, 0.39)
    Xo, _ = omlp.features(s.xyz, s.box, s.frame, s.alpha, E, E1)
    np.testing.assert_allclose(feat.cpu().numpy(), Xo, rtol=2e-6, atol=2e-6)
    params = omlp.init_params(5)
    mu0 = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    binding.ap_learned_guess(c.ctx, _packed(params), mu0)
    torch.cuda.synchronize()
    want = omlp.guess(_bf16_params(params), s.xyz, s.box, s.frame, s.alpha, E, E1,
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


@pytest.mark.parametrize("n", [128, 777, 5000])
def test_gradient_matches_oracle(n):
    """Tensor-core backward (BF16 operands) vs the oracle's FP64 analytic gradients at
    the BF16-rounded parameters and inputs: relative error per parameter block."""
    params = omlp.init_params(21)
    params[1] = np.random.default_rng(4).normal(size=128) * 0.1
    params[3] = np.random.default_rng(5).normal(size=128) * 0.1
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, 16))
    T = rng.normal(size=(n, 3))
    grad = torch.zeros(binding.ap_mlp_param_count(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    binding.ap_mlp_gradient(_packed(params), torch.tensor(X, dtype=torch.float32, device="cuda"),
                            torch.tensor(T, dtype=torch.float32, device="cuda"), grad, loss)
    torch.cuda.synchronize()
    assert binding.ap_mlp_status() == 0
    L, G = omlp.loss_and_grads(_bf16_params(params), omlp.bf16_round(X), T)
    assert abs(float(loss.cpu()[0]) - L) < 1e-2 * L
    g = omlp.unflatten(grad.cpu().numpy().astype(np.float64))
    for k, (gg, go) in enumerate(zip(g, G)):
        err = np.linalg.norm(gg - go) / max(np.linalg.norm(go), 1e-30)
        assert err < 4e-2, (k, err)


def test_training_reduces_loss():
    """Fit a seeded teacher network's outputs: 300 Adam steps on the GPU kernels."""
    teacher = omlp.init_params(99)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(4096, 16))
    T, _ = omlp.forward(teacher, X)
    P = binding.ap_mlp_param_count()
    params = torch.tensor(omlp.flatten(omlp.init_params(1)), dtype=torch.float32, device="cuda")
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    m = torch.zeros(P, dtype=torch.float32, device="cuda")
    v = torch.zeros(P, dtype=torch.float32, device="cuda")
    packed = torch.zeros(binding.ap_mlp_packed_bytes(), dtype=torch.uint8, device="cuda")
    binding.ap_mlp_pack(params, packed)
    feat = torch.tensor(X, dtype=torch.float32, device="cuda")
    tgt = torch.tensor(T, dtype=torch.float32, device="cuda")
    losses = []
    for step in range(1, 301):
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        binding.ap_mlp_train_step(params, grad, m, v, step, 2e-3, feat, tgt, loss, packed)
        losses.append(loss)
    torch.cuda.synchronize()
    assert binding.ap_mlp_status() == 0
    l0, l1 = float(losses[0].cpu()[0]), float(losses[-1].cpu()[0])
    assert l1 < 0.1 * l0, (l0, l1)
