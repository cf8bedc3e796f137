"""The network's tensor-core kernels against the FP64 reference.

The GPU rounds inputs, W1, W2 and the first hidden layer to bfloat16 and
accumulates in FP32; the reference takes the same bfloat16-rounded weights
and inputs in FP64.  Bound: activations carry a relative bfloat16 rounding of
2^-8, so outputs and gradient blocks must agree to a few 2^-8 in norm.
"""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

REL = 3e-2   # ~8 x 2^-8


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def setup(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.25, mlp.NPARAMS)
    p[512:576] = rng.normal(0.1, 0.05, 64)      # b1 > 0 keeps most units active
    p[4672:4736] = rng.normal(0.1, 0.05, 64)
    x = rng.normal(0.0, 1.0, (n, 8))
    t = np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2]
    return p, x, t


def reference_params(p):
    q = p.copy()
    q[0:512] = mlp.bf16_round(q[0:512])
    q[576:4672] = mlp.bf16_round(q[576:4672])
    return q


@pytest.mark.parametrize("n", [1, 17, 1000, 100003])
def test_forward(kl, n):
    import torch
    p, x, _ = setup(n, n)
    y = kl.mlp_forward(torch.tensor(p, dtype=torch.float32, device="cuda"),
                       torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = mlp.forward(reference_params(p), mlp.bf16_round(x))
    assert np.linalg.norm(y - ref) <= REL * np.linalg.norm(ref)
    assert np.max(np.abs(y - ref)) <= REL * max(1.0, np.max(np.abs(ref)))


BLOCKS = {"W1": (0, 512), "b1": (512, 576), "W2": (576, 4672), "b2": (4672, 4736),
          "w3": (4736, 4800), "b3": (4800, 4801)}


@pytest.mark.parametrize("n,under", [(37, 1.0), (4096, 1.0), (65539, 1.0), (4096, 4.0)])
def test_gradient(kl, n, under):
    import torch
    p, x, t = setup(n, 100 + n)
    tr = kl.MlpTrainer(torch.tensor(p, dtype=torch.float32, device="cuda"), under_weight=under)
    g, loss = tr.gradient(torch.tensor(x, dtype=torch.float32, device="cuda"),
                          torch.tensor(t, dtype=torch.float32, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    ref_loss, ref = mlp.loss_and_grad(reference_params(p), mlp.bf16_round(x), t, under)
    assert abs(float(loss.item()) - ref_loss) <= REL * ref_loss
    for name, (a, b) in BLOCKS.items():
        num = np.linalg.norm(g[a:b] - ref[a:b])
        den = np.linalg.norm(ref[a:b])
        assert num <= REL * den + 1e-7, (name, num / max(den, 1e-30))
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    assert cos > 0.999


def test_training_reduces_loss(kl):
    import torch
    p, x, t = setup(32768, 5)
    params = torch.tensor(p * 0.5, dtype=torch.float32, device="cuda")
    tr = kl.MlpTrainer(params, lr=3e-3)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    first = None
    for k in range(300):
        loss = float(tr.step(X, T).item())
        first = first if first is not None else loss
    # the loss value reported by the last step is that of the parameters before it
    final = mlp.loss_and_grad(params.double().cpu().numpy(), x, t)[0]
    assert final < 0.1 * first, (first, loss, final)


def test_training_is_deterministic(kl):
    """Gradients are summed in a fixed order: two runs from the same start on
    the same batches give bit-identical losses and parameters."""
    import torch
    p, x, t = setup(20000, 11)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    runs = []
    for _ in range(2):
        params = torch.tensor(p * 0.5, dtype=torch.float32, device="cuda")
        tr = kl.MlpTrainer(params, lr=3e-3, under_weight=4.0)
        losses = [float(tr.step(X, T).item()) for _ in range(20)]
        runs.append((losses, params.cpu().numpy().copy()))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])


def test_train_step_equals_gradient_then_adam(kl):
    """kl_mlp_train_step (gradient, fixed-order sum and Adam in one pass) gives
    bit for bit the parameters, moments and losses of kl_mlp_grad followed by
    kl_mlp_adam."""
    import torch
    p, x, t = setup(9000, 21)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    runs = []
    for fused in (True, False):
        params = torch.tensor(p * 0.5, dtype=torch.float32, device="cuda")
        tr = kl.MlpTrainer(params, lr=3e-3, under_weight=4.0)
        step = tr.step if fused else tr.step_separate
        losses = [float(step(X, T).item()) for _ in range(10)]
        runs.append((losses, params.cpu().numpy().copy(), tr.m.cpu().numpy().copy(),
                     tr.v.cpu().numpy().copy()))
    assert runs[0][0] == runs[1][0]
    for a, b in zip(runs[0][1:], runs[1][1:]):
        assert np.array_equal(a, b)


def test_bounded_wait_gives_up_and_the_device_stays_usable(kl):
    """The tensor-core kernels wait for their MMAs on an mbarrier with a
    bound.  A wait that nothing completes gives up after its bound and says
    so; a completed one succeeds; and the device still works afterwards."""
    import torch
    gave_up, completed, cycles = kl.binding.wait_selftest(2_000_000)
    assert gave_up and completed
    assert 2_000_000 <= cycles < 200_000_000
    with pytest.raises(kl.KlError):
        kl.binding.wait_selftest(0)
    # a forward pass right after still matches the oracle
    p, x, _ = setup(300, 300)
    y = kl.mlp_forward(torch.tensor(p, dtype=torch.float32, device="cuda"),
                       torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = mlp.forward(reference_params(p), mlp.bf16_round(x))
    assert np.linalg.norm(y - ref) <= REL * np.linalg.norm(ref)
