"""Warm-start network on the GPU (tensor-core BF16 GEMMs, FP32 accumulation)
against the FP64 oracle of oracle/mlp.py: forward values, loss and gradients
of every parameter block, Adam updates, normalisation statistics, save/load.

Tolerances: BF16 keeps 8 significant bits (relative rounding 2^-9 ~ 2e-3 per
operand); the forward rounds the input, the weights and two hidden
activations, so values agree to about 1e-2 relative and gradients, which
also round dZ, to about 2e-2 (the bar set for this network).  Adam runs in
FP32 on given gradients and agrees to FP32 rounding."""
import numpy as np
import pytest
import torch

from oracle import mlp as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2107_02010_gb300 import otgb
    return otgb.Context()


def _setup(D, H, n, seed):
    r = np.random.default_rng(seed)
    theta = om.init_params(D, H, seed).astype(np.float32)
    k = 0
    for s in om.shapes(D, H):
        sz = int(np.prod(s))
        if len(s) == 1:
            theta[k:k + sz] = r.normal(0, 0.2, sz)
        k += sz
    x = r.normal(40.0, 25.0, (n, D)).astype(np.float32)
    y = r.normal(-30.0, 8.0, n).astype(np.float32)
    mean = r.normal(40.0, 2.0, D).astype(np.float32)
    scale = r.uniform(20.0, 30.0, D).astype(np.float32)
    norm = (mean.astype(np.float64), scale.astype(np.float64), -28.0, 6.0)
    return theta, x, y, norm


def _net(ctx, D, H, theta, norm):
    from paper_2107_02010_gb300 import otgb
    net = otgb.Mlp(ctx, D, H, seed=1)
    net.set_params(theta)
    net.set_normalization(norm[0], norm[1], norm[2], norm[3])
    return net


# inference runs the fused kernel (all layers per 128-row tile on chip); the sizes cover a single row, one
# tile, ragged tails of one row, inputs whose rows are not 16-byte aligned (D = 7, 3), H = 128, and many tiles
# per persistent CTA
@pytest.mark.parametrize("D,H,n", [(60, 256, 1000), (60, 256, 128), (60, 256, 1), (60, 128, 129), (7, 128, 333),
                                   (3, 256, 2049), (60, 256, 200_001)])
def test_forward_matches_oracle(ctx, D, H, n):
    theta, x, _, norm = _setup(D, H, n, seed=n + D)
    net = _net(ctx, D, H, theta, norm)
    pred = net.infer(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref, cache = om.forward(theta.astype(np.float64), x.astype(np.float64), D, H, norm)
    o = cache[-1]
    err = np.abs(pred - ref) / norm[3]               # in normalised units
    scale = np.sqrt(np.mean(o ** 2)) + 1.0
    assert np.max(err) <= 3e-2 * scale, (np.max(err), scale)
    assert np.mean(err) <= 1e-2 * scale, (np.mean(err), scale)


def test_forward_unaligned_input_is_identical(ctx):
    # D % 4 == 0 but the rows start 4 bytes past a 16-byte boundary: the fused kernel reads the input directly
    # instead of with one bulk copy per tile; the normalisation is the same float arithmetic, so the outputs
    # are bit-identical
    D, H, n = 60, 256, 300
    theta, x, _, norm = _setup(D, H, n, seed=11)
    net = _net(ctx, D, H, theta, norm)
    xa = torch.from_numpy(x).cuda()
    buf = torch.empty(n * D + 1, dtype=torch.float32, device="cuda")
    xu = buf[1:].view(n, D)
    xu.copy_(xa)
    assert xu.data_ptr() % 16 != 0
    pa = net.infer(xa)
    pu = net.infer(xu)
    assert torch.equal(pa, pu)


@pytest.mark.parametrize("D,H,n", [(60, 256, 777), (60, 256, 4096), (5, 128, 300)])
def test_gradient_matches_oracle(ctx, D, H, n):
    theta, x, y, norm = _setup(D, H, n, seed=3 * n + D)
    net = _net(ctx, D, H, theta, norm)
    loss, g = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    g = g.cpu().numpy().astype(np.float64)
    L, gr = om.loss_and_grad(theta.astype(np.float64), x.astype(np.float64), y.astype(np.float64), D, H, norm)
    assert abs(loss - L) <= 1e-2 * L, (loss, L)
    k = 0
    names = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]
    for name, s in zip(names, om.shapes(D, H)):
        sz = int(np.prod(s))
        a, b = g[k:k + sz], gr[k:k + sz]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 2e-2, (name, rel)
        k += sz
    # the network's own parameters are untouched by a gradient evaluation
    assert np.array_equal(net.get_params(), theta)


def test_adam_matches_oracle(ctx):
    D, H, n = 60, 256, 512
    theta, x, y, norm = _setup(D, H, n, seed=11)
    net = _net(ctx, D, H, theta, norm)
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t, lr in ((1, 1e-3), (2, 5e-4), (3, 2e-3)):
        _, g = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
        net.adam_step(g, lr)
        th, m, v = om.adam_step(th, m, v, g.cpu().numpy().astype(np.float64), t, lr)
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - th) / (np.abs(th) + 1e-3)) <= 1e-5, t


def test_training_step_equals_grad_then_adam(ctx):
    D, H, n = 60, 256, 700
    theta, x, y, norm = _setup(D, H, n, seed=12)
    a = _net(ctx, D, H, theta, norm)
    b = _net(ctx, D, H, theta, norm)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    la = a.train_step(xt, yt, 1e-3)
    lb, g = b.grad(xt, yt)
    b.adam_step(g, 1e-3)
    assert la == lb
    assert np.array_equal(a.get_params(), b.get_params())


def test_fit_normalization_matches_numpy(ctx):
    from paper_2107_02010_gb300 import otgb
    r = np.random.default_rng(5)
    D, n = 60, 12345
    x = (r.normal(0, 1, (n, D)) * r.uniform(1, 30, D) + r.uniform(-50, 80, D)).astype(np.float32)
    x[:, 7] = 3.25                                     # a constant feature gets scale 1
    f = r.normal(-12.0, 4.0, n).astype(np.float32)
    net = otgb.Mlp(ctx, D, 256)
    net.fit_normalization(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda())
    mean, scale, om_, os_ = net.get_normalization()
    xd = x.astype(np.float64)
    sd = xd.std(0)
    sd[7] = 1.0
    assert np.max(np.abs(mean - xd.mean(0)) / (np.abs(xd.mean(0)) + 1)) < 1e-6
    assert np.max(np.abs(scale - sd) / sd) < 1e-5
    assert abs(om_ - f.astype(np.float64).mean()) < 1e-5
    assert abs(os_ - f.astype(np.float64).std()) / f.std() < 1e-5


def test_save_load_roundtrip(ctx, tmp_path):
    from paper_2107_02010_gb300 import otgb
    D, H, n = 60, 256, 600
    theta, x, y, norm = _setup(D, H, n, seed=13)
    a = _net(ctx, D, H, theta, norm)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for _ in range(3):
        a.train_step(xt, yt, 1e-3)
    path = tmp_path / "net.bin"
    a.save(path)
    b = otgb.Mlp(ctx, D, H, seed=99)
    b.load_file(path)
    assert np.array_equal(a.get_params(), b.get_params())
    assert torch.equal(a.infer(xt), b.infer(xt))
    # the Adam state travels too: one more identical step stays identical
    a.train_step(xt, yt, 1e-3)
    b.train_step(xt, yt, 1e-3)
    assert np.array_equal(a.get_params(), b.get_params())
    with pytest.raises(otgb.OtgbError):
        otgb.Mlp(ctx, 30, H).load_file(path)


def test_training_fits_a_smooth_function(ctx):
    from paper_2107_02010_gb300 import otgb
    r = np.random.default_rng(21)
    D, n = 60, 40000
    x = r.normal(0, 1, (n, D)).astype(np.float32)
    w = r.normal(0, 1, D) / np.sqrt(D)
    y = (3.0 * np.sin(x @ w) + 0.5 * (x[:, :3] ** 2).sum(1)).astype(np.float32)
    net = otgb.Mlp(ctx, D, 256, seed=4)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net.fit_normalization(xt, yt)
    first = net.train_epoch(xt, yt, 2048, 1e-3, seed=0)
    for e in range(1, 15):
        last = net.train_epoch(xt, yt, 2048, 1e-3, seed=e)
    assert last < 0.05 * first, (first, last)
    # held-out rows
    xv = r.normal(0, 1, (4000, D)).astype(np.float32)
    yv = 3.0 * np.sin(xv @ w) + 0.5 * (xv[:, :3] ** 2).sum(1)
    pv = net.infer(torch.from_numpy(xv).cuda()).cpu().numpy()
    assert np.sqrt(np.mean((pv - yv) ** 2)) < 0.25 * yv.std()


def test_invalid_arguments(ctx):
    from paper_2107_02010_gb300 import otgb
    with pytest.raises(otgb.OtgbError):
        otgb.Mlp(ctx, 65, 256)
    with pytest.raises(otgb.OtgbError):
        otgb.Mlp(ctx, 60, 200)
    net = otgb.Mlp(ctx, 4, 128)
    with pytest.raises(otgb.OtgbError):
        net.set_params(np.zeros(3, np.float32))
    with pytest.raises(otgb.OtgbError):
        net.set_normalization(np.zeros(4), np.array([1, 1, 0, 1.0]), 0.0, 1.0)
