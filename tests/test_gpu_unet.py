"""The tcgen05 BF16 GEMM and the U-Net of the warm start on the GPU against
numpy and the U-Net oracle (BF16 rounding emulated at the device's rounding
points, so only FP32 accumulation order differs)."""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2303_04679_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def unet():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import unet as u
    return u


def _bf16_tensor(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 32, 16), (256, 64, 200), (200, 48, 136),
                                   (1024, 128, 640), (384, 256, 1000), (512, 864, 96),
                                   (136, 200, 72)])
def test_gemm_store_f32(unet, M, N, K):
    import torch
    rng = np.random.default_rng(M + N + K)
    A = U.bf16(rng.normal(size=(M, K)))
    B = U.bf16(rng.normal(size=(N, K)))
    bias = rng.normal(size=N).astype(np.float32)
    Kp = (K + 7) // 8 * 8
    At = torch.zeros((M, Kp), dtype=torch.bfloat16, device="cuda")
    Bt = torch.zeros((N, Kp), dtype=torch.bfloat16, device="cuda")
    At[:, :K] = _bf16_tensor(A)
    Bt[:, :K] = _bf16_tensor(B)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    unet.gemm_bf16(At[:, :K], Bt[:, :K], D, mode=1, bias=torch.from_numpy(bias).cuda())
    torch.cuda.synchronize()
    ref = A @ B.T + bias
    scale = np.abs(A) @ np.abs(B).T + np.abs(bias)
    err = np.abs(D.cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * scale + 1e-30), float(np.max(err / scale))


def test_gemm_bf16_bias_relu(unet):
    import torch
    rng = np.random.default_rng(3)
    M, N, K = 512, 64, 288
    A, B = U.bf16(rng.normal(size=(M, K))), U.bf16(rng.normal(size=(N, K)))
    bias = rng.normal(size=N).astype(np.float32)
    D = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    unet.gemm_bf16(_bf16_tensor(A), _bf16_tensor(B), D, mode=0, relu=True,
                   bias=torch.from_numpy(bias).cuda())
    torch.cuda.synchronize()
    exact = np.maximum(A @ B.T + bias, 0.0)
    got = D.float().cpu().numpy()
    # one BF16 rounding of an FP32 sum: within one BF16 ulp of the exact value
    assert np.all(np.abs(got - exact) <= 2.0 ** -7 * np.abs(exact) + 1e-6)
    assert np.mean(got == U.bf16(exact)) > 0.99


def test_gemm_split_k_atomic(unet):
    import torch
    rng = np.random.default_rng(4)
    M, N, K = 256, 32, 8192
    A, B = U.bf16(rng.normal(size=(M, K))), U.bf16(rng.normal(size=(N, K)))
    D = torch.ones((M, N), dtype=torch.float32, device="cuda")
    unet.gemm_bf16(_bf16_tensor(A), _bf16_tensor(B), D, mode=2, splits=16)
    torch.cuda.synchronize()
    ref = 1.0 + A @ B.T
    scale = 1.0 + np.abs(A) @ np.abs(B).T
    assert np.max(np.abs(D.cpu().numpy() - ref) / scale) <= 2e-6


def _net(unet, spec, side, batch, seed):
    net = unet.UNet(side, batch=batch, in_ch=spec.in_ch, out_ch=spec.out_ch, base_ch=spec.base,
                    levels=spec.levels, lr=1e-3)
    shapes = [s for _, s in [(k, s) for k, s in net.param_shapes()]]
    assert [tuple(s) for s in shapes] == [tuple(s) for s in spec.param_shapes()]
    params = inputs.unet_params(spec.param_shapes(), seed, bias_scale=0.05)
    net.write_params(params)
    return net, [p.astype(np.float64) for p in params]


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("implicit", [True, False])
@pytest.mark.parametrize("levels,base,side,batch", [(2, 8, 8, 1), (4, 8, 16, 2), (4, 32, 16, 1), (3, 16, 32, 1)])
def test_unet_forward_and_gradients(unet, levels, base, side, batch, implicit):
    """Forward pass, loss and every parameter gradient against the oracle,
    with the 3x3x3 convolutions as implicit GEMMs (grids of 8^3 and more) or
    through im2col."""
    import torch
    spec = U.Spec(levels=levels, base=base, in_ch=4, out_ch=5)
    net, params = _net(unet, spec, side, batch, seed=10 + levels + base)
    net.set_implicit(implicit)
    rng = np.random.default_rng(20)
    x = rng.normal(size=(batch, side, side, side, 4)).astype(np.float32)
    y = rng.normal(size=(batch, side, side, side, 5)).astype(np.float32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = net.forward(xt).cpu().numpy()
    ref, _ = U.forward(spec, params, x.astype(np.float64))
    assert _rel(out, ref) <= 5e-3, _rel(out, ref)
    loss = net.eval_grad(xt, yt)
    lref, gref = U.loss_and_grads(spec, params, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - lref) <= 1e-3 * lref
    grads = net.read_grads()
    errs = []
    for i, (g, r) in enumerate(zip(grads, gref)):
        assert g.shape == r.shape
        errs.append(_rel(g, r))
    # exact FP64 network (no BF16 rounding): how far BF16 arithmetic itself is
    _, gexact = U.loss_and_grads(spec, params, x.astype(np.float64), y.astype(np.float64),
                                 emulate=False)
    bf16_noise = [_rel(a, b) for a, b in zip(gref, gexact)]
    print("gpu vs emulated:", np.round(errs, 4).tolist())
    print("emulated vs exact:", np.round(bf16_noise, 4).tolist())
    # BF16 criterion: the device may deviate from the BF16-emulating oracle by
    # no more than BF16 arithmetic itself deviates from the exact network
    # (rounding-boundary flips differ between FP32 and FP64 accumulation and
    # propagate through later roundings and ReLU masks), floor 1e-2
    for i, (e, nz) in enumerate(zip(errs, bf16_noise)):
        assert e <= max(1e-2, nz), (i, e, nz)
    net.close()


def test_unet_first_adam_step(unet):
    """First Adam step from zero moments: p - lr g / (|g| + eps) (bias-corrected),
    i.e. a step of lr against the sign of the oracle gradient wherever |g| >> eps."""
    import torch
    spec = U.Spec(levels=3, base=8, in_ch=4, out_ch=5)
    net, params = _net(unet, spec, 8, 1, seed=40)
    rng = np.random.default_rng(41)
    x = rng.normal(size=(1, 8, 8, 8, 4)).astype(np.float32)
    y = rng.normal(size=(1, 8, 8, 8, 5)).astype(np.float32)
    net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    _, gref = U.loss_and_grads(spec, params, x.astype(np.float64), y.astype(np.float64))
    new = net.read_params()
    lr = 1e-3
    agree = total = 0
    for p0, p1, g in zip(params, new, gref):
        big = np.abs(g) > 0.05 * np.max(np.abs(g))  # sign not decided by BF16 noise
        exp = p0 - lr * np.sign(g)
        agree += int(np.sum(np.abs(p1 - exp)[big] <= 1e-6 + 1e-6 * np.abs(exp[big])))
        total += int(np.sum(big))
    assert agree >= 0.99 * total, (agree, total)
    net.close()


def test_unet_training_reduces_loss(unet):
    """A learnable map (a scaled copy of the input channels and a product of
    two of them) fitted by Adam through the device's own forward and backward
    passes."""
    import torch
    spec = U.Spec(levels=4, base=8, in_ch=4, out_ch=5)
    net = unet.UNet(8, batch=2, in_ch=4, out_ch=5, base_ch=8, levels=4, lr=1e-3)
    net.write_params(inputs.unet_params(spec.param_shapes(), 30))
    rng = np.random.default_rng(31)
    x = rng.normal(size=(2, 8, 8, 8, 4)).astype(np.float32)
    y = np.concatenate([0.5 * x, (x[..., :1] * x[..., 1:2])], axis=-1).astype(np.float32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    first = net.train_step(xt, yt)
    for _ in range(300):
        last = net.train_step(xt, yt)
    # the FP64 oracle with the same Adam settings goes from 0.48 to 0.15 here
    assert last < 0.45 * first, (first, last)
    net.close()


def test_graph_replayed_steps_equal_direct_steps(unet):
    """Training steps replayed from the captured graph (inputs copied into the
    network's buffers, Adam's coefficients on the device) match the same steps
    launched directly, with a new input tensor every step.  The loss and the
    split-K weight gradients are summed with atomics, so the two agree to the
    order of those sums: the losses to 1e-12, the parameters within 1e-6
    except where Adam's sign step flips on a near-zero gradient (a stale input
    would change the loss, a wrong bias correction every parameter)."""
    import torch
    spec = U.Spec(levels=3, base=8, in_ch=4, out_ch=5)
    nets = []
    for graph in (True, False):
        net, _ = _net(unet, spec, 16, 1, seed=60)
        net.set_graph(graph)
        nets.append(net)
    rng = np.random.default_rng(61)
    for _ in range(4):
        x = torch.from_numpy(rng.normal(size=(1, 16, 16, 16, 4)).astype(np.float32)).cuda()
        y = torch.from_numpy(rng.normal(size=(1, 16, 16, 16, 5)).astype(np.float32)).cuda()
        losses = [net.train_step(x.clone(), y.clone()) for net in nets]
        assert abs(losses[0] - losses[1]) <= 1e-12 * abs(losses[1]), losses
    close = total = 0
    for a, b in zip(nets[0].read_params(), nets[1].read_params()):
        d = np.abs(a - b)
        assert np.all(d <= 8e-3), float(d.max())  # at most one sign flip per step (lr 1e-3)
        close += int(np.sum(d <= 1e-6))
        total += d.size
    assert close >= 0.99 * total, (close, total)
    for net in nets:
        net.close()
