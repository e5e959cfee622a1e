"""The learned warm start end to end at a small size: plain-mODIL forward
solutions around 32 seeded ellipsoids on 16^3 (batched in one problem), a
3-level U-Net trained on them by the library's own kernels, then the inverse
problem on 32^3 from wake-slab data, zero-initialised against warm-started
(network prediction on level 2 of the decomposition)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import inputs, unet, warmstart
    return warmstart, inputs, unet


def test_warm_start_beats_zero_init(ws):
    W, inputs, unet = ws
    side, L = 16, 5
    cases = [inputs.ns3d_ellipsoid(10000 + i) for i in range(32)]
    fields, terms = W.forward_solves(cases, side, L, 2000)
    assert np.all(np.isfinite(terms)) and np.median(terms[:, 0]) < 1e-3
    xs = np.stack([W.unet_input((side,) * 3, *W.slab((side,) * 3, 10000 + i, c, a, fields[i]), side)
                   for i, (c, a) in enumerate(cases)])
    norm = W.Normaliser(fields)
    net, hist, _ = W.train(xs, norm.to_net(fields), epochs=40, batch=2, lr=1e-3, base_ch=8, levels=3)
    assert hist[-1] < 0.4 * hist[0]
    inf = unet.UNet(side, batch=1, in_ch=4, out_ch=5, base_ch=8, levels=3)
    inf.write_params(net.read_params())
    big = 2 * side
    c, a = inputs.ns3d_ellipsoid(5)
    fb, _ = W.forward_solves([(c, a)], big, L + 1, 4000)
    cells, fidx, vals = W.slab((big,) * 3, 5, c, a, fb[0])
    pred = W.predict(inf, norm, W.unet_input((big,) * 3, cells, fidx, vals, side))
    desc = W.inverse_problem((big,) * 3, L + 1, cells, fidx, vals)
    tol = [1e-3]
    hz, histz = W.steps_to_losses(desc, W.zero_levels((big,) * 3, L + 1), tol, 4000)
    hw, histw = W.steps_to_losses(desc, W.warm_levels((big,) * 3, L + 1, 1, pred), tol, 4000)
    # measured: zero init stalls near 6e-2, the warm start passes 1e-3 within ~200 steps
    assert hw[1e-3] is not None and hw[1e-3][0] <= 2000, (hw, histw[:5])
    assert hz[1e-3] is None or hz[1e-3][0] > 2 * hw[1e-3][0], (hz, hw)
    assert min(histw) < 0.1 * min(histz)
