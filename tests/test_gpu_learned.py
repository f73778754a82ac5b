"""The learned initialiser end to end on the GPU: the network's backward pass
through all six layers against the FP64 reference chain, training on stamps
rendered by gm_model, and what the trained network gains over the default
start of the LM fit on held-out galaxies."""
import numpy as np
import pytest

from oracle import cnn as ref
from paper_2404_07780_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2404_07780_b300 import cnn
    from paper_2404_07780_b300.build import build_lib
    build_lib()
    cnn.lib()
    return cnn


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_network_gradients_match_the_reference_chain(C):
    import torch
    net = C.Net(seed=3)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.normal(size=(6, 64, 64, 1)).astype(np.float32)).cuda().to(torch.bfloat16)
    t = torch.from_numpy(rng.normal(size=(6, 14)).astype(np.float32)).cuda()
    acts, pred = net.forward(x)
    loss, dpred = C.mse(pred, t, 14)
    net.backward(acts, dpred)
    # the reference chain runs on the GPU's own BF16 activations and weights, layer by layer
    A = [_np(a) for a in acts]
    _, d = ref.mse(A[-1], _np(t), 14)
    grads = []
    for li in range(len(C.LAYERS) - 1, -1, -1):
        kind, i, o = C.LAYERS[li]
        W = _np(net.w(li))
        x_in = A[li]
        if kind == "dense":
            xf = x_in.reshape(x_in.shape[0], -1)
            dw, db = ref.dense_bwd_weight(xf, d)
            d = ref.dense_bwd_data(d, W, mask=xf)
        else:
            d4 = d.reshape(x_in.shape[0], (x_in.shape[1] + 1) // 2, (x_in.shape[2] + 1) // 2, o)
            dw, db = ref.conv_bwd_weight(x_in, d4)
            d = ref.conv_bwd_data(d4, W, x_in.shape[1], x_in.shape[2], mask=x_in)
        grads.append((li, dw, db))
    for li, dw, db in grads:
        gw = _np(net._view(net.grad, 2 * li))
        gb = _np(net._view(net.grad, 2 * li + 1))
        # BF16 rounding of the upstream gradients at every layer: 2 % in the Frobenius norm
        assert np.linalg.norm(gw - dw) <= 2e-2 * np.linalg.norm(dw) + 1e-12, li
        assert np.linalg.norm(gb - db) <= 2e-2 * np.linalg.norm(db) + 1e-12, li


def test_trained_network_saves_lm_iterations(C):
    import torch
    from paper_2404_07780_b300 import gm, workloads
    X, T, codec = C.make_training_set(65536, seed=7)
    net = C.Net(seed=0)
    losses = C.train(net, X, T, codec.dv, epochs=2, batch=512, lr=2e-3)
    assert losses[-1] < 0.5 * losses[0], losses

    rb = synth.draw_uneven_bulge_disk(seed=99, G=512, sides=(128,))
    dev = torch.device("cuda")
    image, sigma, psf = workloads.render_uneven(rb, dev)
    G = rb.G
    p_def = torch.from_numpy(rb.init).to(dev)
    opts = gm.FitOptions(tol=1e-6, max_iter=200)
    f = gm.Fitter(rb.spec, G, device=dev, geom=rb.geom)
    d = {k: v.clone() for k, v in f.fit(p_def.clone(), image, sigma, None, psf, opts).items()}
    p_learn = C.learned_start(net, image.view(G, 128, 128), codec, rb.spec)
    r, info = C.fit_with_fallback(f, rb.spec, p_learn, p_def, image, sigma, None, psf, opts, geom=rb.geom)
    refits = info["refits"]
    it_d = d["iters"].float().mean().item()
    it_l = r["iters"].float().mean().item()
    conv_d = (d["status"] == 1).float().mean().item()
    conv_l = (r["status"] == 1).float().mean().item()
    c2_d, c2_l = d["chi2"].cpu().numpy(), r["chi2"].cpu().numpy()
    rel = (c2_l - c2_d) / c2_d
    dof = d["dof"].cpu().numpy().astype(np.float64)
    dchi = (c2_l - c2_d) / np.sqrt(2 * dof)  # in units of the chi^2 scatter
    print(f"default: {it_d:.1f} iterations, {conv_d:.3f} converged; learned: {it_l:.1f} iterations, "
          f"{conv_l:.3f} converged, {refits} refits; chi2 relative change quantiles "
          f"{np.quantile(rel, [0.01, 0.05, 0.5, 0.95, 0.99])}; worse by > 1 sigma_chi2 {np.mean(dchi > 1):.3f}, "
          f"better by > 1 sigma_chi2 {np.mean(dchi < -1):.3f}")
    assert it_l < 0.8 * it_d
    assert conv_l >= conv_d - 0.01
    # the learned start may land in another local minimum than the default one; it must not
    # do so to the detriment of the fits more often than the default start does
    assert np.mean(dchi > 1) <= np.mean(dchi < -1) + 0.02
