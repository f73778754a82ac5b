"""Parity at the size the bench times: the SDSS-shaped batch of 8,192 stamps of
128 x 128 with 41 x 41 PSFs (1.2 GB of inputs), in the launch shape the tuning
table gives it, against the FP64 oracle on sampled galaxies.

The oracle cannot render or fit 8,192 galaxies in a test's time, so the batch
is made of a few galaxies of the recipe rendered by the oracle, repeated: slot g
holds source g % S.  The GPU runs over the whole batch exactly as the bench
launches it (every tile of every slot through the persistent item queue); its
outputs at sampled slots (the first, the last and across the batch) must match
the oracle's values for their source to the tolerances of test_gpu_parity.py,
and every copy of a source must give bit-identical results (no interference
between galaxies, tiles or queue items at full size)."""
import math

import numpy as np
import pytest

import oracle
from cases import from_batch
from paper_2404_07780_b300 import synth
from test_gpu_parity import FIT_TIGHT, _compare_fits, _oracle_normal, oracle_inputs

pytestmark = pytest.mark.gpu

G_FULL = 8192  # the bench's batch
S = 6          # oracle-rendered sources


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2404_07780_b300 import gm as gmod
    from paper_2404_07780_b300.build import build_lib
    build_lib()
    gmod.load()
    c = from_batch(synth.draw_sdss(seed=1000, G=S), at="init")
    src = np.arange(G_FULL) % S
    t = dict(params=torch.from_numpy(np.ascontiguousarray(c.params[src])).cuda(),
             psf=torch.from_numpy(np.ascontiguousarray(c.psf[src])).cuda(),
             image=torch.from_numpy(np.ascontiguousarray(c.image[src])).cuda(),
             sigma=torch.from_numpy(np.ascontiguousarray(c.sigma[src])).cuda(),
             mask=torch.from_numpy(np.ascontiguousarray(c.mask[src])).cuda())
    return gmod, c, src, t


def _sampled():
    rng = np.random.default_rng(0)
    return sorted(set([0, 1, S - 1, G_FULL // 2, G_FULL - 2, G_FULL - 1] + list(rng.integers(0, G_FULL, 6))))


def _same_per_source(x, src):
    for s in range(S):
        rows = x[src == s]
        assert (rows == rows[0]).all(), s  # bit-identical copies


def test_fullsize_normal_equations(full):
    gm, c, src, t = full
    chi2, grad, jtj = gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                      want_grad=True, want_jtj=True)
    # the launch shape the bench runs for this workload (K = 41, 8 free parameters)
    from paper_2404_07780_b300 import tune
    entries = tune.read_cache().get(tune.device_name(), {}).get("entries", [])
    tuned = [(e["pairs_per_pass"], e["pairs_per_thread"], e["groups"]) for e in entries if (e["K"], e["P"]) == (41, 8)]
    if tuned:
        assert gm.gm_tune_last_shape() == tuned[0]
    chi2, grad, jtj = (x.cpu().numpy() for x in (chi2, grad, jtj))
    for x in (chi2, grad, jtj):
        _same_per_source(x, src)
    rchi2, rg, rA = _oracle_normal(c)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for g in _sampled():
        s = src[g]
        assert abs(chi2[g] - rchi2[s]) <= 1e-5 * rchi2[s], g
        d = np.sqrt(np.diag(rA[s]))
        assert (np.abs(grad[g, free] + 2.0 * rg[s]) <= 1e-4 * d * math.sqrt(rchi2[s])).all(), g
        assert (np.abs(jtj[g][np.ix_(free, free)] - rA[s]) <= 1e-4 * np.outer(d, d)).all(), g


def test_fullsize_fit(full):
    gm, c, src, t = full
    got = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                          gm.FitOptions(**FIT_TIGHT))
    got = {k: v.cpu().numpy() for k, v in got.items()}
    for k in ("params", "chi2", "status", "iters", "sigma_p"):
        _same_per_source(got[k], src)
    n = 4  # sources fitted by the oracle
    oi = oracle_inputs(c)
    ref = oracle.fit(c.spec, c.params[:n], oi["psf"][:n], oi["image"][:n], oi["sigma"][:n], c.mask[:n],
                     oracle.FitOptions(**FIT_TIGHT))
    picks = [g for g in _sampled() if src[g] < n]
    sub = {k: v[picks] for k, v in got.items()}
    rsub = {k: np.asarray(v)[src[picks]] for k, v in ref.items() if np.ndim(v) > 0}
    same, rel = _compare_fits(c.spec, sub, rsub)
    # from the default start every fit ends with the oracle's status, and every converged
    # fit at the oracle's minimum: the same chi^2 and the same parameters
    np.testing.assert_array_equal(sub["status"], rsub["status"])
    assert (same == (rsub["status"] == 1)).all(), (sub["chi2"], rsub["chi2"])
    assert rel[same].max() <= 1e-4, rel[same].max(axis=1)


def test_fullsize_uneven_normal_equations(full):
    """The uneven workload's batch as the bench draws it: 32,768 bulge+disk stamps of side
    48-256 with PSF sides 25-51, every slot at its recipe geometry and start.  Sampled slots
    carry their galaxy rendered by the oracle; the others hold flat images (10 +- 2) and delta
    PSFs made on the host, so that the pass runs over the full geometry mix while the oracle
    renders only what is compared."""
    import torch
    from test_gpu_uneven import _oracle_normal_one
    gm = full[0]
    G = 32768
    rb = synth.draw_uneven_bulge_disk(seed=2000, G=G, sides=(48, 64, 96, 128, 192, 256), ks=tuple(range(25, 52, 2)))
    po, ko = rb.pix_offsets(), rb.psf_offsets()
    image = np.full(po[-1], 10.0, np.float32)
    sigma = np.full(po[-1], 2.0, np.float32)
    mask = np.zeros(po[-1], np.uint8)
    psf = np.zeros(ko[-1], np.float32)
    k = rb.geom[:, 2].astype(np.int64)
    psf[ko[:-1] + (k * k) // 2] = 1.0  # centre tap of each odd-sided PSF
    rng = np.random.default_rng(1)
    picks = sorted(set([0, G // 2, G - 1] + list(rng.integers(0, G, 9))))
    cases = {}
    for g in picks:
        cg = from_batch(rb.galaxy(g), at="init")
        cases[g] = cg
        image[po[g]:po[g + 1]] = cg.image.ravel()
        sigma[po[g]:po[g + 1]] = cg.sigma.ravel()
        if cg.mask is not None:
            mask[po[g]:po[g + 1]] = cg.mask.ravel()
        psf[ko[g]:ko[g + 1]] = cg.psf.ravel()
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    chi2, grad, jtj = gm.gm_chi2_grad(rb.spec, t(rb.init), t(image), t(sigma), t(mask), t(psf),
                                      want_grad=True, want_jtj=True, geom=rb.geom)
    chi2, grad, jtj = (x.cpu().numpy() for x in (chi2, grad, jtj))
    free = [i for i in range(rb.spec.n_slots) if rb.spec.free[i]]
    for g in picks:
        rc, rg, rA = _oracle_normal_one(cases[g])
        assert abs(chi2[g] - rc) <= 1e-5 * rc, g
        d = np.sqrt(np.diag(rA))
        assert (np.abs(grad[g, free] + 2.0 * rg) <= 1e-4 * d * math.sqrt(rc)).all(), g
        assert (np.abs(jtj[g][np.ix_(free, free)] - rA) <= 1e-4 * np.outer(d, d)).all(), g


def test_fullsize_adjoint_gradient(full):
    """The gradient workload's batch: 4,096 bulge+bar+nucleus stamps of 96 x 96 with 41 x 41
    PSFs (15 free parameters) through the adjoint pass, from five oracle-rendered galaxies
    repeated (an odd count, so that the two galaxies sharing a lane pair differ from pair to
    pair); sampled slots against the oracle's chi^2 and gradient for their source."""
    import torch
    gm = full[0]
    G, S5 = 4096, 5
    c = from_batch(synth.draw_bulge_bar_nucleus(seed=3000, G=S5, H=96, W=96, K=41), at="init")
    src = np.arange(G) % S5
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a[src])).cuda()
    chi2, grad = gm.gm_grad_adjoint(c.spec, t(c.params), t(c.image), t(c.sigma), t(c.mask), t(c.psf))
    chi2, grad = chi2.cpu().numpy(), grad.cpu().numpy()
    rchi2, rg, rA = _oracle_normal(c)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    rng = np.random.default_rng(2)
    for g in sorted(set([0, 1, G // 2, G - 1] + list(rng.integers(0, G, 8)))):
        s = src[g]
        assert abs(chi2[g] - rchi2[s]) <= 1e-5 * rchi2[s], g
        d = np.sqrt(np.diag(rA[s]))
        assert (np.abs(grad[g, free] + 2.0 * rg[s]) <= 1e-4 * d * math.sqrt(rchi2[s])).all(), g


def test_fullsize_cnn_inference():
    # the initialiser's inference as the bench times it: 65,536 stamps through predict() in
    # batches of 16,384 (the fused first two layers take ~221 tiles per block, both
    # accumulators and both operand sets many times over); sampled rows equal the training
    # forward pass on the same stamps bit for bit, and the first layer of the sample equals the
    # FP64 reference to the BF16 bounds
    import torch
    from oracle import cnn as ref
    from paper_2404_07780_b300 import cnn
    cnn.lib()
    net = cnn.Net(seed=11, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)
    n = 65536
    x = torch.asinh(3.0 * torch.randn((n, 64, 64, 1), generator=gen, device="cuda")).to(torch.bfloat16)
    pred = net.predict(x)
    idx = torch.tensor([0, 1, 16383, 16384, 40000, 65534, 65535] + list(range(997, 65536, 4099)), device="cuda")
    want = net.forward(x[idx].contiguous())[1]
    assert torch.equal(pred[idx], want)
    a1 = cnn.conv_fwd(x[idx].contiguous(), net.w(0), net.b(0), relu=True).float().cpu().numpy().astype(np.float64)
    xr = x[idx].float().cpu().numpy().astype(np.float64)
    w1 = net.w(0).float().cpu().numpy().astype(np.float64)
    b1 = net.b(0).float().cpu().numpy().astype(np.float64)
    r1 = ref.conv_fwd(xr, w1, b1, relu=True)
    scale = np.sqrt(ref.conv_fwd(xr ** 2, w1 ** 2) + b1 ** 2)
    assert np.all(np.abs(a1 - r1) <= 2.0 ** -8 * np.abs(r1) + 1e-4 * scale + 1e-30)
    cnn.check_device_error()
