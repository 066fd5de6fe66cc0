"""GPU checks of the warm-start network kernels (lbm_wsnet_*) against the FP64
numpy oracle: forward output, masked MSE loss and every parameter gradient.

Tolerance: the CUDA path computes in FP32 with atomically accumulated weight
gradients, the oracle in FP64; with O(1) activations and ~10^3-term sums the
FP32 error is ~1e-5 of the largest value, so forward and gradients are
compared at 2e-4 of their maximum magnitude and the loss at 1e-5 relative."""
import numpy as np
import pytest

from oracle import wsnet_oracle as N

pytestmark = pytest.mark.gpu
CH = (8, 16, 32)


@pytest.fixture(scope="module")
def net():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    from paper_1806_10589_gb300 import WarmStartNet

    n = WarmStartNet(*CH)
    yield n
    n.close()


def _case(seed, B=2, shape=(8, 12, 8)):
    rng = np.random.default_rng(seed)
    masks = (rng.random((B,) + shape) < 0.35).astype(np.uint8)
    targets = rng.standard_normal((B, 3) + shape).astype(np.float32)
    params = (rng.standard_normal(N.n_params(*CH)) * 0.15).astype(np.float32)
    return masks, targets, params


def test_param_count(net):
    assert net.n_params == N.n_params(*CH)


def test_forward_matches_oracle(net):
    masks, _, p = _case(1, B=1)
    net.set_params(p)
    y = net.predict(masks[0])
    ref = N.forward(p.astype(np.float64), 1.0 - masks[0], CH)
    assert np.abs(y - ref).max() <= 2e-4 * max(1.0, np.abs(ref).max())
    assert np.all(y[:, masks[0] == 1] == 0)


def test_loss_and_gradient_match_oracle(net):
    masks, targets, p = _case(2)
    net.set_params(p)
    loss, g = net.loss_grad(masks, targets)
    # the oracle's loss is per sample; a batch of B shares one normalisation by
    # the total pore count, so sum the per-sample parts with that weight
    npore = float((masks == 0).sum())
    ref_loss, ref_g = 0.0, np.zeros(p.size)
    for b in range(masks.shape[0]):
        nb = float((masks[b] == 0).sum())
        lb, gb = N.loss_and_grad(p.astype(np.float64), 1.0 - masks[b], targets[b], CH)
        ref_loss += lb * nb / npore
        ref_g += gb * nb / npore
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.abs(g - ref_g).max() <= 2e-4 * np.abs(ref_g).max()


def test_training_reduces_loss(net):
    rng = np.random.default_rng(5)
    masks = (rng.random((6, 8, 8, 8)) < 0.3).astype(np.uint8)
    # a learnable target: a smooth function of the local pore fraction
    pore = 1.0 - masks.astype(np.float32)
    t = np.stack([pore * 0.5, pore * -0.2, pore * (1.0 + 0.1 * np.arange(8)[None, :, None, None])], axis=1)
    p = (rng.standard_normal(net.n_params) * 0.1).astype(np.float32)
    net.set_params(p)
    hist = net.train(masks, t.astype(np.float32), epochs=60, batch=3, lr=3e-3, seed=1)
    assert np.isfinite(hist).all()
    assert hist[-1] < 0.2 * hist[0], hist[[0, -1]]


def test_warm_start_pipeline_small(net):
    """End to end at small scale: steady targets from the batched LBM, a short
    training run, Kozeny-Carman calibration and a warm-started lattice that
    reaches the 0.1 % rule of a reference run."""
    import torch

    from lbm_inputs import sphere_pack
    from paper_1806_10589_gb300 import Batch, Lattice, convergence as cv, warmstart as ws

    st = torch.cuda.current_stream()
    masks = [sphere_pack(32, 5.0, 8.0, 0.4, seed=300 + k, cache=False)[0] for k in range(8)]
    targets, ks = ws.steady_targets(Batch, masks, 0.8, 1e-4, 3000, stream=st)
    assert np.isfinite(targets).all() and (ks > 0).all()
    c_kc = ws.fit_kc(masks, ks)
    assert c_kc > 0
    net.set_params(ws.he_init(net, 0))
    hist = net.train(np.stack(masks), targets, epochs=20, batch=4, lr=1e-3, seed=0)
    assert hist[-1] < hist[0]
    m = sphere_pack(32, 5.0, 8.0, 0.4, seed=999, cache=False)[0]
    Q = 1e-4 * int((m[0] == 0).sum())
    with Lattice(m, 0.8, "mrt", "fp32", stream=st) as lat:
        lat.set_flux_bc(Q)
        ref = cv.run_to_residual(lat, Q, 0.8, lag=500, tol=1e-6, max_steps=40000)
    res = ws.warm_vs_cold(Lattice, net, m, Q, 0.8, c_kc, ref["k"], stream=st, max_steps=40000)
    info = {"res": res, "k_ref": ref["k"]}
    assert res["cold"]["reached"] and res["warm"]["reached"], info
    assert abs(res["warm"]["k"] - ref["k"]) <= 1e-3 * ref["k"]
