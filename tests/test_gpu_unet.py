"""GPU parity of the learned warm start network (BF16 kernels, FP32
accumulation) against the FP64 network oracle, through the C ABI.

The oracle is fed the BF16-rounded weights and inputs, so the remaining
difference is the BF16 rounding of activations and gradients inside the
network: about 2^-9 relative per stored value, accumulated over 21 layers.
Bars (relative L2): output <= 2e-2, loss <= 1e-2, each layer's weight and
bias gradient <= 5e-2.  A wrong tap, transposed weight, missing bias or a
skip connection in the wrong place gives errors of order 1.
"""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

DIMS = (24, 16, 16)   # (nx, ny, nz); coarsest level 3 x 2 x 2; untiled convolutions only
# (32, 16, 16): levels 0 and 1 run the shared-memory tiled convolution (16 x 8 x 2 tiles)
GRIDS = [DIMS, (32, 16, 16)]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16(t):
    return torch.as_tensor(t).to(torch.bfloat16).to(torch.float64)


def params(seed):
    """He-initialised weights with small random biases (so every bias path is exercised)."""
    flat = U.init_params(seed)
    g = torch.Generator().manual_seed(seed + 100)
    for name, (w, b) in U.unpack(flat).items():
        b.copy_((torch.rand(b.shape, generator=g, dtype=torch.float64) - 0.5) * 0.2)
    return flat


def inputs(seed, batch, dims=DIMS, ch=4):
    g = torch.Generator().manual_seed(seed)
    nx, ny, nz = dims
    return torch.rand((batch, ch, nz, ny, nx), generator=g, dtype=torch.float64) * 2 - 1


def layer_slices():
    i = 0
    for name, kind, cin, cout in U.LAYERS:
        w = int(np.prod(U.weight_shape(kind, cin, cout)))
        yield name, slice(i, i + w), slice(i + w, i + w + cout)
        i += w + cout


@pytest.mark.parametrize("dims", GRIDS)
def test_forward_matches_oracle(dims):
    flat = params(3)
    x = inputs(5, 2, dims)
    net = api.Net(dims, max_batch=2)
    y = net.forward(flat.float().cuda(), x.float().cuda()).double().cpu()
    net.status()
    ref = U.forward(bf16(flat), bf16(x))
    for s in range(2):
        assert rel(y[s], ref[s]) <= 2e-2, (s, rel(y[s], ref[s]))


def test_forward_full_training_size_matches_oracle():
    dims = (64, 64, 64)
    flat = params(4)
    x = inputs(6, 1, dims)
    net = api.Net(dims, max_batch=1)
    y = net.forward(flat.float().cuda(), x.float().cuda()).double().cpu()
    net.status()
    assert rel(y, U.forward(bf16(flat), bf16(x))) <= 2e-2


@pytest.mark.parametrize("dims", GRIDS)
def test_gradients_match_oracle(dims):
    flat = params(7)
    x = inputs(8, 2, dims)
    t = inputs(9, 2, dims, ch=6)
    net = api.Net(dims, max_batch=2, train=True)
    g, loss = net.grad(flat.float().cuda(), x.float().cuda(), t.float().cuda())
    g = g.double().cpu()
    p = bf16(flat).requires_grad_(True)
    lo = U.loss(U.forward(p, bf16(x)), t.float().double())
    gref, = torch.autograd.grad(lo, p)
    lo = float(lo.detach())
    assert abs(float(loss.item()) - lo) <= 1e-2 * lo
    for name, ws, bs in layer_slices():
        assert rel(g[ws], gref[ws]) <= 5e-2, (name, "weight", rel(g[ws], gref[ws]))
        assert rel(g[bs], gref[bs]) <= 5e-2, (name, "bias", rel(g[bs], gref[bs]))


def test_gradient_is_deterministic():
    flat = params(10).float().cuda()
    x = inputs(11, 2).float().cuda()
    t = inputs(12, 2, ch=6).float().cuda()
    net = api.Net(DIMS, max_batch=2, train=True)
    g1, l1 = net.grad(flat, x, t)
    g1 = g1.clone()
    g2, l2 = net.grad(flat, x, t)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)


def test_adam_matches_oracle():
    gen = torch.Generator().manual_seed(13)
    n = _lib.NET_PARAMS
    w, g, m = (torch.randn(n, generator=gen, dtype=torch.float64) for _ in range(3))
    v = torch.rand(n, generator=gen, dtype=torch.float64)
    w, g, m, v = (a.float().double() for a in (w, g, m, v))
    dev = [a.float().cuda() for a in (w, g, m, v)]
    net = api.Net((8, 8, 8))
    net.adam(dev[0], dev[1], dev[2], dev[3], 3, 1e-3)
    U.adam_step(w, g, m, v, 3, lr=1e-3)
    assert rel(dev[0].cpu(), w) <= 1e-6
    assert rel(dev[2].cpu(), m) <= 1e-6 and rel(dev[3].cpu(), v) <= 1e-6


def test_training_steps_reduce_the_loss():
    flat = params(14).float().cuda()
    xc = inputs(15, 2)
    x = xc.float().cuda()
    t = U.forward(params(16), xc).float().cuda()     # a target the network can represent
    net = api.Net(DIMS, max_batch=2, train=True)
    grad = torch.empty_like(flat)
    m = torch.zeros_like(flat)
    v = torch.zeros_like(flat)
    losses = [float(net.train_step(flat, grad, m, v, k, 1e-3, x, t).item()) for k in range(1, 31)]
    assert np.isfinite(losses).all() and losses[-1] < 0.8 * losses[0], losses


def test_prepare_predict_and_surrogate_match_oracle_features():
    p = W.config_c5_sample(3, n=32)
    phases = [tuple(q) for q in p.phases]
    mus = [q[1] for q in phases]
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    eps = torch.randn((6,) + tuple(b.shape[1:]), dtype=torch.float64, device="cuda")
    net = api.Net(p.dims, max_batch=2)
    x, tgt = net.prepare(b, ph, phases, eps=eps)
    xr, s = U.features(b.cpu(), ph.cpu(), mus)
    assert rel(x.cpu(), xr) <= 1e-6
    assert rel(tgt.cpu(), U.targets(eps.cpu(), b.cpu(), mus)) <= 1e-6
    flat = params(17)
    fl = flat.float().cuda()
    pred = net.predict(fl, [b, b], [ph, ph], phases)
    y = net.forward(fl, x[None])
    want = y[0].double() * (s / max(mus))
    assert rel(pred[0].cpu(), want.cpu()) <= 1e-6 and torch.equal(pred[0], pred[1])
    assert rel(pred[0].cpu(), U.forward(bf16(flat), bf16(xr[None]))[0] * (s / max(mus))) <= 2e-2
    with api.Plan(p.dims, "mixed") as plan:
        sur = plan.surrogate_infer(fl, b, ph, phases)
    assert torch.equal(sur, pred[0])


def test_trained_warm_start_reduces_sweeps_and_matches_cold_solver():
    """The committed trained network, on held-out 64^3 samples (seeds 0..7; the
    training seeds start at 1000000): its prediction is within 35% relative L2 of
    the solution, the warm-started batched ladder needs fewer FP32 sweeps than
    the cold one, and both land within the tolerance of each other (the cold
    solver is the reference)."""
    from paper_2601_00822_gb300 import surrogate as S
    params = S.load(S.DEFAULT_WEIGHTS)
    res = S.warm_start_benchmark(params, list(range(8)), 64, tol=1e-6, batch=8, plain=False)
    assert res["prediction_rel_l2_mean"] < 0.35, res
    assert res["batched_warm"]["mean_sweeps"] < res["batched_cold"]["mean_sweeps"], res
    assert res["batched_warm"]["max_resid"] <= 1e-6 and res["batched_cold"]["max_resid"] <= 1e-6
    assert res["warm_vs_cold_eps_rel_l2_max"] < 1e-5, res
