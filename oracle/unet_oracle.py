"""FP64 CPU oracle of the learned warm start / surrogate network.

TEST INFRASTRUCTURE ONLY (tests/, smoke and bench.py's baseline legs).  It
shares no code with the CUDA path.  Plain PyTorch CPU operations in float64;
gradients by torch.autograd (pinned by finite differences in the tests).

The network maps the load and the microstructure to the strain field that
warm-starts Algorithm 1 (the paper motivates learned surrogates of the
averaged response in Sec. 6, Eqs. 6.9-6.10, and Fig. 5; the architecture is
the project's): a 4-level 3D U-net on periodic volumes.

  inputs  (4 channels): b1, b2, b3 scaled by 1/max|b|, and the phase shear
          modulus mu(x) / mu_max - 1/2
  outputs (6 channels): eps * mu_max / max|b|, tensorial components
          (xx yy zz yz xz xy)
  level widths 32, 32, 32, 48; two 3^3 convolutions per level (circular
  padding: the fields are periodic), leaky ReLU (slope 0.1), 2^3 average
  pooling down, 2^3 stride-2 transposed convolution up, skip connections by
  channel concatenation (upsampled first, skip second), 1^3 head.

Flat parameter layout (shared interface with the CUDA path, FP32 there):
for each layer in LAYERS order, the weight in PyTorch's shape followed by the
bias: conv (cout, cin, k, k, k); transposed conv (cin, cout, 2, 2, 2).
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

SLOPE = 0.1

# (name, kind, cin, cout): kind conv3 | conv1 | up
LAYERS = (
    ("e0a", "conv3", 4, 32), ("e0b", "conv3", 32, 32),
    ("e1a", "conv3", 32, 32), ("e1b", "conv3", 32, 32),
    ("e2a", "conv3", 32, 32), ("e2b", "conv3", 32, 32),
    ("e3a", "conv3", 32, 48), ("e3b", "conv3", 48, 48),
    ("u2", "up", 48, 32), ("d2a", "conv3", 64, 32), ("d2b", "conv3", 32, 32),
    ("u1", "up", 32, 32), ("d1a", "conv3", 64, 32), ("d1b", "conv3", 32, 32),
    ("u0", "up", 32, 32), ("d0a", "conv3", 64, 32), ("d0b", "conv3", 32, 32),
    ("head", "conv1", 32, 6),
)


def weight_shape(kind, cin, cout):
    if kind == "conv3":
        return (cout, cin, 3, 3, 3)
    if kind == "conv1":
        return (cout, cin, 1, 1, 1)
    return (cin, cout, 2, 2, 2)


def param_count():
    n = 0
    for _, kind, cin, cout in LAYERS:
        s = weight_shape(kind, cin, cout)
        w = 1
        for d in s:
            w *= d
        n += w + cout
    return n


def unpack(flat):
    """Flat parameter vector -> {name: (weight, bias)} views."""
    out = {}
    i = 0
    for name, kind, cin, cout in LAYERS:
        s = weight_shape(kind, cin, cout)
        w = 1
        for d in s:
            w *= d
        out[name] = (flat[i:i + w].view(s), flat[i + w:i + w + cout])
        i += w + cout
    return out


def conv3_circ(x, w, b):
    """3^3 convolution with circular padding (cross-correlation, PyTorch convention)."""
    return F.conv3d(F.pad(x, (1, 1, 1, 1, 1, 1), mode="circular"), w, b)


def act(x):
    return F.leaky_relu(x, SLOPE)


def forward(flat, x):
    """x: (B, 4, nz, ny, nx) float64 -> (B, 6, nz, ny, nx)."""
    p = unpack(flat)

    def block(h, a, b):
        h = act(conv3_circ(h, *p[a]))
        return act(conv3_circ(h, *p[b]))

    s0 = block(x, "e0a", "e0b")
    s1 = block(F.avg_pool3d(s0, 2), "e1a", "e1b")
    s2 = block(F.avg_pool3d(s1, 2), "e2a", "e2b")
    h = block(F.avg_pool3d(s2, 2), "e3a", "e3b")
    for up, (a, b), skip in (("u2", ("d2a", "d2b"), s2), ("u1", ("d1a", "d1b"), s1),
                             ("u0", ("d0a", "d0b"), s0)):
        w, bias = p[up]
        h = F.conv_transpose3d(h, w, bias, stride=2)
        h = block(torch.cat([h, skip], dim=1), a, b)
    w, bias = p["head"]
    return F.conv3d(h, w, bias)


def loss(pred, target):
    """Mean over the batch of the squared relative L2 error ||pred - t||^2 / ||t||^2."""
    b = pred.shape[0]
    d = (pred - target).reshape(b, -1)
    t = target.reshape(b, -1)
    return ((d * d).sum(1) / (t * t).sum(1)).mean()


def init_params(seed):
    """He-style uniform initialisation (reproducible)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for _, kind, cin, cout in LAYERS:
        s = weight_shape(kind, cin, cout)
        fan_in = cin * (27 if kind == "conv3" else 1 if kind == "conv1" else 1)
        bound = (6.0 / fan_in) ** 0.5 * (0.5 if kind == "conv1" else 1.0)
        parts.append((torch.rand(s, generator=g, dtype=torch.float64) * 2 - 1).flatten() * bound)
        parts.append(torch.zeros(cout, dtype=torch.float64))
    return torch.cat(parts)


def features(b, phase, mus):
    """Network inputs from a load b (3, nz, ny, nx) and phase ids with shear moduli mus.
    Returns (x (4, ...), scale) with scale = max|b|."""
    b = torch.as_tensor(b, dtype=torch.float64)
    s = float(b.abs().max())
    mu = torch.as_tensor([m for m in mus], dtype=torch.float64)[torch.as_tensor(phase).long()]
    x = torch.cat([b / s, (mu / mu.max() - 0.5)[None]], dim=0)
    return x, s


def targets(eps, b, mus):
    """Training target of a strain field eps (6, ...): eps * mu_max / max|b|."""
    eps = torch.as_tensor(eps, dtype=torch.float64)
    s = float(torch.as_tensor(b, dtype=torch.float64).abs().max())
    return eps * (max(float(m) for m in mus) / s)


def adam_step(flat, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma and Ba 2014), bias-corrected, in place on flat, m, v."""
    m.mul_(beta1).add_(grad, alpha=1 - beta1)
    v.mul_(beta2).addcmul_(grad, grad, value=1 - beta2)
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    flat.sub_(lr * mh / (vh.sqrt() + eps))
