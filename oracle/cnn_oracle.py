"""FP64 CPU oracle of the subimage surrogate network -- TEST INFRASTRUCTURE ONLY.

The paper has no learned part. The library adds one for the first
hierarchical level: a small 3D CNN that maps a buffered subimage's phase
voxels to the 21 upper-triangle components of its core's effective Voigt
stiffness, trained on subimages that the FFT solver homogenized, and a gate
that defers to the FFT solver whenever the ensemble's prediction is not
trustworthy. This module states what that network computes, plainly and in
FP64, so that the CUDA kernels (BF16 operands, FP32 accumulation) can be
checked against it:

  input   one-hot of the labels 0, 1, 2 and the core mask (4 channels, box
          Omega_B of any shape: the core Omega_R is 1, the buffer 0)
  conv1   4 -> 16, 3x3x3, stride 1, zero padding 1, bias, ReLU
  conv2  16 -> 32, stride 2, ReLU
  conv3  32 -> 64, stride 2, ReLU
  conv4  64 -> 64, stride 1, ReLU
  pool    mean over the remaining voxels -> 64
  fc1     64 -> 128, ReLU
  fc2    128 -> 21 (normalised stiffness components)

Flat parameter layout (shared with the CUDA path): for each conv layer the
weights W[tap][ci][co] with tap = (kz * 3 + ky) * 3 + kx, then the bias[co];
for each fully connected layer W[in][out], then bias[out]; layers in order.

A core is given as (ox, oy, oz, cnx, cny, cnz): origin and size of Omega_R
inside the box, x fastest like the boxes of the solver; None is the whole box.

Only tests/, the package's smoke check and bench.py may use this module.
"""

import numpy as np

CONVS = [(4, 16, 1), (16, 32, 2), (32, 64, 2), (64, 64, 1)]  # (ci, co, stride)
FCS = [(64, 128), (128, 21)]
NCH = 3
NOUT = 21


def layer_shapes():
    """[(name, shape)] of the flat parameter vector, in order."""
    out = []
    for i, (ci, co, _) in enumerate(CONVS):
        out += [("conv%d.w" % (i + 1), (27, ci, co)), ("conv%d.b" % (i + 1), (co,))]
    for i, (a, b) in enumerate(FCS):
        out += [("fc%d.w" % (i + 1), (a, b)), ("fc%d.b" % (i + 1), (b,))]
    return out


def n_params() -> int:
    return int(sum(np.prod(s) for _, s in layer_shapes()))


def unflatten(theta):
    theta = np.asarray(theta, dtype=np.float64)
    p, o = {}, 0
    for name, shape in layer_shapes():
        n = int(np.prod(shape))
        p[name] = theta[o:o + n].reshape(shape)
        o += n
    assert o == theta.size
    return p


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in layer_shapes()])


def one_hot(labels: np.ndarray) -> np.ndarray:
    """(D, H, W) uint8 labels -> (3, D, H, W) one-hot (labels >= 3 give a zero vector)."""
    lab = np.asarray(labels)
    return np.stack([(lab == c).astype(np.float64) for c in range(NCH)])


def core_mask(shape, core=None) -> np.ndarray:
    """(D, H, W) mask: 1 on the core Omega_R = (ox, oy, oz, cnx, cny, cnz), 0 on
    the buffer (all ones when core is None)."""
    m = np.zeros(shape)
    if core is None:
        m[...] = 1.0
    else:
        ox, oy, oz, cx, cy, cz = (int(v) for v in core)
        m[oz:oz + cz, oy:oy + cy, ox:ox + cx] = 1.0
    return m


def net_input(labels, core=None) -> np.ndarray:
    """(4, D, H, W): the one-hot labels and the core mask."""
    lab = np.asarray(labels)
    return np.concatenate([one_hot(lab), core_mask(lab.shape, core)[None]])


def out_size(n: int, stride: int) -> int:
    return (n + 2 - 3) // stride + 1


def _tap_slices(n_out, stride):
    """For each kernel offset k = 0, 1, 2: the slice of the zero-padded input
    that output index o reads (input index o * stride + k - 1, padded + 1)."""
    return [slice(k, k + stride * (n_out - 1) + 1, stride) for k in range(3)]


def conv3d(x, w, b, stride):
    """Cross-correlation with zero padding 1: y[o, d] = b[o] + sum over taps and
    input channels of w[tap, c, o] x[c, d * stride + t - 1]. x (Ci, D, H, W)."""
    ci, D, H, W = x.shape
    Do, Ho, Wo = out_size(D, stride), out_size(H, stride), out_size(W, stride)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    sz, sy, sx = _tap_slices(Do, stride), _tap_slices(Ho, stride), _tap_slices(Wo, stride)
    y = np.broadcast_to(b[:, None, None, None], (w.shape[2], Do, Ho, Wo)).copy()
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                tap = (kz * 3 + ky) * 3 + kx
                y += np.einsum("co,cdhw->odhw", w[tap], xp[:, sz[kz], sy[ky], sx[kx]])
    return y


def conv3d_backward(x, w, stride, dy):
    """Gradients of conv3d with respect to x, w and b for output gradient dy."""
    ci, D, H, W = x.shape
    _, Do, Ho, Wo = dy.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    sz, sy, sx = _tap_slices(Do, stride), _tap_slices(Ho, stride), _tap_slices(Wo, stride)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                tap = (kz * 3 + ky) * 3 + kx
                sl = (slice(None), sz[kz], sy[ky], sx[kx])
                dw[tap] = np.einsum("cdhw,odhw->co", xp[sl], dy)
                dxp[sl] += np.einsum("co,odhw->cdhw", w[tap], dy)
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, dy.sum(axis=(1, 2, 3))


def relu(a):
    return np.maximum(a, 0.0)


def forward(theta, labels, core=None):
    """Network output (21,) for one subimage (with its core), and the
    activations for backward."""
    p = unflatten(theta)
    acts = [net_input(labels, core)]
    for i, (_, _, s) in enumerate(CONVS):
        acts.append(relu(conv3d(acts[-1], p["conv%d.w" % (i + 1)], p["conv%d.b" % (i + 1)], s)))
    h0 = acts[-1].mean(axis=(1, 2, 3))
    h1 = relu(h0 @ p["fc1.w"] + p["fc1.b"])
    out = h1 @ p["fc2.w"] + p["fc2.b"]
    return out, dict(acts=acts, h0=h0, h1=h1)


def backward(theta, cache, dout):
    """Gradient of the flat parameters for output gradient dout (21,)."""
    p = unflatten(theta)
    g = {}
    h0, h1, acts = cache["h0"], cache["h1"], cache["acts"]
    g["fc2.w"] = np.outer(h1, dout)
    g["fc2.b"] = dout.copy()
    dh1 = (p["fc2.w"] @ dout) * (h1 > 0)
    g["fc1.w"] = np.outer(h0, dh1)
    g["fc1.b"] = dh1
    dh0 = p["fc1.w"] @ dh1
    a = acts[-1]
    dy = np.broadcast_to(dh0[:, None, None, None] / np.prod(a.shape[1:]), a.shape) * (a > 0)
    for i in range(len(CONVS) - 1, -1, -1):
        s = CONVS[i][2]
        dx, dw, db = conv3d_backward(acts[i], p["conv%d.w" % (i + 1)], s, dy)
        g["conv%d.w" % (i + 1)] = dw
        g["conv%d.b" % (i + 1)] = db
        if i > 0:
            dy = dx * (acts[i] > 0)
    return flatten(g)


def batch_loss_and_grad(theta, labels_batch, targets, cores=None):
    """Mean squared error over the batch and the 21 outputs, and its gradient."""
    B = len(labels_batch)
    loss = 0.0
    grad = np.zeros(n_params())
    outs = []
    for i, (lab, t) in enumerate(zip(labels_batch, targets)):
        out, cache = forward(theta, lab, None if cores is None else cores[i])
        outs.append(out)
        r = out - np.asarray(t, dtype=np.float64)
        loss += float(r @ r)
        grad += backward(theta, cache, 2.0 * r / (B * NOUT))
    return loss / (B * NOUT), grad, np.array(outs)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) with bias correction; t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def cosine_step_size(lr, step, total_steps):
    """Step size of update `step` (counted from 0) of a run of `total_steps`
    updates: the base rate lr decayed along half a cosine period,
    lr (1 + cos(pi step / total_steps)) / 2 (lr at the first update, lr / 2
    half way, approaching 0 at the end)."""
    return 0.5 * lr * (1.0 + np.cos(np.pi * step / total_steps))


def train_full_batch(theta, labels_batch, targets, steps, lr, cores=None):
    """`steps` Adam updates, each on the gradient of the whole batch, with the
    cosine step size: update t (from 0) uses cosine_step_size(lr, t, steps)
    and Adam's bias correction at t + 1. Returns the final parameters and the
    batch loss before each update."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t in range(steps):
        loss, g, _ = batch_loss_and_grad(theta, labels_batch, targets, cores)
        losses.append(loss)
        theta, m, v = adam_step(theta, g, m, v, t + 1, cosine_step_size(lr, t, steps))
    return theta, np.array(losses)


def init_params(uniform01: np.ndarray) -> np.ndarray:
    """He-uniform initial weights from uniform draws in [0, 1) (one per
    parameter, supplied by the caller's seeded generator); biases zero."""
    u = np.asarray(uniform01, dtype=np.float64)
    assert u.size == n_params()
    theta = np.zeros(n_params())
    o = 0
    for name, shape in layer_shapes():
        n = int(np.prod(shape))
        if name.endswith(".w"):
            fan_in = int(np.prod(shape[:-1]))
            bound = np.sqrt(6.0 / fan_in)
            theta[o:o + n] = (2.0 * u[o:o + n] - 1.0) * bound
        o += n
    return theta


# --------------------------------------------------------------------------
# Gate: accept the ensemble's prediction or defer to the FFT solver.
# --------------------------------------------------------------------------

def c21_to_full(c21):
    C = np.zeros((6, 6))
    iu = np.triu_indices(6)
    C[iu] = c21
    C.T[iu] = c21
    return C


def moduli_voigt(C):
    K = (C[0, 0] + C[1, 1] + C[2, 2] + 2.0 * (C[0, 1] + C[0, 2] + C[1, 2])) / 9.0
    G = (C[0, 0] + C[1, 1] + C[2, 2] - (C[0, 1] + C[0, 2] + C[1, 2]) + 3.0 * (C[3, 3] + C[4, 4] + C[5, 5])) / 15.0
    return K, G


def phase_bounds(labels, phases, core=None):
    """Voigt (arithmetic) and Reuss (harmonic) means of the phase K and G over
    the core of the subimage (the whole subimage when core is None):
    (K_R, K_V, G_R, G_V)."""
    lab = np.asarray(labels)
    if core is not None:
        ox, oy, oz, cx, cy, cz = (int(v) for v in core)
        lab = lab[oz:oz + cz, oy:oy + cy, ox:ox + cx]
    lab = lab.ravel()
    ph = np.asarray(phases, dtype=np.float64)
    f = np.bincount(lab, minlength=len(ph)).astype(np.float64) / lab.size
    K, G = ph[:, 0], ph[:, 1]
    return 1.0 / np.sum(f / K), float(np.sum(f * K)), 1.0 / np.sum(f / G), float(np.sum(f * G))


def gate(members_c21, labels, phases, spread, core=None):
    """Accept (True, mean C21) when every member's Voigt-projected K and G lie in
    the [Reuss, Voigt] bounds of the core's own phase fractions, the relative
    spread (max - min) / mean of the members' K and of their G is <= spread,
    and the mean stiffness is positive definite; else (False, mean C21)."""
    mem = np.asarray(members_c21, dtype=np.float64)
    KR, KV, GR, GV = phase_bounds(labels, phases, core)
    Ks, Gs = zip(*[moduli_voigt(c21_to_full(c)) for c in mem])
    Ks, Gs = np.array(Ks), np.array(Gs)
    mean = mem.mean(axis=0)
    ok = bool(np.all((Ks >= KR) & (Ks <= KV) & (Gs >= GR) & (Gs <= GV)))
    ok = ok and (Ks.max() - Ks.min()) <= spread * Ks.mean() and (Gs.max() - Gs.min()) <= spread * Gs.mean()
    ok = ok and bool(np.linalg.eigvalsh(c21_to_full(mean)).min() > 0.0)
    return ok, mean
