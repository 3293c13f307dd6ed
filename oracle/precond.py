"""Oracle: the block-diagonal and the learned preconditioners of the FGMRES solve.

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy; used by tests/ to check the library.

Block-diagonal preconditioner.  With B the block-diagonal part of the system matrix (blocks of
size `block` on the diagonal; one panel per block when block = 16 Mth), z = B^{-1} r blockwise.
numpy.linalg.solve is the step.

Learned preconditioner.  A 4-layer convolutional network on the (t, theta) grid of the unknowns
(unknown index t * Mth + theta, t = panel * 16 + node):
  layer l: y[b, o, t, th] = bias[o] + sum_{c, a, e} W[o, c, a, e] x[b, c, t + d (a - 1), th + d (e - 1)]
  with a, e in {0, 1, 2}, the theta index periodic (mod Mth), x = 0 outside 0 <= t < nt;
  (cin, cout, d) = (4, 32, 1), (32, 32, 2), (32, 32, 4), (32, 2, 1); ReLU after the first three.
Features of a residual r: Re r / s, Im r / s, J / mean(J), k / 25 with s = rms(r); the
preconditioner is z = B^{-1} r + s (o_0 + i o_1).
Flat parameter vector: per layer W (cout, cin, 3, 3) then bias (cout).
Training loss for residuals r_v of a system A:
  L = (1/nv) sum_v ||A z_v - r_v||^2 / ||r_v||^2.
Its gradient follows by the chain rule: dL/dz_v = (2 / (nv ||r_v||^2)) A^H (A z_v - r_v) as a
complex vector (real part: d/dRe z, imaginary part: d/dIm z), then d/do_v = s_v (Re, Im) of that,
then back through the layers (the adjoint of a layer is the same correlation with transposed
channels and mirrored taps).
"""
import numpy as np

LAYERS = [(4, 32, 1, True), (32, 32, 2, True), (32, 32, 4, True), (32, 2, 1, False)]
N_PARAMS = sum(co * ci * 9 + co for ci, co, _, _ in LAYERS)


# ----------------------------------------------------------------------------
# block-diagonal preconditioner
# ----------------------------------------------------------------------------
def block_diag_apply(A, block, r):
    """z = B^{-1} r for the block-diagonal part B of A; r [..., n]."""
    A = np.asarray(A)
    n = A.shape[0]
    r = np.asarray(r, dtype=complex)
    z = np.empty_like(r)
    for b0 in range(0, n, block):
        sl = slice(b0, b0 + block)
        z[..., sl] = np.linalg.solve(A[sl, sl], r[..., sl].T).T
    return z


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------
def bf16_round(w):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    w32 = np.asarray(w, dtype=np.float32)
    bits = w32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    """[(W, b)] per layer from the flat parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for ci, co, _, _ in LAYERS:
        W = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def _shifted(x, dt, dth):
    """s[..., t, th] = x[..., t + dt, (th + dth) mod mt], zero where t + dt is outside [0, nt)."""
    nt = x.shape[-2]
    s = np.zeros_like(x)
    lo, hi = max(0, -dt), min(nt, nt - dt)
    if lo < hi:
        s[..., lo:hi, :] = np.roll(x[..., lo + dt:hi + dt, :], -dth, axis=-1)
    return s


def conv(x, W, b, d):
    """One layer, x [B, cin, nt, mt] -> [B, cout, nt, mt] (no activation)."""
    y = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
    for a in range(3):
        for e in range(3):
            y += np.einsum("oc,bcij->boij", W[:, :, a, e], _shifted(x, d * (a - 1), d * (e - 1)))
    if b is not None:
        y += b[None, :, None, None]
    return y


def conv_adjoint(g, W, d):
    """Adjoint of conv (without bias) w.r.t. its input: g [B, cout, nt, mt] -> [B, cin, nt, mt]."""
    x = np.zeros((g.shape[0], W.shape[1]) + g.shape[2:])
    for a in range(3):
        for e in range(3):
            x += np.einsum("oc,boij->bcij", W[:, :, a, e], _shifted(g, -d * (a - 1), -d * (e - 1)))
    return x


def conv_weight_grad(x, g, d):
    """d/dW of sum(g * conv(x, W, b, d)) and d/db: ([cout, cin, 3, 3], [cout])."""
    gW = np.zeros((g.shape[1], x.shape[1], 3, 3))
    for a in range(3):
        for e in range(3):
            gW[:, :, a, e] = np.einsum("boij,bcij->oc", g, _shifted(x, d * (a - 1), d * (e - 1)))
    return gW, g.sum(axis=(0, 2, 3))


def forward(params, x):
    """Network output [B, 2, nt, mt] and the post-activation outputs of every layer."""
    acts = []
    h = np.asarray(x, dtype=np.float64)
    for (W, b), (_, _, d, relu) in zip(unpack(params), LAYERS):
        h = conv(h, W, b, d)
        if relu:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def backward(params, x, gy):
    """Gradients of sum(gy * forward(x)) w.r.t. the flat parameters and x."""
    layers = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    _, acts = forward(params, x)
    inputs = [x] + acts[:-1]
    g = np.asarray(gy, dtype=np.float64)
    grads = [None] * len(LAYERS)
    for li in range(len(LAYERS) - 1, -1, -1):
        W, _ = layers[li]
        _, _, d, relu = LAYERS[li]
        if relu:
            g = g * (acts[li] > 0)
        grads[li] = conv_weight_grad(inputs[li], g, d)
        g = conv_adjoint(g, W, d)
    return pack(grads), g


def features(r, J, k, nt, mt):
    """[nv, 4, nt, mt] features of residuals r [nv, N] and the scales s_v."""
    r = np.atleast_2d(np.asarray(r, dtype=complex))
    s = np.sqrt(np.mean(np.abs(r) ** 2, axis=1))
    u = r / s[:, None]
    nv = r.shape[0]
    f = np.empty((nv, 4, nt, mt))
    f[:, 0] = u.real.reshape(nv, nt, mt)
    f[:, 1] = u.imag.reshape(nv, nt, mt)
    f[:, 2] = (np.asarray(J) / np.mean(J)).reshape(nt, mt)
    f[:, 3] = k / 25.0
    return f, s


def precond_apply(params, r, J, k, nt, mt, zb):
    """z = zb + s (o_0 + i o_1), zb = B^{-1} r given (zeros without a block preconditioner)."""
    f, s = features(r, J, k, nt, mt)
    o, _ = forward(params, f)
    nv = f.shape[0]
    return np.asarray(zb).reshape(nv, -1) + s[:, None] * (o[:, 0] + 1j * o[:, 1]).reshape(nv, -1)


def loss_and_grad(params, A, r, J, k, nt, mt, zb):
    """Training loss of residuals r [nv, N] on system A, and its gradient w.r.t. the parameters."""
    r = np.atleast_2d(np.asarray(r, dtype=complex))
    nv = r.shape[0]
    f, s = features(r, J, k, nt, mt)
    o, _ = forward(params, f)
    z = np.asarray(zb).reshape(nv, -1) + s[:, None] * (o[:, 0] + 1j * o[:, 1]).reshape(nv, -1)
    e = z @ np.asarray(A).T - r                        # rows: A z_v - r_v
    rsq = np.sum(np.abs(r) ** 2, axis=1)
    loss = np.mean(np.sum(np.abs(e) ** 2, axis=1) / rsq)
    gz = (2.0 / (nv * rsq))[:, None] * (e @ np.conj(np.asarray(A)))   # rows: A^H e_v, scaled
    go = np.empty_like(o)
    go[:, 0] = (s[:, None] * gz.real).reshape(nv, nt, mt)
    go[:, 1] = (s[:, None] * gz.imag).reshape(nv, nt, mt)
    gp, _ = backward(params, f, go)
    return loss, gp
