"""Plain FP64 definitions of the learned convergence accelerator (numpy).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the CUDA library or its binding.  The
paper has no learned component; this is the accelerator the project adds around its explicit
pseudo-time iteration (Sec. 2.3's convergence loop): a 3-layer 3D convolutional network reads
the current state and residual and predicts the state change over K = 20 pseudo-time steps, and
the prediction is kept only if the residual norm then drops.

Definitions (written out, no blocking or fusion):
  conv3d      y[o](p) = b[o] + sum_c sum_t W[o][c][t] x[c](p + d_t), d_t = (dz, dy, dx) in
              {-1,0,1}^3, tap t = 9 (dz+1) + 3 (dy+1) + (dx+1); x is zero outside the volume in
              x and y, periodic in z when zper (the channel is periodic in z)
  network     z1 = conv(x; W1, b1), a1 = silu(z1), z2 = conv(a1; W2, b2), a2 = silu(z2),
              y = conv(a2; W3, b3); channels 10 -> 32 -> 32 -> 5; silu(z) = z / (1 + e^-z)
  precision   the GPU path stores x, a1, a2 and the weights in bfloat16 and accumulates in FP32;
              forward(..., bf16=True) rounds the same tensors to bfloat16 (round to nearest even)
              and computes everything else in FP64
  loss        mean over cells and the 5 output channels of (y - target)^2
  adam        Kingma & Ba: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
              w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
  features    channels 0-4: 10 (Q - Q_inf) / ref, channels 5-9: (-dt_cell R) / ref / s, with
              ref = (rho_inf, rho_inf c_inf, rho_inf c_inf, rho_inf c_inf, rho_inf c_inf^2) and
              s the RMS over cells and the 5 channels of (-dt_cell R) / ref
  target      (Q_after - Q_before) / ref / (K s);  prediction: Q + K s ref y
"""
import numpy as np

K_STEPS = 20
CH = (10, 32, 32, 5)
STATE_GAIN = 10.0


def tap_offsets():
    return [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def bf16(a):
    """round to the nearest bfloat16 (ties to even), returned as float64"""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def _pad(x, zper):
    x = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    if zper:
        return np.concatenate([x[:, -1:], x, x[:, :1]], axis=1)
    return np.pad(x, ((0, 0), (1, 1), (0, 0), (0, 0)))


def conv3d(x, W, b, zper=True):
    """x [C][Z][Y][X], W [O][C][27], b [O] -> [O][Z][Y][X]"""
    C, Z, Y, X = x.shape
    xp = _pad(np.asarray(x, dtype=np.float64), zper)
    out = np.zeros((W.shape[0], Z, Y, X)) + np.asarray(b, dtype=np.float64)[:, None, None, None]
    for t, (dz, dy, dx) in enumerate(tap_offsets()):
        sl = xp[:, 1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X]
        out += np.einsum("oc,czyx->ozyx", W[:, :, t], sl)
    return out


def conv3d_transpose(g, W, zper=True):
    """adjoint of conv3d in x: [O][Z][Y][X] -> [C][Z][Y][X] (a conv3d with the taps mirrored and
    the channel roles swapped)"""
    Wt = np.transpose(W[:, :, ::-1], (1, 0, 2))
    return conv3d(g, Wt, np.zeros(Wt.shape[0]), zper)


def conv3d_weight_grad(x, g, zper=True):
    """d/dW of sum(g * conv3d(x, W, 0)): [O][C][27]"""
    C, Z, Y, X = x.shape
    xp = _pad(np.asarray(x, dtype=np.float64), zper)
    dW = np.zeros((g.shape[0], C, 27))
    for t, (dz, dy, dx) in enumerate(tap_offsets()):
        sl = xp[:, 1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X]
        dW[:, :, t] = np.einsum("ozyx,czyx->oc", g, sl)
    return dW


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def split_params(p):
    """flat parameter vector -> [(W1, b1), (W2, b2), (W3, b3)] (the library's host layout)"""
    out, o = [], 0
    for ci, co in zip(CH[:-1], CH[1:]):
        W = p[o:o + co * ci * 27].reshape(co, ci, 27)
        o += co * ci * 27
        b = p[o:o + co]
        o += co
        out.append((W, b))
    return out


def n_params():
    return sum(co * ci * 27 + co for ci, co in zip(CH[:-1], CH[1:]))


def forward(p, x, zper=True, bf16_storage=True):
    """network output and the intermediates (z1, a1, z2, a2) for the backward pass"""
    r = bf16 if bf16_storage else (lambda a: np.asarray(a, dtype=np.float64))
    (W1, b1), (W2, b2), (W3, b3) = [(r(W), np.asarray(b, dtype=np.float64)) for W, b in split_params(p)]
    a0 = r(x)
    z1 = conv3d(a0, W1, b1, zper)
    a1 = r(silu(z1))
    z2 = conv3d(a1, W2, b2, zper)
    a2 = r(silu(z2))
    y = conv3d(a2, W3, b3, zper)
    return y, (a0, z1, a1, z2, a2)


def loss_and_grad(p, x, target, zper=True, bf16_storage=True):
    """mean squared error and its gradient (flat, the layout of p); roundings are treated as the
    identity in the backward pass"""
    y, (a0, z1, a1, z2, a2) = forward(p, x, zper, bf16_storage)
    n = y.size
    d = y - target
    loss = float(np.sum(d * d) / n)
    g3 = 2.0 * d / n
    r = bf16 if bf16_storage else (lambda a: np.asarray(a, dtype=np.float64))
    (W1, _), (W2, _), (W3, _) = [(r(W), b) for W, b in split_params(p)]
    dW3, db3 = conv3d_weight_grad(a2, g3, zper), g3.sum(axis=(1, 2, 3))
    g2 = conv3d_transpose(g3, W3, zper) * dsilu(z2)
    dW2, db2 = conv3d_weight_grad(a1, g2, zper), g2.sum(axis=(1, 2, 3))
    g1 = conv3d_transpose(g2, W2, zper) * dsilu(z1)
    dW1, db1 = conv3d_weight_grad(a0, g1, zper), g1.sum(axis=(1, 2, 3))
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """one Adam step (t counts from 1); returns new (w, m, v)"""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def reference_scales(inf, gamma=1.4):
    rho, p = inf[0], inf[4]
    c = np.sqrt(gamma * p / rho)
    return np.array([rho, rho * c, rho * c, rho * c, rho * c * c])


def conserved_inf(inf, gamma=1.4):
    rho, u, v, w, p = inf
    return np.array([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def features(Q, R, dtl, inf, gamma=1.4):
    """Q, R [5][Z][Y][X] (conserved state and its residual), dtl [Z][Y][X] (each cell's pseudo-time
    step) -> (x [10][Z][Y][X], s)"""
    ref = reference_scales(inf, gamma)[:, None, None, None]
    qinf = conserved_inf(inf, gamma)[:, None, None, None]
    inc = -dtl[None] * R / ref
    s = float(np.sqrt(np.mean(inc * inc)))
    x = np.concatenate([STATE_GAIN * (Q - qinf) / ref, inc / s])
    return x, s


def target(Q_before, Q_after, s, inf, gamma=1.4):
    ref = reference_scales(inf, gamma)[:, None, None, None]
    return (Q_after - Q_before) / ref / (K_STEPS * s)


def apply_prediction(Q, y, s, inf, gamma=1.4):
    ref = reference_scales(inf, gamma)[:, None, None, None]
    return Q + K_STEPS * s * ref * y
