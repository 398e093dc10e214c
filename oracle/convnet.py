"""FP64 oracle of the learned initial-guess network (test infrastructure
only; see the package docstring).

The paper couples trained networks with its physics solvers only as a
motivation (Sec. 1 (iii), Sec. 5 items (3) and (4)); the network itself is
the workload's definition: a bias-free 3D U-Net with 16 channels and three
resolutions.  Everything here is plain numpy in float64:

* ``conv3d``: 3x3x3 cross-correlation with zero padding (the convention of
  Eq. define_convolution), arrays ``[C, Z, Y, X]``, weights ``[27, Cin, Cout]``
  with tap t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1).
* ``forward``: e1 = R(W1 x), e1 = R(W2 e1); e2 = R(W3 P e1), e2 = R(W4 e2);
  e3 = R(W5 P e2), e3 = R(W6 e3); d2 = R(W7 (U e3 + e2)); d1 = R(W8 (U d2 + e1));
  y = W9 d1 -- R = ReLU, P = 2x2x2 average, U = nearest (copy) upsampling.
  No biases, so the network is positively homogeneous: f(c x) = c f(x).
* ``backward``: the analytic gradient of 0.5 * mean((y - t)^2), checked
  against finite differences in the tests.
* ``adam``: Kingma & Ba's update (beta1 0.9, beta2 0.999, eps 1e-8).
* ``bf16_round`` and the ``rnd`` argument of ``forward`` / ``backward``:
  the same arithmetic with every stored tensor rounded to bfloat16, the
  storage format the workload fixes for the network's activations (BF16
  weights and activations, FP32 accumulation); the weight gradients and
  all arithmetic stay float64.
* ``residual_loss``: the warm-start objective.  The solve that follows
  stops on ||b - A x|| / ||b||, so a guess is worth what its residual is
  worth: 0.5 * sum over interior fluid cells of (A_crop y - b)^2 / size,
  with A_crop the 7-point pressure operator of the crop (spacing h; links
  only between fluid cells inside the crop).  On cells whose six neighbours
  all lie inside the crop it equals the full grid's operator.
"""
import numpy as np

NLAYERS = 9
LAYER_IO = [(2, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 1)]


def tap_offsets():
    """(dz, dy, dx) of tap t, t = (dz+1)*9 + (dy+1)*3 + (dx+1)."""
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(x, dz, dy, dx):
    """x[:, z+dz, y+dy, x+dx] with zeros outside (zero padding)."""
    out = np.zeros_like(x)
    C, Z, Y, X = x.shape
    zs, ys, xs = slice(max(0, -dz), Z - max(0, dz)), slice(max(0, -dy), Y - max(0, dy)), slice(max(0, -dx), X - max(0, dx))
    zs2, ys2, xs2 = slice(max(0, dz), Z + min(0, dz)), slice(max(0, dy), Y + min(0, dy)), slice(max(0, dx), X + min(0, dx))
    out[:, zs, ys, xs] = x[:, zs2, ys2, xs2]
    return out


def conv3d(x, w):
    """y[co] = sum_t sum_ci w[t, ci, co] * x[ci] shifted by tap t."""
    y = np.zeros((w.shape[2],) + x.shape[1:])
    for t, (dz, dy, dx) in enumerate(tap_offsets()):
        xs = shifted(x, dz, dy, dx)
        y += np.einsum("czyx,cd->dzyx", xs, w[t])
    return y


def conv3d_dgrad(g, w):
    """Gradient of conv3d with respect to its input: correlation of g with
    the transposed weights at the mirrored taps."""
    gx = np.zeros((w.shape[1],) + g.shape[1:])
    for t, (dz, dy, dx) in enumerate(tap_offsets()):
        gs = shifted(g, -dz, -dy, -dx)
        gx += np.einsum("dzyx,cd->czyx", gs, w[t])
    return gx


def conv3d_wgrad(x, g):
    """Gradient of conv3d with respect to its weights."""
    dw = np.zeros((27, x.shape[0], g.shape[0]))
    for t, (dz, dy, dx) in enumerate(tap_offsets()):
        xs = shifted(x, dz, dy, dx)
        dw[t] = np.einsum("czyx,dzyx->cd", xs, g)
    return dw


def pool(x):
    C, Z, Y, X = x.shape
    return x.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(2, 4, 6))


def pool_bwd(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_bwd(g):
    C, Z, Y, X = g.shape
    return g.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(a):
    """The value of float array ``a`` stored as bfloat16: rounded to float32,
    then to the nearest bfloat16 (8 significant bits, ties to the even
    significand), returned as float64.  bfloat16 is the upper half of a
    float32, so rounding adds half an ulp of the lower half (plus the
    tie-breaking bit) and clears it.  Inf/NaN are not expected here."""
    u = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _identity(a):
    return a


def forward(W, x, rnd=None):
    """Returns (y, cache).  ``rnd`` (default: none) rounds every tensor the
    way a storage format would, at the points where an implementation that
    keeps its activations in that format stores them: the input, each
    activation after its ReLU, each pooled and each upsampled-plus-skip
    tensor; the output y is rounded to float32 when ``rnd`` is given.  The
    pre-activations a_k stay as computed (they decide the ReLU masks)."""
    r = rnd or _identity
    c = {"x": r(x)}
    c["a1"] = conv3d(c["x"], W[0]); c["e1a"] = r(relu(c["a1"]))
    c["a2"] = conv3d(c["e1a"], W[1]); c["e1"] = r(relu(c["a2"]))
    c["p1"] = r(pool(c["e1"]))
    c["a3"] = conv3d(c["p1"], W[2]); c["e2a"] = r(relu(c["a3"]))
    c["a4"] = conv3d(c["e2a"], W[3]); c["e2"] = r(relu(c["a4"]))
    c["p2"] = r(pool(c["e2"]))
    c["a5"] = conv3d(c["p2"], W[4]); c["e3a"] = r(relu(c["a5"]))
    c["a6"] = conv3d(c["e3a"], W[5]); c["e3"] = r(relu(c["a6"]))
    c["s2"] = r(up(c["e3"]) + c["e2"])
    c["a7"] = conv3d(c["s2"], W[6]); c["d2"] = r(relu(c["a7"]))
    c["s1"] = r(up(c["d2"]) + c["e1"])
    c["a8"] = conv3d(c["s1"], W[7]); c["d1"] = r(relu(c["a8"]))
    y = conv3d(c["d1"], W[8])
    if rnd is not None:
        y = y.astype(np.float32).astype(np.float64)
    return y, c


def loss(y, t):
    """0.5 * mean((y - t)^2) over all output entries."""
    return 0.5 * float(np.mean((y - t) ** 2))


def backward(W, c, y, t, rnd=None):
    """Gradients of ``loss(forward(W, x), t)`` with respect to every W[k]."""
    return backward_from(W, c, (y - t) / y.size, rnd)


def backward_from(W, c, g, rnd=None):
    """Gradients of a loss with respect to every W[k], given its gradient
    ``g`` with respect to the network output y ([1, Z, Y, X]).  ``rnd``
    (default: none) rounds the output gradient and every gradient tensor
    an implementation would store (after each data gradient with its ReLU
    mask, and the data gradients that feed a skip or a pooling branch), as
    in ``forward``; the weight gradients themselves are exact sums."""
    r = rnd or _identity
    dW = [None] * NLAYERS
    g = r(g)
    dW[8] = conv3d_wgrad(c["d1"], g)
    g = r(conv3d_dgrad(g, W[8]) * (c["a8"] > 0))
    dW[7] = conv3d_wgrad(c["s1"], g)
    g_s1 = r(conv3d_dgrad(g, W[7]))
    g_e1 = g_s1.copy()
    g = r(up_bwd(g_s1) * (c["a7"] > 0))
    dW[6] = conv3d_wgrad(c["s2"], g)
    g_s2 = r(conv3d_dgrad(g, W[6]))
    g_e2 = g_s2.copy()
    g = r(up_bwd(g_s2) * (c["a6"] > 0))
    dW[5] = conv3d_wgrad(c["e3a"], g)
    g = r(conv3d_dgrad(g, W[5]) * (c["a5"] > 0))
    dW[4] = conv3d_wgrad(c["p2"], g)
    g_e2 = g_e2 + pool_bwd(r(conv3d_dgrad(g, W[4])))
    g = r(g_e2 * (c["a4"] > 0))
    dW[3] = conv3d_wgrad(c["e2a"], g)
    g = r(conv3d_dgrad(g, W[3]) * (c["a3"] > 0))
    dW[2] = conv3d_wgrad(c["p1"], g)
    g_e1 = g_e1 + pool_bwd(r(conv3d_dgrad(g, W[2])))
    g = r(g_e1 * (c["a2"] > 0))
    dW[1] = conv3d_wgrad(c["e1a"], g)
    g = r(conv3d_dgrad(g, W[1]) * (c["a1"] > 0))
    dW[0] = conv3d_wgrad(c["x"], g)
    return dW


class Adam:
    def __init__(self, W, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(w) for w in W]
        self.v = [np.zeros_like(w) for w in W]
        self.t = 0

    def step(self, W, dW):
        self.t += 1
        out = []
        for k, (w, g) in enumerate(zip(W, dW)):
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g * g
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            out.append(w - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out


def rms_or_one(a):
    r = float(np.sqrt(np.mean(a * a)))
    return r if r > 0 else 1.0


def net_input(b, p):
    """The network's input: (b / rms(b), p^n / rms(p^n)) -> [2, Z, Y, X];
    returns (x, rms(b)).  The output is multiplied back by rms(b), so the
    guess is positively homogeneous in b (as the solution of A dp = b is
    linear in b) while p^n enters by its shape only (its scale relative to
    b spans orders of magnitude between flows and time steps)."""
    rb, rp = rms_or_one(b), rms_or_one(p)
    return np.stack([b / rb, p / rp]), rb


def crop_operator(v, fluid, h=1.0):
    """(A_crop v)_c = (1/h^2) sum over fluid face neighbours n inside the
    array of (v_c - v_n), on fluid cells c; 0 on solid cells.  v, fluid:
    [Z, Y, X] (fluid boolean)."""
    fl = np.asarray(fluid, bool)
    out = np.zeros_like(v, dtype=np.float64)
    Z, Y, X = v.shape
    for axis in range(3):
        n = v.shape[axis]
        for d in (-1, 1):
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            dst[axis] = slice(max(0, -d), n - max(0, d))
            src[axis] = slice(max(0, d), n + min(0, d))
            both = fl[tuple(dst)] & fl[tuple(src)]
            out[tuple(dst)] += both * (v[tuple(dst)] - v[tuple(src)])
    return out * fl / (h * h)


def interior(shape):
    """Cells whose six face neighbours all lie inside the array."""
    m = np.zeros(shape, bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def residual_loss(y, b, fluid, h=1.0):
    """(loss, dloss/dy) of 0.5 * sum_{interior fluid} (A_crop y - b)^2 / size
    for one sample; y, b: [Z, Y, X]."""
    w = interior(y.shape) & np.asarray(fluid, bool)
    r = (crop_operator(y, fluid, h) - b) * w
    loss = 0.5 * float(np.sum(r * r)) / y.size
    # A_crop is symmetric, so the gradient is A_crop applied to the masked
    # residual
    return loss, crop_operator(r, fluid, h) / y.size
