"""Per-patch convolutional network and its training step (oracle; test
infrastructure only).

The learned right preconditioner has no counterpart in the paper (which uses
Jacobi preconditioning, Sec. 4 item 3).  Its definition here:

* A complex vector of the spline space S_{p,m} is, patch by patch, an image
  with two channels (real and imaginary part) of n1 x n1 pixels; pixel (jv, ju)
  of patch k holds dof k * n1^2 + jv * n1 + ju.
* The network has four 3 x 3 convolutions with zero padding, channels
  2 -> C -> C -> C -> 2, and ReLU after the first three:
      out[b, o, y, x] = bias[o] + sum_{c, dy, dx} W[o, c, dy, dx] in[b, c, y + dy - 1, x + dx - 1].
* Parameters are stored flat, layer by layer: W[cout][cin][3][3], then bias[cout].
* Loss of a batch of B images: L = 1 / (2B) * sum (out - target)^2.
* Adam (Kingma and Ba 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and
  bias-corrected moments.

Everything is FP64, with the convolution as an explicit sum over the nine
taps.  Pinned by: central finite differences of the loss against the gradient;
a one-channel convolution equals scipy.signal.correlate2d ('same', zero
fill); the response to a unit impulse is the flipped kernel
(tests/test_oracle_cnn.py).
"""
import numpy as np


def layer_channels(C):
    return [(2, C), (C, C), (C, C), (C, 2)]


def n_params(C):
    return sum(co * ci * 9 + co for ci, co in layer_channels(C))


def unpack(params, C):
    """List of (W [cout, cin, 3, 3], bias [cout]) views into the flat vector."""
    out, off = [], 0
    for ci, co in layer_channels(C):
        W = params[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = params[off:off + co]
        off += co
        out.append((W, b))
    return out


def conv3x3(x, W, b):
    """x [B, Cin, H, W] -> [B, Cout, H, W], zero padding."""
    B, _, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((B, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + Wd])
    return out + b[None, :, None, None]


def forward(params, x, C, keep=False):
    """Network output; with keep=True also the list of layer inputs and
    pre-activations."""
    layers = unpack(params, C)
    acts, pres = [x], []
    h = x
    for l, (W, b) in enumerate(layers):
        z = conv3x3(h, W, b)
        pres.append(z)
        h = np.maximum(z, 0.0) if l + 1 < len(layers) else z
        acts.append(h)
    return (h, acts, pres) if keep else h


def backward(params, acts, pres, gout, C):
    """dL/dparams (flat) given dL/d(network output) = gout and the layer inputs
    and pre-activations of ``forward(..., keep=True)``."""
    g = gout
    layers = unpack(params, C)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        if l + 1 < len(layers):
            g = g * (pres[l] > 0.0)              # through the ReLU
        W, _ = layers[l]
        inp = acts[l]
        H, Wd = inp.shape[2], inp.shape[3]
        ip = np.pad(inp, ((0, 0), (0, 0), (1, 1), (1, 1)))
        gW = np.zeros_like(W)
        for dy in range(3):
            for dx in range(3):
                gW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", g, ip[:, :, dy:dy + H, dx:dx + Wd])
        gb = g.sum(axis=(0, 2, 3))
        grads[l] = (gW, gb)
        if l > 0:
            # d in[b, c, y', x'] = sum_{o, dy, dx} W[o, c, dy, dx] g[b, o, y' - dy + 1, x' - dx + 1]
            gp = np.pad(g, ((0, 0), (0, 0), (1, 1), (1, 1)))
            gin = np.zeros_like(inp)
            for dy in range(3):
                for dx in range(3):
                    gin += np.einsum("oc,bohw->bchw", W[:, :, dy, dx],
                                     gp[:, :, 2 - dy:2 - dy + H, 2 - dx:2 - dx + Wd])
            g = gin
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def loss_and_grad(params, x, target, C):
    """L = 1/(2B) sum (net(x) - target)^2 and dL/dparams (flat, same layout)."""
    B = x.shape[0]
    out, acts, pres = forward(params, x, C, keep=True)
    d = out - target
    loss = 0.5 * np.sum(d * d) / B
    return loss, backward(params, acts, pres, d / B, C)


class Adam:
    def __init__(self, n, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, params, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return params - self.lr * mh / (np.sqrt(vh) + self.eps)


def vector_to_images(v, n1):
    """Complex vector [npatch * n1^2] -> images [npatch, 2, n1, n1]."""
    g = v.reshape(-1, n1, n1)
    return np.stack((g.real, g.imag), axis=1)


def images_to_vector(img):
    return (img[:, 0] + 1j * img[:, 1]).reshape(-1)
