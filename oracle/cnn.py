"""FP64 NumPy forward/backward of the solver's U-Net (test infrastructure only).

The network supplies the learned initial guess and coarse interface fields of
the solve (an addition to the paper's method, which has no learned part).  It
is a 4-level U-Net on the node grid, every convolution 3x3 with zero padding
and bias, followed by ReLU:

  e0 = conv(conv(x)),            C0 channels, full resolution
  e1 = conv(conv(pool(e0))),     C1, 1/2
  e2 = conv(conv(pool(e1))),     C2, 1/4
  e3 = conv(conv(pool(e2))),     C3, 1/8
  d2 = conv([up(e3), e2])        C2
  d1 = conv([up(d2), e1])        C1
  d0 = conv([up(d1), e0])        C0
  y  = head(d0)                  1x1 convolution, no activation

pool = 2x2 average, up = 2x nearest-neighbour, [a, b] = channel concatenation.
Parameters are packed layer by layer as (weights [Cout, Cin, kh, kw], bias
[Cout]) in the order e0a e0b e1a e1b e2a e2b e3a e3b d2 d1 d0 head.  Loss is
0.5 * mean over all output entries of (y - target)^2.
"""
import numpy as np


def layer_shapes(in_ch, out_ch, C=(16, 32, 48, 64)):
    c0, c1, c2, c3 = C
    convs = [(c0, in_ch), (c0, c0), (c1, c0), (c1, c1), (c2, c1), (c2, c2), (c3, c2), (c3, c3),
             (c2, c3 + c2), (c1, c2 + c1), (c0, c1 + c0)]
    shapes = [(co, ci, 3, 3) for co, ci in convs] + [(out_ch, c0, 1, 1)]
    return shapes


def num_params(in_ch, out_ch, C=(16, 32, 48, 64)):
    return sum(int(np.prod(s)) + s[0] for s in layer_shapes(in_ch, out_ch, C))


def unpack(theta, in_ch, out_ch, C=(16, 32, 48, 64)):
    layers, off = [], 0
    for s in layer_shapes(in_ch, out_ch, C):
        n = int(np.prod(s))
        W = theta[off:off + n].reshape(s)
        off += n
        b = theta[off:off + s[0]]
        off += s[0]
        layers.append((W, b))
    return layers


def conv(x, W, b):
    """x [N, Ci, H, W], W [Co, Ci, k, k] (k = 1 or 3, zero padding k//2)."""
    k = W.shape[2]
    p = k // 2
    N, Ci, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    y = np.zeros((N, W.shape[0], H, Wd))
    for dy in range(k):
        for dx in range(k):
            y += np.einsum("oc,nchw->nohw", W[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + Wd])
    return y + b[None, :, None, None]


def conv_backward(x, W, gy):
    """Gradients of conv with respect to x, W and b."""
    k = W.shape[2]
    p = k // 2
    N, Ci, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(k):
        for dx in range(k):
            gW[:, :, dy, dx] = np.einsum("nohw,nchw->oc", gy, xp[:, :, dy:dy + H, dx:dx + Wd])
            gxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("oc,nohw->nchw", W[:, :, dy, dx], gy)
    gx = gxp[:, :, p:p + H, p:p + Wd]
    return gx, gW, gy.sum(axis=(0, 2, 3))


def pool(x):
    N, C, H, W = x.shape
    return x.reshape(N, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=2), 2, axis=3) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_backward(gy):
    N, C, H, W = gy.shape
    return gy.reshape(N, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(theta, x, out_ch, C=(16, 32, 48, 64), keep=False):
    L = unpack(theta, x.shape[1], out_ch, C)
    acts = {}

    def cr(name, inp, i):
        z = conv(inp, *L[i])
        a = np.maximum(z, 0.0)
        acts[name] = (inp, z)
        return a

    e0 = cr("e0b", cr("e0a", x, 0), 1)
    e1 = cr("e1b", cr("e1a", pool(e0), 2), 3)
    e2 = cr("e2b", cr("e2a", pool(e1), 4), 5)
    e3 = cr("e3b", cr("e3a", pool(e2), 6), 7)
    d2 = cr("d2", np.concatenate([up(e3), e2], axis=1), 8)
    d1 = cr("d1", np.concatenate([up(d2), e1], axis=1), 9)
    d0 = cr("d0", np.concatenate([up(d1), e0], axis=1), 10)
    y = conv(d0, *L[11])
    acts["head"] = (d0, y)
    return (y, acts, L) if keep else y


def loss_and_grad(theta, x, target, C=(16, 32, 48, 64)):
    """0.5 mean((y - t)^2) and its gradient with respect to theta."""
    out_ch = target.shape[1]
    y, acts, L = forward(theta, x, out_ch, C, keep=True)
    diff = y - target
    loss = 0.5 * np.mean(diff ** 2)
    gy = diff / diff.size
    grads = [None] * len(L)

    def back_conv(name, i, g_out, relu=True):
        inp, z = acts[name]
        g = g_out * (z > 0) if relu else g_out
        gx, gW, gb = conv_backward(inp, L[i][0], g)
        grads[i] = (gW, gb)
        return gx

    g = back_conv("head", 11, gy, relu=False)
    c0, c1, c2, c3 = C
    gcat = back_conv("d0", 10, g)
    g_e0 = gcat[:, c1:]
    g = up_backward(gcat[:, :c1])
    gcat = back_conv("d1", 9, g)
    g_e1 = gcat[:, c2:]
    g = up_backward(gcat[:, :c2])
    gcat = back_conv("d2", 8, g)
    g_e2 = gcat[:, c3:]
    g = up_backward(gcat[:, :c3])
    g = back_conv("e3a", 6, back_conv("e3b", 7, g))
    g = g_e2 + pool_backward(g)
    g = back_conv("e2a", 4, back_conv("e2b", 5, g))
    g = g_e1 + pool_backward(g)
    g = back_conv("e1a", 2, back_conv("e1b", 3, g))
    g = g_e0 + pool_backward(g)
    back_conv("e0a", 0, back_conv("e0b", 1, g))
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba) with bias correction; t counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
