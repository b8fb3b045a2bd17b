"""FP64 reference of the per-block refinement-proposal network (test infrastructure).

Plain NumPy, written from the network's definition; used to check the CUDA
forward and backward kernels.  Network on an input x[2][T][T]:

  h1 = relu(conv3x3(x;  W1, b1), stride 1, zero padding 1)      16 x T  x T
  h2 = relu(conv3x3(h1; W2, b2), stride 2, zero padding 1)      16 x T2 x T2
  h3 = relu(conv3x3(h2; W3, b3), stride 2, zero padding 1)      16 x T3 x T3
  z  = max over (i, j) of h3                                     16
  p  = sigmoid(wl . z + bl)

with T2 = (T - 1) // 2 + 1, T3 = (T2 - 1) // 2 + 1.  Loss of a batch: mean of
the weighted binary cross entropy -(w_pos y log p + (1 - y) log(1 - p)).
Parameters are packed in the order W1, b1, W2, b2, W3, b3, wl, bl.
"""
import numpy as np

C_IN, C = 2, 16
SHAPES = [(C, C_IN, 3, 3), (C,), (C, C, 3, 3), (C,), (C, C, 3, 3), (C,), (C,), (1,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def conv(x, W, b, stride):
    """3x3 convolution, zero padding 1: out[o,i,j] = b[o] + sum W[o,c,di,dj] x[c, s i + di - 1, s j + dj - 1]."""
    cin, T, _ = x.shape
    To = (T - 1) // stride + 1
    xp = np.zeros((cin, T + 2, T + 2))
    xp[:, 1:T + 1, 1:T + 1] = x
    out = np.zeros((W.shape[0], To, To))
    for di in range(3):
        for dj in range(3):
            patch = xp[:, di:di + stride * (To - 1) + 1:stride, dj:dj + stride * (To - 1) + 1:stride]
            out += np.einsum("oc,cij->oij", W[:, :, di, dj], patch)
    return out + b[:, None, None]


def conv_backward(x, W, stride, gout):
    """Gradients of conv(x, W, b, stride) given dL/dout: (dx, dW, db)."""
    cin, T, _ = x.shape
    To = gout.shape[1]
    xp = np.zeros((cin, T + 2, T + 2))
    xp[:, 1:T + 1, 1:T + 1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for di in range(3):
        for dj in range(3):
            sl = (slice(None), slice(di, di + stride * (To - 1) + 1, stride),
                  slice(dj, dj + stride * (To - 1) + 1, stride))
            dW[:, :, di, dj] = np.einsum("oij,cij->oc", gout, xp[sl])
            dxp[sl] += np.einsum("oc,oij->cij", W[:, :, di, dj], gout)
    return dxp[:, 1:T + 1, 1:T + 1], dW, gout.sum(axis=(1, 2))


def forward(theta, x):
    W1, b1, W2, b2, W3, b3, wl, bl = unpack(theta)
    a1 = conv(x, W1, b1, 1); h1 = np.maximum(a1, 0)
    a2 = conv(h1, W2, b2, 2); h2 = np.maximum(a2, 0)
    a3 = conv(h2, W3, b3, 2); h3 = np.maximum(a3, 0)
    z = h3.reshape(C, -1).max(axis=1)
    logit = float(wl @ z + bl[0])
    p = 1.0 / (1.0 + np.exp(-logit))
    return p, dict(a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, z=z, logit=logit)


def loss_and_grad(theta, xs, ys, w_pos):
    """Mean weighted BCE over the batch and its gradient w.r.t. theta."""
    W1, b1, W2, b2, W3, b3, wl, bl = unpack(theta)
    g = [np.zeros(s) for s in SHAPES]
    L = 0.0
    n = len(xs)
    for x, y in zip(xs, ys):
        p, c = forward(theta, x)
        L += -(w_pos * y * np.log(p) + (1 - y) * np.log(1 - p)) / n
        dlogit = (y * w_pos * (p - 1.0) + (1 - y) * p) / n
        g[6] += dlogit * c["z"]
        g[7] += dlogit
        dz = dlogit * wl
        h3 = c["h3"].reshape(C, -1)
        arg = h3.argmax(axis=1)  # first maximum
        dh3 = np.zeros_like(h3)
        dh3[np.arange(C), arg] = dz
        da3 = dh3.reshape(c["h3"].shape) * (c["a3"] > 0)
        dh2, dW3, db3 = conv_backward(c["h2"], W3, 2, da3)
        da2 = dh2 * (c["a2"] > 0)
        dh1, dW2, db2 = conv_backward(c["h1"], W2, 2, da2)
        da1 = dh1 * (c["a1"] > 0)
        _, dW1, db1 = conv_backward(x, W1, 1, da1)
        for k, d in enumerate((dW1, db1, dW2, db2, dW3, db3)):
            g[k] += d
    return L, pack(g)
