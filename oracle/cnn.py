"""FP64 plaintext CNN (O1) by direct loops -- the result the encrypted path
must reproduce (paper Sec. VII validation: decrypted outputs equal the plaintext
model's outputs).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Shapes: images [C][H][W] (1-D signals [C][1][W]); conv weights [co][ci][K][K]
(1-D: [co][ci][K]); average pooling c x c with stride c (1-D: c); flatten is
channel-major, row-major (index o*H*W + r*W + c); FC y = M x + b.
"""
import numpy as np


def conv(x, w, b, S):
    w = np.asarray(w, dtype=np.float64)
    if w.ndim == 3:
        w = w[:, :, None, :]
    co, ci, kh, kw = w.shape
    C, H, W = x.shape
    assert C == ci
    Ho, Wo = (H - kh) // S + 1, (W - kw) // S + 1
    y = np.zeros((co, Ho, Wo))
    for o in range(co):
        for r in range(Ho):
            for c in range(Wo):
                acc = 0.0
                for i in range(ci):
                    for j in range(kh):
                        for k in range(kw):
                            acc += w[o, i, j, k] * x[i, S * r + j, S * c + k]
                y[o, r, c] = acc + b[o]
    return y


def avgpool(x, c, dims=2):
    C, H, W = x.shape
    if dims == 1:
        Wo = W // c
        return np.stack([[x[i, 0, c * k: c * k + c].mean() for k in range(Wo)] for i in range(C)])[:, None, :]
    Ho, Wo = H // c, W // c
    y = np.zeros((C, Ho, Wo))
    for i in range(C):
        for r in range(Ho):
            for k in range(Wo):
                y[i, r, k] = x[i, c * r: c * r + c, c * k: c * k + c].mean()
    return y


def forward(x, layers, dims=2):
    """x: [H][W] or [C][H][W] (or [W] for dims=1) -> output vector."""
    x = np.asarray(x, dtype=np.float64)
    if dims == 1:
        x = x[None, None, :]
    elif x.ndim == 2:
        x = x[None, :, :]
    for spec in layers:
        op = spec["op"]
        if op in ("conv2d", "conv1d"):
            x = conv(x, spec["w"], spec["b"], spec["stride"])
        elif op == "square":
            x = x * x
        elif op == "approx_relu":   # Sec. IV-F: 0.375373 + 0.5 x + 0.117071 x^2
            x = 0.375373 + 0.5 * x + 0.117071 * x * x
        elif op == "avgpool":
            x = avgpool(x, spec["k"], dims)
        elif op == "flatten":
            x = x.reshape(-1)
        elif op == "fc":
            x = np.asarray(spec["w"], dtype=np.float64) @ x.reshape(-1) + np.asarray(spec["b"], dtype=np.float64)
        else:
            raise ValueError(op)
    return x.reshape(-1)
