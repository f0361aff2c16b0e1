"""FP64 reference of the warm-start network (test infrastructure only).

The paper has no network; this module is the plain definition the GPU
network is checked against:
  * layers l = 0 .. L-1, H_{l+1} = relu(H_l W_l^T + b_l) for the hidden layers,
    Y = H_{L-1} W_{L-1}^T + b_{L-1} for the output (W_l: d_{l+1} x d_l);
  * loss = mean over the batch and the outputs of (Y - T)^2;
  * gradients by the chain rule (backpropagation), written out layer by layer;
  * Adam, Kingma and Ba (2015), Algorithm 1, with bias-corrected moments.
"""
import numpy as np


def glorot_uniform(rng, dims):
    """Weights U(-a, a), a = sqrt(6 / (d_in + d_out)); zero biases."""
    params = []
    for din, dout in zip(dims[:-1], dims[1:]):
        a = np.sqrt(6.0 / (din + dout))
        params.append((rng.uniform(-a, a, size=(dout, din)), np.zeros(dout)))
    return params


def forward(params, X):
    """Returns the output and the list of layer inputs H_0 = X, H_1, ..."""
    H = np.asarray(X, dtype=np.float64)
    inputs = [H]
    for l, (W, b) in enumerate(params):
        Z = H @ W.T + b
        if l + 1 < len(params):
            H = np.maximum(Z, 0.0)
            inputs.append(H)
        else:
            H = Z
    return H, inputs


def loss(params, X, T):
    Y, _ = forward(params, X)
    return float(np.mean((Y - T) ** 2))


def gradients(params, X, T):
    """(loss, [(dW_l, db_l)]) of the mean squared error."""
    Y, inputs = forward(params, X)
    B, out = Y.shape
    G = 2.0 * (Y - T) / (B * out)          # d loss / d Y
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        H = inputs[l]
        grads[l] = (G.T @ H, G.sum(axis=0))
        if l > 0:
            G = (G @ W) * (H > 0)          # through the ReLU of layer l - 1
    return float(np.mean((Y - T) ** 2)), grads


class Adam:
    """Adam state for a parameter list."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for k, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[l][k] + (1.0 - self.b1) * g
                v = self.b2 * self.v[l][k] + (1.0 - self.b2) * g * g
                new.append((p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps), m, v))
            out.append((new[0][0], new[1][0]))
            self.m[l] = (new[0][1], new[1][1])
            self.v[l] = (new[0][2], new[1][2])
        return out
