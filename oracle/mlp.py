"""Per-element MLP for the learned initial guess, in plain FP64 (test infrastructure).

The paper has no learned component; this follows the build's own
definition of the learned guess of a physical time step:

  features   x_e = [U^n_e / s0, (U^n - U^{n-1})_e / s1,
                    (U^n - 2 U^{n-1} + U^{n-2})_e / s2]
             (element e, each block flattened as (variable, point), s0, s1, s2
             per-variable scales), K = 3 n_v (p+1)^d values.  This is an
             invertible linear map of the three previous levels: the network
             sees the same information, but each block is O(1) after scaling,
             so BF16 operands keep the small time differences that a BF16
             copy of the raw levels would round away;
  network    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3;
  guess      U^{n+1}_e ~ U*_e + t (.) y, with the plain extrapolation
             U* = 3 U^n - 3 U^{n-1} + U^{n-2} and per-variable output scale t;
  loss       mean over samples and outputs of (y - (U^{n+1} - U*)/t)^2;
  training   Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the full batch.

Matrices act on columns: W is (out x in), a batch is stored with samples
as columns (X is K x B), matching the element-fastest state layout.

Pins (tests/test_oracle_mlp.py): backward against central finite
differences; the blend weight of the two guesses minimises a linear
residual along the segment (brute-force scan); weight decay alone (zero gradient) shrinks the weights by the
factor 1 - lr * weight_decay per step and leaves the biases; a network built to represent a known piecewise-linear map;
Adam's first step moves every parameter by lr times the sign of its
gradient; features/targets reproduce the extrapolation identity on data
that is quadratic in time.
"""
import numpy as np


def forward(params, X):
    """params = [(W1, b1), (W2, b2), (W3, b3)]; X is K x B.  Returns (Y, cache)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    Z1 = W1 @ X + b1[:, None]
    H1 = np.maximum(Z1, 0.0)
    Z2 = W2 @ H1 + b2[:, None]
    H2 = np.maximum(Z2, 0.0)
    Y = W3 @ H2 + b3[:, None]
    return Y, (X, Z1, H1, Z2, H2)


def loss(Y, Tgt):
    return float(np.mean((Y - Tgt) ** 2))


def backward(params, cache, Y, Tgt):
    """Gradients of loss(Y, Tgt) with respect to all parameters."""
    (W1, b1), (W2, b2), (W3, b3) = params
    X, Z1, H1, Z2, H2 = cache
    dY = 2.0 * (Y - Tgt) / Y.size
    dW3 = dY @ H2.T
    db3 = dY.sum(axis=1)
    dH2 = W3.T @ dY
    dZ2 = dH2 * (Z2 > 0.0)
    dW2 = dZ2 @ H1.T
    db2 = dZ2.sum(axis=1)
    dH1 = W2.T @ dZ2
    dZ1 = dH1 * (Z1 > 0.0)
    dW1 = dZ1 @ X.T
    db1 = dZ1.sum(axis=1)
    return [(dW1, db1), (dW2, db2), (dW3, db3)]


class Adam:
    """Adam on a list of (W, b) layers; with weight_decay > 0 the decoupled
    form (AdamW, Loshchilov & Hutter): each step also subtracts
    lr * weight_decay * W from the weights (not the biases)."""

    def __init__(self, params, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.wd = weight_decay
        self.m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for i in range(len(params)):
            layer = []
            for j in range(2):
                p, g = params[i][j], grads[i][j]
                self.m[i][j] = self.b1 * self.m[i][j] + (1.0 - self.b1) * g
                self.v[i][j] = self.b2 * self.v[i][j] + (1.0 - self.b2) * g * g
                mh = self.m[i][j] / (1.0 - self.b1 ** self.t)
                vh = self.v[i][j] / (1.0 - self.b2 ** self.t)
                decay = self.wd * p if j == 0 else 0.0
                layer.append(p - self.lr * (mh / (np.sqrt(vh) + self.eps) + decay))
            out.append(tuple(layer))
        return out


def features(Un, Unm1, Unm2, scales, elems):
    """K x B feature matrix of the listed elements; states are [nv, npts, ne],
    scales = (s0, s1, s2), each of length nv."""
    blocks = (Un, Un - Unm1, Un - 2.0 * Unm1 + Unm2)
    parts = []
    for B, s in zip(blocks, scales):
        s = np.asarray(s, dtype=np.float64)[:, None, None]
        parts.append((B[:, :, elems] / s).reshape(-1, len(elems)))
    return np.concatenate(parts, axis=0)


def extrapolate(Un, Unm1, Unm2):
    return 3.0 * Un - 3.0 * Unm1 + Unm2


def targets(Unp1, Un, Unm1, Unm2, out_scale, elems):
    """(n_v npts) x B normalised corrections to the plain extrapolation."""
    t = np.asarray(out_scale, dtype=np.float64)[:, None, None]
    D = (Unp1 - extrapolate(Un, Unm1, Unm2))[:, :, elems] / t
    return D.reshape(-1, len(elems))


def apply_guess(Y, Un, Unm1, Unm2, out_scale):
    """Guess for every element from the network output Y ((n_v npts) x ne)."""
    nv, npts, ne = Un.shape
    t = np.asarray(out_scale, dtype=np.float64)[:, None, None]
    return extrapolate(Un, Unm1, Unm2) + t * Y.reshape(nv, npts, ne)


def blend_weight(r0, r1):
    """Weight alpha in [0, 1] of the network's guess on the segment from the
    extrapolation (residual r0) to the network's guess (residual r1) that
    minimises the linearised residual |r0 + alpha (r1 - r0)|_2 (the build's
    own fallback rule for the learned guess)."""
    d = np.asarray(r1, dtype=np.float64) - np.asarray(r0, dtype=np.float64)
    dd = float(np.sum(d * d))
    if dd == 0.0:
        return 0.0
    return float(np.clip(-np.sum(np.asarray(r0) * d) / dd, 0.0, 1.0))


def degree_projector(order, q):
    """1-D L2 projection onto polynomials of degree <= q, as an (m x m)
    matrix acting on values at the m = order + 1 Gauss-Legendre points:
    P[i, k] = sum_{n <= q} phi_n(x_i) phi_n(x_k) w_k with the orthonormal
    Legendre polynomials phi_n = sqrt((2n + 1) / 2) P_n (the m-point rule is
    exact for the products, degree <= 2 order).  No counterpart in the paper:
    it smooths the learned correction of the initial guess."""
    from oracle.ops1d import gauss_legendre, legendre
    x, w = gauss_legendre(order + 1)
    phi = np.stack([np.sqrt((2 * n + 1) / 2.0) * legendre(n, x)[0] for n in range(q + 1)],
                   axis=1)
    return phi @ (phi.T * w[None, :])


def project_degree(Y, order, dim, q):
    """Per-element, per-variable tensor-product projection of Y ((n_v npts) x
    B, point index i + m j + m^2 k) onto degree <= q along every axis."""
    m = order + 1
    P = degree_projector(order, q)
    B = Y.shape[1]
    Z = np.asarray(Y, dtype=np.float64).reshape((-1,) + (m,) * dim + (B,))
    # axes of Z: (v, [k,] j, i, B); the x axis (i) is the last spatial one
    for ax in range(1, dim + 1):
        Z = np.moveaxis(np.tensordot(P, Z, axes=([1], [ax])), 0, ax)
    return Z.reshape(Y.shape)

