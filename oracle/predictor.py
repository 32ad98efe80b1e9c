"""Learned reuse predictor for the cache of derived Gaussians: the oracle's
plain definition of its inputs, its reuse decision, its training labels and
its training (forward, backward, Adam).

TEST INFRASTRUCTURE (see oracle/__init__.py).

The paper decides reuse with the depth rule of Alg. 1 / Eq. 4 only; the
predictor is an extension of that cache (it replaces "age <= depth" by a
learned per-anchor decision, with full re-derivation as the fallback).  Its
definition here:

Inputs z (36 values) of a visible anchor a holding a valid cache line:
  z[0:32]  the anchor feature f_a (Eq. 3's feature),
  z[32:35] 1024 (dir_now - dir_line): change of the unit direction from the
           derivation camera's centre to the anchor since the line was decoded
           (the 1024 makes ~1 mrad changes ~1),
  z[35]    plog2(|x_a - p|) - 8, with plog2(m 2^e) = e + (m - 1) for m in
           [1, 2): the piecewise-linear log2 (exact at powers of two, within
           0.086 of log2), centred near 256 m.
Decision: p = sigmoid(w2 . relu(W1^T z + b1) + b2) >= 0.5, i.e. logit >= 0.
Everything that feeds this integer decision is float32 in a fixed operation
order (no fused multiply-add), with the weights rounded to bfloat16 (round to
nearest even):
  dx = (x_a - p_hi) - p_lo          (p_hi = fl32(p), p_lo = fl32(p - p_hi))
  |dx| = sqrt((dx0 dx0 + dx1 dx1) + dx2 dx2),  dir = dx / |dx|
  h_j = max(0, ((...(w[0,j] z0 + w[1,j] z1) + ...) + w[35,j] z35) + b1_j)
  logit = ((...(w2_0 h_0 + w2_1 h_1) + ...) + w2_63 h_63) + b2
so that any implementation following the same steps takes the same decision.

Label (reuse acceptable) of a candidate: the cached and freshly derived
Gaussians agree on which are kept (alpha > 0), and over the kept ones
max |alpha_cached - alpha_fresh| <= 1/255 and
max_channel |c_cached - c_fresh| * alpha_fresh <= 1/255 (a reading: colour
and opacity errors below one 8-bit level).

Training: mean binary cross-entropy on the logits; Adam (beta1 0.9,
beta2 0.999, eps 1e-8, bias-corrected) on float32 master weights; the
forward and backward passes use the bfloat16-rounded weights.  Flat
parameter layout: W1 [36][64] (input-major), b1 [64], w2 [64], b2 [1].
"""
from __future__ import annotations

import numpy as np

NZ = 36
NH = 64
NPARAM = NZ * NH + NH + NH + 1
DIR_SCALE = np.float32(1024.0)
LABEL_THR = 1.0 / 255.0


# ------------------------------------------------------------------ parameters
def unpack(theta: np.ndarray):
    theta = np.asarray(theta)
    assert theta.shape == (NPARAM,)
    W1 = theta[: NZ * NH].reshape(NZ, NH)
    b1 = theta[NZ * NH: NZ * NH + NH]
    w2 = theta[NZ * NH + NH: NZ * NH + 2 * NH]
    b2 = theta[NPARAM - 1]
    return W1, b1, w2, b2


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(np.asarray(x, np.float32))
    r = np.where(nan, b | 0x00400000, r)
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).reshape(np.shape(x))


# ------------------------------------------------------------------ inputs (pinned float32)
def split_center(pc64: np.ndarray):
    pc64 = np.asarray(pc64, np.float64)
    hi = pc64.astype(np.float32)
    lo = (pc64 - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def pinned_dir(pos: np.ndarray, pc64: np.ndarray):
    """Unit directions [n,3] and distances [n] from the centre to the anchors, float32."""
    hi, lo = split_center(pc64)
    pos = np.asarray(pos, np.float32)
    dx = (pos - hi[None, :]) - lo[None, :]
    n2 = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]
    n = np.sqrt(n2)
    safe = np.where(n > 0, n, np.float32(1.0))
    d = np.where((n > 0)[:, None], dx / safe[:, None], np.float32(0.0))
    return d.astype(np.float32), n.astype(np.float32)


def _exp_mant(x: np.ndarray):
    b = np.asarray(x, np.float32).view(np.uint32)
    e = ((b >> 23) & 0xFF).astype(np.int32) - 127
    m = ((b & 0x7FFFFF) | 0x3F800000).astype(np.uint32).view(np.float32)
    return e, m


def plog2(x: np.ndarray, offset: int = 0) -> np.ndarray:
    """(e - offset) + (m - 1) for x = m 2^e, m in [1, 2) (x > 0 normal), one
    float32 rounding; x <= 0 gives -127 - offset."""
    x = np.asarray(x, np.float32)
    e, m = _exp_mant(x)
    out = (e - offset).astype(np.float32) + (m - np.float32(1.0))
    return np.where(x > 0, out, np.float32(-127 - offset)).astype(np.float32)


def features(feat: np.ndarray, d_now: np.ndarray, d_line: np.ndarray, dist: np.ndarray) -> np.ndarray:
    """z [n,36] float32."""
    n = feat.shape[0]
    z = np.zeros((n, NZ), np.float32)
    z[:, :32] = np.asarray(feat, np.float32)
    z[:, 32:35] = (np.asarray(d_now, np.float32) - np.asarray(d_line, np.float32)) * DIR_SCALE
    z[:, 35] = plog2(dist, 8)
    return z


def logit_f32(z: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """The pinned float32 logit with bfloat16-rounded weights (see header)."""
    W1, b1, w2, b2 = unpack(bf16_round(np.asarray(theta, np.float32)))
    z = np.asarray(z, np.float32)
    acc = np.zeros((z.shape[0], NH), np.float32)
    for k in range(NZ):
        acc = acc + W1[k][None, :] * z[:, k: k + 1]
    acc = acc + b1[None, :]
    h = np.where(acc > 0, acc, np.float32(0.0))
    out = np.zeros(z.shape[0], np.float32)
    for j in range(NH):
        out = out + w2[j] * h[:, j]
    return out + np.float32(b2)


def decide(z: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Reuse iff sigmoid(logit) >= 0.5, i.e. logit >= 0."""
    return logit_f32(z, theta) >= 0


# ------------------------------------------------------------------ labels
def label(cached: np.ndarray, fresh: np.ndarray, thr: float = LABEL_THR) -> np.ndarray:
    """cached, fresh: [n,k,11] attributes (alpha, colour, scale, quaternion)."""
    cached = np.asarray(cached, np.float64)
    fresh = np.asarray(fresh, np.float64)
    kc, kf = cached[..., 0] > 0, fresh[..., 0] > 0
    same = np.all(kc == kf, axis=1)
    da = np.where(kf, np.abs(cached[..., 0] - fresh[..., 0]), 0.0).max(axis=1)
    dc = np.where(kf, np.abs(cached[..., 1:4] - fresh[..., 1:4]).max(axis=2) * fresh[..., 0], 0.0).max(axis=1)
    return same & (da <= thr) & (dc <= thr)


def label_margin(cached: np.ndarray, fresh: np.ndarray, thr: float = LABEL_THR) -> np.ndarray:
    """Per sample, the distance of the label's closest comparison to its
    threshold: |alpha| for the kept tests, |d alpha - thr| and |d c alpha - thr|
    over the kept Gaussians."""
    cached = np.asarray(cached, np.float64)
    fresh = np.asarray(fresh, np.float64)
    kf = fresh[..., 0] > 0
    m_keep = np.minimum(np.abs(cached[..., 0]), np.abs(fresh[..., 0])).min(axis=1)
    da = np.abs(np.abs(cached[..., 0] - fresh[..., 0]) - thr)
    dc = np.abs(np.abs(cached[..., 1:4] - fresh[..., 1:4]).max(axis=2) * fresh[..., 0] - thr)
    m_cmp = np.where(kf, np.minimum(da, dc), np.inf).min(axis=1)
    return np.minimum(m_keep, m_cmp)


# ------------------------------------------------------------------ training (float64)
def _weights(theta: np.ndarray, round_weights: bool):
    if round_weights:
        return unpack(bf16_round(np.asarray(theta, np.float32)).astype(np.float64))
    return unpack(np.asarray(theta, np.float64))


def forward64(theta: np.ndarray, Z: np.ndarray, round_weights: bool = True):
    """Pre-activations, hidden and logits in float64 (weights bf16-rounded unless told not to)."""
    W1, b1, w2, b2 = _weights(theta, round_weights)
    Z = np.asarray(Z, np.float64)
    pre = Z @ W1 + b1[None, :]
    h = np.maximum(pre, 0.0)
    return pre, h, h @ w2 + b2


def bce(logit: np.ndarray, y: np.ndarray) -> float:
    """Mean of softplus(l) - y l (binary cross-entropy of sigmoid(l) against y)."""
    l = np.asarray(logit, np.float64)
    y = np.asarray(y, np.float64)
    return float(np.mean(np.maximum(l, 0.0) - y * l + np.log1p(np.exp(-np.abs(l)))))


def loss64(theta: np.ndarray, Z: np.ndarray, y: np.ndarray, round_weights: bool = True) -> float:
    return bce(forward64(theta, Z, round_weights)[2], y)


def grad64(theta: np.ndarray, Z: np.ndarray, y: np.ndarray, round_weights: bool = True):
    """(loss, d loss / d theta) by backpropagation through the float64 forward
    (with the bf16-rounded weights by default: the gradient is then taken with
    respect to the weights the forward pass used)."""
    W1, b1, w2, b2 = _weights(theta, round_weights)
    Z = np.asarray(Z, np.float64)
    y = np.asarray(y, np.float64)
    n = Z.shape[0]
    pre = Z @ W1 + b1[None, :]
    h = np.maximum(pre, 0.0)
    l = h @ w2 + b2
    p = 1.0 / (1.0 + np.exp(-l))
    g = (p - y) / n                      # d loss / d logit
    dh = g[:, None] * w2[None, :] * (pre > 0)
    grad = np.concatenate([(Z.T @ dh).reshape(-1), dh.sum(axis=0), h.T @ g, [g.sum()]])
    return bce(l, y), grad


class Adam:
    def __init__(self, n: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta: np.ndarray, grad: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def train64(theta0: np.ndarray, Z: np.ndarray, y: np.ndarray, batches, lr: float):
    """Adam over the given mini-batches (lists of sample indices); returns
    (theta, per-batch losses).  theta is kept in float64 here."""
    theta = np.asarray(theta0, np.float64).copy()
    opt = Adam(theta.shape[0], lr)
    losses = []
    for idx in batches:
        loss, g = grad64(theta, Z[idx], y[idx])
        losses.append(loss)
        theta = opt.step(theta, g)
    return theta, losses
