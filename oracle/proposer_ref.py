"""CPU reference of the learned jhat proposer (not part of the paper).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests compare the
CUDA feature, network, loss, optimiser and top-K kernels with these plain
float64 numpy definitions.  Nothing here is imported by the product path.

The proposer ranks the candidate preserved coordinates jhat of Algorithm 1 so
that only the best K are scored exactly; the exact scores still decide.

* Features of column jhat: l1 norm, l2 norm and the lower median of |x_i,jhat|
  (the element of 0-based rank floor((n-1)/2) in ascending order), and the
  objective z_jhat of Algorithm 1 (penalty lambda) restricted to the R rows of
  largest l1 norm (R = proxy_rows(n)), each then standardised across the m
  columns of the instance (mean 0, population standard deviation 1; a feature
  constant over the columns becomes 0).  The restricted objective uses the
  exact method itself (the C oracle) on those rows.
* Network: 4 -> 128 -> 128 -> 1 with ReLU.  The weight matrices are used at
  half precision (the caller passes them already rounded); biases, activations
  and sums are exact here (float64).
* Loss per instance: cross entropy between softmax(target logits) and
  softmax(scores) over that instance's columns, averaged over the instances of
  the batch.
* Optimiser: Adam (Kingma and Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

H = 128
NF = 4  # input features
N_PARAMS = H * NF + H + H * H + H + H + 1  # W1, b1, W2, b2, w3, b3 in that order


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def unpack(theta):
    """Flat parameter vector -> (W1 [H,NF], b1 [H], W2 [H,H], b2 [H], w3 [H], b3)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    o = 0
    W1 = theta[o:o + NF * H].reshape(H, NF)
    o += NF * H
    b1 = theta[o:o + H]
    o += H
    W2 = theta[o:o + H * H].reshape(H, H)
    o += H * H
    b2 = theta[o:o + H]
    o += H
    w3 = theta[o:o + H]
    o += H
    b3 = float(theta[o])
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def half_weights(theta):
    """The parameters as the network uses them: weight matrices rounded to
    IEEE binary16 (round to nearest even), biases unchanged."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    r = lambda a: a.astype(np.float16).astype(np.float64)
    return pack(r(W1), b1, r(W2), b2, r(w3), b3)


# ---------------------------------------------------------------------------
# features
# ---------------------------------------------------------------------------
def column_features(X):
    """(m, 3): l1 norm, l2 norm, lower median of |x| for every column of X."""
    A = np.abs(np.asarray(X, dtype=np.float64))
    n = A.shape[0]
    l1 = A.sum(axis=0)
    l2 = np.sqrt((A * A).sum(axis=0))
    med = np.sort(A, axis=0)[(n - 1) // 2]
    return np.stack([l1, l2, med], axis=1)


def proxy_rows(n):
    """Rows of the restricted fit: min(n, max(256, ceil(n / 8)))."""
    return min(n, max(256, -(-n // 8)))


def heavy_rows(X, R):
    """The R rows of largest l1 norm, in ascending index order.  The norm of a
    row is the double sum of its |x_ij| taken left to right over j; rows are
    ranked by that sum rounded to float, ties to the smaller index."""
    A = np.abs(np.asarray(X, dtype=np.float64))
    rho = np.cumsum(A, axis=1)[:, -1] if A.shape[1] else np.zeros(A.shape[0])
    key = rho.astype(np.float32).astype(np.float64)
    order = np.lexsort((np.arange(key.size), -key))
    return np.sort(order[:R])


def proxy_objective(X, lam, R=None):
    """z_jhat of Algorithm 1 on the R heaviest rows (every jhat), by the oracle."""
    import oracle
    X = np.asarray(X)
    R = proxy_rows(X.shape[0]) if R is None else R
    rows = heavy_rows(X, R)
    return oracle.fit(np.ascontiguousarray(X[rows]), [lam])["z_all"][0]


def raw_features(X, lam):
    """(m, 4): the three column features and the restricted objective."""
    return np.concatenate([column_features(X), proxy_objective(X, lam)[:, None]], axis=1)


def standardise(F):
    """Per feature: subtract the mean over the columns, divide by the
    population standard deviation (0 where that deviation is 0)."""
    F = np.asarray(F, dtype=np.float64)
    mu = F.mean(axis=0)
    sd = np.sqrt(((F - mu) ** 2).mean(axis=0))
    out = np.zeros_like(F)
    for c in range(F.shape[1]):
        if sd[c] > 0:
            out[:, c] = (F[:, c] - mu[c]) / sd[c]
    return out


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def forward(theta, F, keep=False):
    """Scores for the rows of F (N, NF).  `theta` is used as given (round it
    with half_weights first to model the half-precision weights)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    F = np.asarray(F, dtype=np.float64)
    a1 = F @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    s = h2 @ w3 + b3
    if keep:
        return s, (a1, h1, a2, h2)
    return s


def backward(theta, F, ds):
    """Gradient of sum_r ds[r] * score[r] with respect to the flat parameters
    (chain rule through the two ReLU layers; ReLU'(0) = 0)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    F = np.asarray(F, dtype=np.float64)
    ds = np.asarray(ds, dtype=np.float64)
    _, (a1, h1, a2, h2) = forward(theta, F, keep=True)
    dw3 = h2.T @ ds
    db3 = ds.sum()
    g2 = np.outer(ds, w3) * (a2 > 0)
    dW2 = g2.T @ h1
    db2 = g2.sum(axis=0)
    g1 = (g2 @ W2) * (a1 > 0)
    dW1 = g1.T @ F
    db1 = g1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dw3, db3)


# ---------------------------------------------------------------------------
# listwise loss
# ---------------------------------------------------------------------------
def _softmax(x):
    e = np.exp(x - x.max())
    return e / e.sum()


def rank_loss(scores, targets, offsets):
    """Mean over instances of CE(softmax(targets_I), softmax(scores_I)) and its
    gradient with respect to the scores.  offsets: instance b owns rows
    offsets[b] .. offsets[b+1]-1."""
    s = np.asarray(scores, dtype=np.float64)
    u = np.asarray(targets, dtype=np.float64)
    nb = len(offsets) - 1
    ds = np.zeros_like(s)
    loss = 0.0
    for b in range(nb):
        r0, r1 = int(offsets[b]), int(offsets[b + 1])
        if r1 <= r0:
            continue
        q = _softmax(u[r0:r1])
        p = _softmax(s[r0:r1])
        lse = s[r0:r1].max() + np.log(np.exp(s[r0:r1] - s[r0:r1].max()).sum())
        loss += -(q * s[r0:r1]).sum() + lse
        ds[r0:r1] = (p - q) / nb
    return loss / nb, ds


def target_logits(z, temperature=0.25, top=16):
    """Training target of one instance from its exact objectives z_jhat:
    logits -(z - z_min) / (temperature * (z_(top) - z_min)), where z_(top) is
    the top-th smallest objective, so that the best columns carry the mass."""
    z = np.asarray(z, dtype=np.float64)
    zs = np.sort(z)
    span = zs[min(top, z.size) - 1] - zs[0]
    if not span > 0:
        span = max(abs(zs[0]), 1.0)
    return -(z - zs[0]) / (temperature * span)


# ---------------------------------------------------------------------------
# optimiser and top-K
# ---------------------------------------------------------------------------
def adam(theta, g, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** step)
    vh = m2 / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2


def topk(scores, K):
    """Indices of the K highest scores, ties to the smaller index, NaN lowest;
    returned in ascending index order."""
    s = np.asarray(scores, dtype=np.float64)
    key = np.where(np.isnan(s), -np.inf, s)
    nanmask = np.isnan(s).astype(np.int8)
    order = np.lexsort((np.arange(s.size), -key, nanmask))
    return np.sort(order[:K])
