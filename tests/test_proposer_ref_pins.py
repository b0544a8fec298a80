"""Pins of the CPU reference of the learned proposer (oracle/proposer_ref.py)
against facts that do not come from that file: finite differences, hand
computed values, invariances, known binary16 roundings, and the paper's toy
example (Figure 1's lines) for the restricted-objective feature."""
import json
import os

import numpy as np
import pytest

from oracle import proposer_ref as P

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "toy_example.json")


def _theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, P.N_PARAMS)


def test_parameter_count_and_pack_roundtrip():
    assert P.N_PARAMS == 128 * 4 + 128 + 128 * 128 + 128 + 128 + 1 == 17281
    th = _theta(0)
    assert np.array_equal(P.pack(*P.unpack(th)), th)


def test_forward_hand_built_network():
    # unit 0 = relu(f0), unit 1 = relu(-f0), unit 2 = relu(f1 - 1): layer 2 passes
    # them through and the output is |f0| + 2 relu(f1 - 1) - 0.5
    W1 = np.zeros((128, 4)); b1 = np.zeros(128)
    W1[0, 0], W1[1, 0], W1[2, 1], b1[2] = 1.0, -1.0, 1.0, -1.0
    W2 = np.zeros((128, 128)); W2[0, 0] = W2[1, 1] = W2[2, 2] = 1.0
    b2 = np.zeros(128)
    w3 = np.zeros(128); w3[0] = w3[1] = 1.0; w3[2] = 2.0
    th = P.pack(W1, b1, W2, b2, w3, -0.5)
    F = np.array([[0.7, 3.0, 9.0, -4.0], [-2.5, 0.2, -1.0, 8.0], [0.0, 1.0, 0.0, 1.0]])
    want = np.abs(F[:, 0]) + 2 * np.maximum(F[:, 1] - 1.0, 0.0) - 0.5
    assert np.allclose(P.forward(th, F), want, rtol=0, atol=1e-15)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    th = _theta(2)
    F = rng.normal(size=(9, 4))
    ds = rng.normal(size=9)
    g = P.backward(th, F, ds)
    f = lambda t: float(ds @ P.forward(t, F))
    # every bias, w3 and b3 entry plus samples of both matrices (W1: 0..511,
    # b1: 512..639, W2: 640..17023, b2, w3, b3: 17024..17280)
    idx = list(range(512, 640)) + list(range(17024, 17281))
    idx += list(rng.choice(512, 40, replace=False)) + list(640 + rng.choice(16384, 200, replace=False))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th); e[i] = h
        fd = (f(th + e) - f(th - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_rank_loss_gradient_and_invariances():
    rng = np.random.default_rng(3)
    offs = np.array([0, 5, 5, 12, 20])  # one empty instance
    s = rng.normal(size=20)
    u = rng.normal(size=20)
    L, ds = P.rank_loss(s, u, offs)
    h = 1e-6
    for i in range(20):
        e = np.zeros(20); e[i] = h
        fd = (P.rank_loss(s + e, u, offs)[0] - P.rank_loss(s - e, u, offs)[0]) / (2 * h)
        assert abs(fd - ds[i]) < 1e-8
    # adding a constant to one instance's scores changes nothing
    s2 = s.copy(); s2[5:12] += 3.7
    L2, ds2 = P.rank_loss(s2, u, offs)
    assert abs(L2 - L) < 1e-12 and np.allclose(ds2, ds, atol=1e-14)
    # scores equal to the targets: zero gradient, loss = mean entropy of q
    L3, ds3 = P.rank_loss(u, u, offs)
    assert np.allclose(ds3, 0.0, atol=1e-15)
    ent = 0.0
    for b in range(4):
        q = np.exp(u[offs[b]:offs[b + 1]]); q /= max(q.sum(), 1e-300)
        ent += -(q * np.log(q)).sum() if q.size else 0.0
    assert abs(L3 - ent / 4) < 1e-12
    # each non-empty instance's gradient sums to zero (softmax minus softmax)
    for b in range(4):
        assert abs(ds[offs[b]:offs[b + 1]].sum()) < 1e-15


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(4)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    t1, m1, m2 = P.adam(th, g, np.zeros(50), np.zeros(50), 1, 0.01, eps=0.0)
    assert np.allclose(t1, th - 0.01 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)



def test_adam_first_step_with_epsilon_outside_the_root():
    """Adam (Kingma & Ba) divides by sqrt(v_hat) + eps; at step 1 the bias
    corrections give m_hat = g and v_hat = g^2, so the step is exactly
    -lr g / (|g| + eps), which for |g| near eps is far from -lr sign(g)."""
    g = np.array([1e-6, -3e-8, 0.0, 2.0, -1e-9])
    th = np.zeros(5)
    t1, _, _ = P.adam(th, g, np.zeros(5), np.zeros(5), 1, 0.01, eps=1e-8)
    want = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(t1, want, rtol=1e-12, atol=0)
    assert abs(t1[0] + 0.01 / 1.01) < 1e-15  # 1e-6 / (1e-6 + 1e-8) = 1 / 1.01


def test_relu_derivative_at_zero_is_zero():
    """A hidden unit whose pre-activation is exactly 0 (zero weights and bias)
    passes no gradient: ReLU'(0) = 0, so its incoming weights and bias get 0
    while its outgoing weight w3 still sees h2 = 0."""
    rng = np.random.default_rng(7)
    W1, b1, W2, b2, w3, b3 = P.unpack(_theta(3))
    u = 5
    W2 = W2.copy(); b2 = b2.copy(); w3 = w3.copy()
    W2[u, :] = 0.0
    b2[u] = 0.0
    w3[u] = 1.5
    th = P.pack(W1, b1, W2, b2, w3, b3)
    F = rng.normal(size=(6, 4))
    ds = rng.normal(size=6)
    _, (a1, h1, a2, h2) = P.forward(th, F, keep=True)
    assert (a2[:, u] == 0.0).all()
    dW1, db1, dW2, db2, dw3, db3 = P.unpack(P.backward(th, F, ds))
    assert (dW2[u, :] == 0.0).all() and db2[u] == 0.0
    assert dw3[u] == 0.0  # h2[:, u] = relu(0) = 0
    # the other units are untouched by unit u: their layer-2 gradients are the
    # closed form g2 = ds w3 [a2 > 0]
    g2 = np.outer(ds, w3) * (a2 > 0)
    assert np.allclose(db2, g2.sum(axis=0), rtol=1e-13, atol=1e-15)

def test_raw_features_hand_values():
    X = np.array([[3.0, 0.0, -1.0],
                  [-4.0, 0.0, 2.0],
                  [0.0, 0.0, -5.0],
                  [1.0, 0.0, 2.0]])
    F = P.column_features(X)
    assert np.allclose(F[:, 0], [8.0, 0.0, 10.0])
    assert np.allclose(F[:, 1], [np.sqrt(26.0), 0.0, np.sqrt(34.0)])
    # lower median of 4 values: rank 1 of the sorted |x|
    assert np.array_equal(F[:, 2], [1.0, 0.0, 2.0])
    F5 = P.column_features(np.array([[5.0], [-1.0], [3.0], [-2.0], [4.0]]))
    assert F5[0, 2] == 3.0


def test_proxy_rows_rule():
    assert [P.proxy_rows(n) for n in (1, 200, 256, 257, 2048, 2049, 5000)] == \
        [1, 200, 256, 256, 256, 257, 625]


def test_heavy_rows_hand_values():
    # row l1 norms: 4, 6, 6, 1, 9, 6; the three heaviest are rows 4 and the
    # first two of the rows tied at 6 (rows 1 and 2, ties to the smaller index)
    X = np.array([[1.0, -3.0], [2.0, 4.0], [-6.0, 0.0], [0.5, 0.5], [9.0, 0.0], [3.0, -3.0]])
    assert list(P.heavy_rows(X, 3)) == [1, 2, 4]
    assert list(P.heavy_rows(X, 1)) == [4]
    assert list(P.heavy_rows(X, 6)) == [0, 1, 2, 3, 4, 5]


def test_proxy_objective_on_the_toy_example():
    """The restricted objective is Algorithm 1 on the heavy rows: the paper's
    five toy points, hidden among light rows that the restriction must drop,
    give Figure 1's objective lines z_jhat(lambda) (intercept + slope lambda,
    to one unit of the last printed digit: the figure truncates 113/3)."""
    g = json.load(open(GOLD))
    toy = np.array(g["points"], dtype=np.float64)
    rng = np.random.default_rng(11)
    light = rng.uniform(-0.01, 0.01, size=(40, 4))
    X = np.concatenate([light[:17], toy, light[17:]])
    rows = P.heavy_rows(X, 5)
    assert list(rows) == list(range(17, 22))

    def tol(s):
        return 10.0 ** -(len(s.split(".")[1]) if "." in s else 0)  # one unit: the figure truncates
    for ln in g["figure1_lines"]:
        lam = (ln["from"] + ln["to"]) / 2
        z = P.proxy_objective(X, lam, R=5)[ln["jhat"] - 1]
        pred = float(ln["intercept"]) + float(ln["slope"]) * lam
        assert abs(z - pred) <= tol(ln["intercept"]) + tol(ln["slope"]) * lam + 1e-9, (ln, z)


def test_standardise():
    rng = np.random.default_rng(5)
    F = rng.gamma(2.0, size=(40, 3))
    F[:, 1] = 7.0  # constant feature
    Z = P.standardise(F)
    assert np.allclose(Z[:, [0, 2]].mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(Z[:, [0, 2]].std(axis=0), 1.0, atol=1e-12)
    assert np.array_equal(Z[:, 1], np.zeros(40))


def test_half_rounding_known_values():
    th = np.zeros(P.N_PARAMS)
    th[0] = 1.0 / 3.0            # nearest binary16: 0.333251953125
    th[1] = 1.0 + 2.0 ** -11     # exactly halfway: ties to even -> 1.0
    th[2] = 1.0 + 3 * 2.0 ** -11  # halfway, ties to even -> 1 + 2^-9
    th[3] = 65504.0              # largest finite binary16
    th[512] = 1.0 / 3.0          # a bias: not rounded
    r = P.half_weights(th)
    assert r[0] == 0.333251953125 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -9
    assert r[3] == 65504.0 and r[512] == 1.0 / 3.0


def test_topk_ties_and_nan():
    s = np.array([0.5, 2.0, np.nan, 2.0, -1.0, 0.5, -np.inf])
    assert list(P.topk(s, 1)) == [1]
    assert list(P.topk(s, 2)) == [1, 3]
    assert list(P.topk(s, 3)) == [0, 1, 3]
    assert list(P.topk(s, 6)) == [0, 1, 3, 4, 5, 6]
    assert list(P.topk(s, 7)) == [0, 1, 2, 3, 4, 5, 6]


def test_target_logits():
    z = np.array([5.0, 3.0, 9.0, 4.0, 3.5])
    u = P.target_logits(z, temperature=0.5, top=3)
    # z_min = 3, third smallest = 4: span 1
    assert np.allclose(u, -(z - 3.0) / 0.5)
    assert u[1] == 0.0 and u.argmax() == 1
