"""Float64 reference of the learned recovery seed: features, network, loss,
gradient and Adam, written out plainly in numpy.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests, the
smoke check and the benchmark's CPU legs use it to check the library's
tensor-core inference and float32 training kernels. The paper has no learned
part; what the network approximates is the paper's primitive recovery (the
Landau eigenproblem of Sec. III, coupling), and only its starting vector is
taken from the network.

Network: 20 -> 64 -> 64 -> 64 -> 4, ReLU after the three hidden layers,
linear output. Parameters are one float vector in the order W1[64][20] b1[64]
W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4], W[out][in].

Pins (tests/test_oracle_mlp.py): gradient against central finite
differences; a hand-built parameter set whose output is a known closed form;
zero loss and zero gradient at an exact fit; the first Adam step against its
closed form lr * g / (|g| + eps); splitmix64 against its published output
sequence; features of a uniform state against the stress tensor of a perfect
fluid written out by hand.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 20, 64, 4
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_H)), ("b3", (N_H,)), ("W4", (N_OUT, N_H)), ("b4", (N_OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
ROW = N_IN + N_OUT

MASK64 = (1 << 64) - 1


def unpack(P):
    """Parameter vector -> dict of arrays (views)."""
    P = np.asarray(P, dtype=np.float64).reshape(-1)
    assert P.size == NPARAM
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = P[o:o + n].reshape(shape)
        o += n
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


# --------------------------------------------------------------------------
# features: normalised moments of one cell (the network's input)
# --------------------------------------------------------------------------
def features(T, N, E_old, B_old) -> np.ndarray:
    """Features of one cell from its streamed moments T^{mu nu} (4 x 4, Eq.
    Cal_T), N^mu (4, Eq. Cal_N) and the previous step's E, B: T^{0a}/T^00,
    (T^xx, T^yy, T^zz, T^xy, T^xz, T^yz)/T^00, N^a/N^0, N^0/T^00,
    E/sqrt(T^00), B/sqrt(T^00), 1."""
    T = np.asarray(T, dtype=np.float64).reshape(4, 4)
    N = np.asarray(N, dtype=np.float64).reshape(4)
    T00 = T[0, 0]
    x = np.empty(N_IN)
    x[0:3] = T[0, 1:4] / T00
    x[3:9] = np.array([T[1, 1], T[2, 2], T[3, 3], T[1, 2], T[1, 3], T[2, 3]]) / T00
    x[9:12] = N[1:4] / N[0]
    x[12] = N[0] / T00
    x[13:16] = np.asarray(E_old, dtype=np.float64) / np.sqrt(T00)
    x[16:19] = np.asarray(B_old, dtype=np.float64) / np.sqrt(T00)
    x[19] = 1.0
    return x


def targets(u, eps, c, T00) -> np.ndarray:
    """Training targets of one cell: beta = u / c (3) and eps / T^00 - 1."""
    return np.concatenate([np.asarray(u, dtype=np.float64) / c, [eps / T00 - 1.0]])


# --------------------------------------------------------------------------
# network, loss, gradient
# --------------------------------------------------------------------------
def relu(a):
    return np.maximum(a, 0.0)


def forward(P, X, keep=False):
    """Outputs (n x 4) for inputs X (n x 20); with keep=True also the hidden
    activations needed by the backward pass."""
    p = unpack(P)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    h1 = relu(X @ p["W1"].T + p["b1"])
    h2 = relu(h1 @ p["W2"].T + p["b2"])
    h3 = relu(h2 @ p["W3"].T + p["b3"])
    y = h3 @ p["W4"].T + p["b4"]
    return (y, (X, h1, h2, h3)) if keep else y


def loss(P, X, Y) -> float:
    """Mean over samples of the squared error summed over the 4 outputs."""
    e = forward(P, X) - np.atleast_2d(Y)
    return float(np.sum(e * e) / e.shape[0])


def loss_and_grad(P, X, Y):
    """Loss and its gradient by back-propagation (chain rule layer by layer)."""
    p = unpack(P)
    y, (X, h1, h2, h3) = forward(P, X, keep=True)
    n = X.shape[0]
    e = y - np.atleast_2d(Y)
    L = float(np.sum(e * e) / n)
    dy = 2.0 * e / n                         # dL/dy
    g = {"W4": dy.T @ h3, "b4": dy.sum(0)}
    d3 = (dy @ p["W4"]) * (h3 > 0)           # dL/d(pre-activation 3)
    g["W3"], g["b3"] = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ p["W3"]) * (h2 > 0)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ p["W2"]) * (h1 > 0)
    g["W1"], g["b1"] = d1.T @ X, d1.sum(0)
    return L, pack(g)


def adam_step(P, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) at step t >= 1;
    returns the new (P, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return P - lr * mhat / (np.sqrt(vhat) + eps), m, v


# --------------------------------------------------------------------------
# mini-batch rows: splitmix64 (Steele, Lea and Flood, 2014) as a counter hash
# --------------------------------------------------------------------------
def splitmix64(x: int) -> int:
    """Output of SplitMix64 for state x (one increment by the golden gamma,
    then the variant-13 finaliser)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def batch_rows(seed: int, t: int, batch: int, n: int) -> np.ndarray:
    """Rows of mini-batch t (0-based) of the training call with this seed: the
    step's key s = splitmix64(seed + t + 1) | 1, then row j = splitmix64(s XOR
    (j * 0x2545F4914F6CDD1D mod 2^64)) mod n."""
    s = splitmix64((seed + t + 1) & MASK64) | 1
    return np.array([splitmix64(s ^ ((j * 0x2545F4914F6CDD1D) & MASK64)) % n for j in range(batch)], dtype=np.int64)


def train(P, m, v, data, steps, batch, lr, seed):
    """Adam on mini-batches drawn by batch_rows; returns (P, m, v, losses)."""
    data = np.asarray(data, dtype=np.float64).reshape(-1, ROW)
    losses = []
    for t in range(steps):
        rows = batch_rows(seed, t, batch, data.shape[0])
        L, g = loss_and_grad(P, data[rows, :N_IN], data[rows, N_IN:])
        losses.append(L)
        P, m, v = adam_step(P, m, v, g, t + 1, lr)
    return P, m, v, np.array(losses)


# --------------------------------------------------------------------------
# bf16 emulation of the tensor-core inference (operands rounded to bfloat16
# with round-to-nearest-even, products accumulated in float32)
# --------------------------------------------------------------------------
def to_bf16(a) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    x = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
    return x.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(P, X):
    """forward() with the inference kernel's roundings: inputs, weights and
    hidden activations in bfloat16, sums and biases in float32."""
    p = unpack(P)
    a = to_bf16(np.atleast_2d(X))
    for i in (1, 2, 3):
        z = (a @ to_bf16(p[f"W{i}"]).T).astype(np.float32) + p[f"b{i}"].astype(np.float32)
        a = to_bf16(relu(z))
    return ((a @ to_bf16(p["W4"]).T).astype(np.float32) + p["b4"].astype(np.float32)).astype(np.float64)
