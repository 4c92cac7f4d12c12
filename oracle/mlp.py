"""Learned BP warm start: features, MLP, loss and Adam (oracle, NumPy).

Test infrastructure (like the rest of oracle/): a plain CPU statement of what
the GPU kernels of the warm start compute.  The paper has no learned part
(its BP starts from the gate-time messages).  The extension: per directed
bond e and Schmidt index k, a small MLP predicts the log of the diagonal of the converged
double-layer message in the bond's Schmidt basis, and damped BP then runs
to its tolerance from the trace-1 diagonal that blends the prediction
exp(y) / sum(exp(y)) with the diag(lambda) start by a weight gamma.

Rows: (bond b, direction dir, k) for k < chi_b.  Features (NF = 12):
  0  log lam_k (Vidal-normalised spectrum, Eq. 12; clamped at 1e-30)
  1  k / chi_b
  2  S_b / log chi_b  (entanglement-entropy fraction; 0 when chi_b = 1)
  3  deg(source site) / 4          4  deg(target site) / 4
  5  |source - obs|_1 / (Lx + Ly)  6  |target - obs|_1 / (Lx + Ly)
  7  t = step * dt                 8  h                 9  J
  10 mean, 11 max of S_e / log chi_e over the other bonds of the source site
     (0 when there are none or chi_e = 1)
MLP: y = W3 g(W2 g(W1 x + b1) + b2) + b3, widths NF -> 256 -> 256 -> 1,
g = GELU (exact, erf form).  Loss: mean squared error of y against the target
log-diagonal.  The GPU keeps weights and activations in BF16 with FP32
accumulation; `bf16` below rounds a float array to the nearest BF16 (ties to
even) so the two can be compared at equal rounding points.

Pinned by: tests/test_oracle_mlp.py -- the gradients equal central finite
differences of the loss (float64, no rounding), GELU matches its closed form
and derivative, Adam's first step moves every parameter by lr * sign(grad),
and the features of a hand-built 3x3 state equal values worked out by hand.
"""
import math

import numpy as np

NF = 12
WIDTH = 256


def bond_list(Lx, Ly):
    """Library bond numbering: horizontal bonds (y (Lx-1) + x) then vertical."""
    bonds = []
    for y in range(Ly):
        for x in range(Lx - 1):
            bonds.append((y * Lx + x, y * Lx + x + 1))
    for y in range(Ly - 1):
        for x in range(Lx):
            bonds.append((y * Lx + x, (y + 1) * Lx + x))
    return bonds


def entropy_fraction(lam, chi):
    if chi < 2:
        return 0.0
    p = np.asarray(lam[:chi], dtype=np.float64) ** 2
    p = p[p > 0]
    return float(-(p * np.log(p)).sum() / math.log(chi))


def features(Lx, Ly, obs_xy, chi, lam, step, dt, h, J):
    """Feature rows in (bond, dir, k) order; returns (X [rows, NF], index [rows, 3])."""
    bonds = bond_list(Lx, Ly)
    deg = np.zeros(Lx * Ly, dtype=int)
    site_bonds = [[] for _ in range(Lx * Ly)]
    for b, (u, v) in enumerate(bonds):
        deg[u] += 1
        deg[v] += 1
        site_bonds[u].append(b)
        site_bonds[v].append(b)
    ox, oy = obs_xy
    dist = np.array([abs(v % Lx - ox) + abs(v // Lx - oy) for v in range(Lx * Ly)], dtype=np.float64)
    sfrac = np.array([entropy_fraction(lam[b], int(chi[b])) for b in range(len(bonds))])
    rows, idx = [], []
    for b, (u, v) in enumerate(bonds):
        for d, (src, dst) in enumerate(((u, v), (v, u))):
            others = [e for e in site_bonds[src] if e != b]
            nb = [sfrac[e] for e in others]
            mean_nb = float(np.mean(nb)) if nb else 0.0
            max_nb = float(np.max(nb)) if nb else 0.0
            c = int(chi[b])
            for k in range(c):
                lk = max(float(lam[b][k]), 1e-30)
                rows.append([math.log(lk), k / c, sfrac[b], deg[src] / 4.0, deg[dst] / 4.0,
                             dist[src] / (Lx + Ly), dist[dst] / (Lx + Ly), step * dt, h, J,
                             mean_nb, max_nb])
                idx.append((b, d, k))
    return np.asarray(rows, dtype=np.float64), np.asarray(idx, dtype=np.int64)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def init_params(seed=0):
    """He-style uniform initialisation (the GPU copy starts from these values)."""
    rng = np.random.default_rng(seed)
    def layer(fan_in, fan_out):
        a = math.sqrt(6.0 / fan_in) * 0.5
        return rng.uniform(-a, a, size=(fan_in, fan_out)), np.zeros(fan_out)
    W1, b1 = layer(NF, WIDTH)
    W2, b2 = layer(WIDTH, WIDTH)
    W3, b3 = layer(WIDTH, 1)
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def forward(p, X, rnd=None):
    """Returns y [rows] and the cache for backward.  rnd: rounding applied to
    weights and stored activations (None = exact float64)."""
    r = rnd if rnd is not None else (lambda a: a)
    x = r(X)
    z1 = x @ r(p["W1"]) + p["b1"]
    a1 = r(gelu(z1))
    z2 = a1 @ r(p["W2"]) + p["b2"]
    a2 = r(gelu(z2))
    y = (a2 @ r(p["W3"]) + p["b3"])[:, 0]
    return y, dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2)


def loss(y, target):
    d = y - target
    return float(np.mean(d * d))


def backward(p, cache, y, target, rnd=None):
    """Gradients of the mean squared error with respect to every parameter."""
    r = rnd if rnd is not None else (lambda a: a)
    n = y.shape[0]
    dy = (2.0 / n) * (y - target)[:, None]
    g = {}
    g["W3"] = cache["a2"].T @ dy
    g["b3"] = dy.sum(axis=0)
    da2 = dy @ r(p["W3"]).T
    dz2 = da2 * gelu_grad(cache["z2"])
    g["W2"] = cache["a1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    da1 = dz2 @ r(p["W2"]).T
    dz1 = da1 * gelu_grad(cache["z1"])
    g["W1"] = cache["x"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return g


class Adam:
    """Adam (Kingma and Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr mhat / (sqrt(vhat) + eps), with bias-corrected mhat, vhat."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * grads[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * grads[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def warm_message(y, plain_diag=None, gamma=1.0):
    """Initial message of one directed bond: the trace-1 diagonal
    (1 - gamma) d / sum(d) + gamma exp(y) / sum(exp(y)), d = the current
    (diag(lambda)) diagonal; gamma = 1 uses the prediction alone."""
    e = np.exp(y - np.max(y))
    p = e / e.sum()
    if plain_diag is not None and gamma < 1.0:
        d = np.asarray(plain_diag, dtype=np.float64)
        p = (1.0 - gamma) * d / d.sum() + gamma * p
    return np.diag(p)
