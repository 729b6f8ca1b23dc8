"""FP64 reference of the learned-alpha network and its training gradient.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests compare
the GPU forward/backward kernels against these plain numpy definitions.

Network (weight block layout as in the library): xhat = (x - mu) / sd,
h1 = tanh(W1 xhat + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3;
loss = mean over samples of (y - t)^2.  The gradient is written out by the
chain rule; `numeric_gradient` is the central-difference check of it.
"""
import numpy as np

NF, H = 32, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * NF
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
OFF_MU = OFF_B3 + 1
OFF_SD = OFF_MU + NF
NWEIGHTS = OFF_SD + NF
NTRAIN = OFF_MU


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    return dict(W1=w[OFF_W1:OFF_B1].reshape(H, NF), b1=w[OFF_B1:OFF_W2], W2=w[OFF_W2:OFF_B2].reshape(H, H),
                b2=w[OFF_B2:OFF_W3], w3=w[OFF_W3:OFF_B3], b3=w[OFF_B3], mu=w[OFF_MU:OFF_SD], sd=w[OFF_SD:NWEIGHTS])


def forward(w, X):
    p = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    xh = (X - p["mu"]) / p["sd"]
    h1 = np.tanh(xh @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["w3"] + p["b3"]
    return y, (xh, h1, h2)


def loss(w, X, T):
    y, _ = forward(w, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def gradient(w, X, T):
    """d loss / d (trainable parameters), in the weight-block order."""
    p = unpack(w)
    T = np.asarray(T, dtype=np.float64)
    y, (xh, h1, h2) = forward(w, X)
    B = len(T)
    dy = 2.0 * (y - T) / B                     # d loss / d y
    dz2 = (dy[:, None] * p["w3"][None, :]) * (1.0 - h2 ** 2)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 ** 2)
    g = np.zeros(NTRAIN)
    g[OFF_W1:OFF_B1] = (dz1.T @ xh).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    g[OFF_W3:OFF_B3] = dy @ h2
    g[OFF_B3] = dy.sum()
    return g


def numeric_gradient(w, X, T, idx, eps=1e-6):
    """Central differences of `loss` for the parameters in `idx`."""
    w = np.asarray(w, dtype=np.float64).copy()
    out = np.zeros(len(idx))
    for t, i in enumerate(idx):
        old = w[i]
        w[i] = old + eps
        lp = loss(w, X, T)
        w[i] = old - eps
        lm = loss(w, X, T)
        w[i] = old
        out[t] = (lp - lm) / (2 * eps)
    return out


def optimal_alpha(sigma):
    """Thm. 1: rho(R0) = max_i |1 - alpha sigma_i^2| over the nonzero singular
    values is minimised by alpha* = 2 / (sigma_1^2 + sigma_r^2)."""
    s = np.sort(np.asarray(sigma, dtype=np.float64))[::-1]
    s = s[s > 0]
    return 2.0 / (s[0] ** 2 + s[-1] ** 2)


def lanczos_ritz(A_chi, steps, start):
    """Ritz values of A^H A from `steps` Lanczos steps (complex representation
    chi(A), start vector chi-form), descending.  With steps equal to the
    dimension they are the eigenvalues of A^H A."""
    Hm = A_chi.conj().T @ A_chi
    q = start / np.linalg.norm(start)
    qp = np.zeros_like(q)
    al, be = [], []
    beta = 0.0
    for j in range(steps):
        w = Hm @ q
        a = float(np.real(np.vdot(q, w)))
        w = w - a * q - beta * qp
        al.append(a)
        beta = float(np.linalg.norm(w))
        if j + 1 < steps:
            if beta <= 1e-30:
                break
            be.append(beta)
            qp, q = q, w / beta
    k = len(al)
    T = np.diag(al) + np.diag(be[: k - 1], 1) + np.diag(be[: k - 1], -1)
    return np.sort(np.linalg.eigvalsh(T))[::-1]
