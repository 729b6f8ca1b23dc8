"""Seeded synthetic quaternion inputs, shared by the tests, the benchmark and
the oracle's callers.  This module holds no arithmetic of the pseudoinverse
method itself: only random draws and the construction of test matrices with a
prescribed singular value decomposition.

Conventions
-----------
* A quaternion matrix is a ``(4, rows, cols)`` float64 array of real component
  planes (s, x, y, z), each row-major.
* Random numbers come from a counter-based splitmix64 stream: draw ``c`` of
  stream ``seed`` is ``splitmix64(seed + (c + 1) * 0x9E3779B97F4A7C15)``;
  uniforms take the top 53 bits; normals are Box-Muller pairs.  Draw order for
  a Gaussian quaternion matrix is plane s, x, y, z, each row-major.
* Matrices with a prescribed spectrum are built through the interleaved
  complex representation chi(q) = [[s + x i, y + z i], [-y + z i, s - x i]]
  (a *-homomorphism from quaternions to 2x2 complex matrices, Sec. 2).
  Orthonormal quaternion factors come from CholeskyQR2 of Gaussian quaternion
  matrices in that representation: the complex Cholesky factor of chi(G^H G)
  is chi(L) of the quaternion Cholesky factor L (unique, positive real
  diagonal), so Q = G L^{-H} is the Q factor of a quaternion QR with positive
  real diagonal in R (Haar distributed).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the splitmix64 stream `seed` (uint64)."""
    c = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + c * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller; normal t uses uniforms 2*(t//2), 2*(t//2)+1."""
    pairs = (count + 1) // 2
    u = uniform(seed, 2 * pairs, 2 * ((offset + 1) // 2) if offset else 0)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    g = np.empty(2 * pairs)
    g[0::2] = r * np.cos(2.0 * math.pi * u2)
    g[1::2] = r * np.sin(2.0 * math.pi * u2)
    return g[:count]


def gaussian_quaternion(m: int, n: int, seed: int) -> np.ndarray:
    """(4, m, n) planes, every component i.i.d. N(0, 1)."""
    return normal(seed, 4 * m * n).reshape(4, m, n)


# ---------------------------------------------------------------- chi tools

def chi(Q: np.ndarray) -> np.ndarray:
    """Interleaved complex representation, (4, m, n) -> (2m, 2n) complex128."""
    s, x, y, z = Q
    m, n = s.shape
    C = np.empty((2 * m, 2 * n), dtype=np.complex128)
    C[0::2, 0::2] = s + 1j * x
    C[0::2, 1::2] = y + 1j * z
    C[1::2, 0::2] = -y + 1j * z
    C[1::2, 1::2] = s - 1j * x
    return C


def unchi(C) -> np.ndarray:
    """Inverse of chi (reads the first row of every 2x2 block)."""
    C = np.asarray(C)
    a = C[0::2, 0::2]
    b = C[0::2, 1::2]
    return np.ascontiguousarray(np.stack([a.real, a.imag, b.real, b.imag]))


def _torch_device(device):
    import torch  # local import: numpy-only callers never need torch
    return torch, torch.device(device)


def _cholqr_chi(C, device):
    """Q factor (in chi form) of CholeskyQR2 applied to chi-form C."""
    torch, dev = _torch_device(device)
    Ct = torch.as_tensor(C, device=dev)
    for _ in range(2):
        H = Ct.mH @ Ct
        H = 0.5 * (H + H.mH)
        L = torch.linalg.cholesky(H)
        # Q = C L^{-H}  <=>  Q^H = L^{-1} C^H
        Ct = torch.linalg.solve_triangular(L, Ct.mH, upper=False).mH
    return Ct


def orthonormal_columns(m: int, r: int, seed: int, device="cpu") -> np.ndarray:
    """(4, m, r) quaternion matrix with orthonormal columns (Haar for m == r)."""
    G = gaussian_quaternion(m, r, seed)
    return unchi(_cholqr_chi(chi(G), device).resolve_conj().cpu().numpy())


def with_spectrum(U: np.ndarray, sigma: np.ndarray, V: np.ndarray, device="cpu") -> np.ndarray:
    """A = U diag(sigma) V^H for U (4,m,r), V (4,n,r), sigma (r,)."""
    torch, dev = _torch_device(device)
    cu = torch.as_tensor(chi(U), device=dev)
    cv = torch.as_tensor(chi(V), device=dev)
    s2 = torch.as_tensor(np.repeat(np.asarray(sigma, dtype=np.float64), 2), device=dev)
    return unchi(((cu * s2[None, :]) @ cv.mH).resolve_conj().cpu().numpy())


# ------------------------------------------------------------ workloads

def dense_gaussian(m: int = 64, n: int = 48, seed: int = 0) -> np.ndarray:
    """Dense Gaussian workload: every component i.i.d. N(0,1) (full rank a.s.)."""
    return gaussian_quaternion(m, n, seed)


def logspaced_square(n: int = 2048, smin: float = 1e-6, seed_u: int = 1, seed_v: int = 2,
                     device="cpu"):
    """Square A = U diag(sigma) V^H, U, V Haar quaternion unitaries, sigma
    log-spaced from 1 down to smin.  Returns (A, U, sigma, V)."""
    sigma = np.logspace(0.0, math.log10(smin), n) if n > 1 else np.ones(1)
    U = orthonormal_columns(n, n, seed_u, device)
    V = orthonormal_columns(n, n, seed_v, device)
    return with_spectrum(U, sigma, V, device), U, sigma, V


def rank_deficient(m: int = 8192, n: int = 4096, r: int = 2048, smin: float = 1e-4,
                   seed_l: int = 4, seed_r: int = 5, device="cpu"):
    """Rank-r A = QL diag(sigma) QR^H with orthonormal Gaussian-derived factors
    and sigma geometric from 1 to smin.  Returns (A, QL, sigma, QR)."""
    sigma = np.geomspace(1.0, smin, r) if r > 1 else np.ones(1)
    QL = orthonormal_columns(m, r, seed_l, device)
    QR = orthonormal_columns(n, r, seed_r, device)
    return with_spectrum(QL, sigma, QR, device), QL, sigma, QR


def pure_quaternion_batch(count: int = 4096, seed: int = 3, lo: int = 16, hi: int = 256,
                          rmin: int = 4):
    """Batch of pure-quaternion matrices A = B W (zero real part): B is m x r
    with i/j/k components uniform in [0, 1], W is r x n real with Dirichlet(1)
    columns, so entries stay in [0, 1] and rank(A) = r almost surely.
    m, n ~ U{lo..hi}, r ~ U{rmin..min(m, n)}.  Matrix b uses stream
    (seed, draws from offset b * 2**32)."""
    mats = []
    for b in range(count):
        off = b << 32
        u = uniform(seed, 3, off)
        m = lo + int(u[0] * (hi - lo + 1))
        n = lo + int(u[1] * (hi - lo + 1))
        rhi = min(m, n)
        r = rmin + int(u[2] * (rhi - rmin + 1))
        Bx = uniform(seed, 3 * m * r, off + 3).reshape(3, m, r)
        e = -np.log1p(-uniform(seed, r * n, off + 3 + 3 * m * r)).reshape(r, n)
        W = e / e.sum(axis=0, keepdims=True)
        A = np.zeros((4, m, n))
        A[1:] = Bx @ W
        mats.append(A)
    return mats


# ------------------------------------------------------- image completion

def synthetic_rgb_image(m: int = 512, n: int = 768, seed: int = 16, texture: float = 0.02) -> np.ndarray:
    """Smooth synthetic colour image as a pure quaternion matrix (zero real
    plane; planes x, y, z = R, G, B in [0, 1]), standing in for a natural
    photograph such as kodim16 (512 x 768).  Channel c: 24 plane waves of
    random orientation with up to 6 cycles across the frame and amplitudes
    falling as 1 / (1 + frequency), plus 8 Gaussian blobs (width 3-15 % of
    the frame), scaled into [0.1, 0.9]; then N(0, texture^2) pixel texture;
    clipped to [0, 1].  Channel c draws from stream `seed` at offset c << 32."""
    y = (np.arange(m, dtype=np.float64)[:, None] + 0.5) / m
    x = (np.arange(n, dtype=np.float64)[None, :] + 0.5) / n
    img = np.zeros((4, m, n))
    for c in range(3):
        off = c << 32
        w = uniform(seed, 4 * 24, off).reshape(24, 4)
        b = uniform(seed, 5 * 8, off + 96).reshape(8, 5)
        f = np.zeros((m, n))
        for fy, fx, ph, amp in w:
            ky, kx = (fy - 0.5) * 12.0, (fx - 0.5) * 12.0
            f += amp / (1.0 + math.hypot(ky, kx)) * np.cos(2.0 * math.pi * (ky * y + kx * x + ph))
        for cy, cx, wd, amp, sgn in b:
            s = 0.03 + 0.12 * wd
            f += (2.0 * amp) * (1.0 if sgn < 0.5 else -1.0) * np.exp(-((y - cy) ** 2 + (x - cx) ** 2) / (2 * s * s))
        f = 0.1 + 0.8 * (f - f.min()) / max(f.max() - f.min(), 1e-300)
        f += texture * normal(seed, m * n, off + 256).reshape(m, n)
        img[1 + c] = np.clip(f, 0.0, 1.0)
    return img


def completion_mask(m: int, n: int, observed: float = 0.3, seed: int = 17) -> np.ndarray:
    """(m, n) uint8 mask, 1 = observed pixel, each independently with
    probability `observed` (0.3: 70 % of the pixels removed)."""
    return (uniform(seed, m * n).reshape(m, n) < observed).astype(np.uint8)


def cur_index_sets(m: int, n: int, r: int, iters: int, seed: int = 18):
    """Row and column index sets of a rank-r cross approximation for each of
    `iters` completion iterations: (iters, r) int32 arrays I and J, each row
    r distinct indices drawn uniformly without replacement (the first r of a
    random permutation), sorted ascending.  Iteration t uses stream `seed`
    at offsets t << 33 (rows) and (t << 33) + (1 << 32) (columns)."""
    I = np.empty((iters, r), dtype=np.int32)
    J = np.empty((iters, r), dtype=np.int32)
    for t in range(iters):
        I[t] = np.sort(np.argsort(uniform(seed, m, t << 33), kind="stable")[:r])
        J[t] = np.sort(np.argsort(uniform(seed, n, (t << 33) + (1 << 32)), kind="stable")[:r])
    return I, J


# ------------------------------------------------- Lorenz signal filtering

def lorenz_trajectory(dt: float, t_end: float, y0=(1.0, 1.0, 1.0), sigma: float = 10.0, delta: float = 8.0 / 3.0,
                      gamma: float = 28.0, substeps: int = 10) -> np.ndarray:
    """Samples (u, v, w) of the Lorenz system du/dt = sigma (v - u),
    dv/dt = u (gamma - w) - v, dw/dt = u v - delta w at t = 0, dt, ..., t_end
    ((K + 1, 3) array), by the classical fourth-order Runge-Kutta method with
    `substeps` steps per sample (stands in for an adaptive ode45 run sampled at
    dt: the flow is chaotic, so two accurate integrators agree only up to
    t ~ 20 in any case)."""
    def rhs(y):
        u, v, w = y
        return np.array([sigma * (v - u), u * (gamma - w) - v, u * v - delta * w])
    K = int(round(t_end / dt))
    h = dt / substeps
    y = np.array(y0, dtype=np.float64)
    out = np.empty((K + 1, 3))
    out[0] = y
    for k in range(K):
        for _ in range(substeps):
            k1 = rhs(y)
            k2 = rhs(y + 0.5 * h * k1)
            k3 = rhs(y + 0.5 * h * k2)
            k4 = rhs(y + h * k3)
            y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        out[k + 1] = y
    return out


def lorenz_signals(dt: float = 0.01, tau: float = 1.0, t_end: float = 40.0, noise: float = 0.5, seed: int = 19):
    """Reference and observed quaternion signals of the filtering example:
    s_k = u(t_k) i + v(t_k) j + w(t_k) k and x_k = s(t_k - tau) + eta_k at
    t_k = tau + k dt, k = 0 .. N-1 (N = t_end / dt + 1), with eta_k purely
    imaginary, each component N(0, noise^2) (stream `seed`).  Returns
    (x, s), each (4, N) planes (zero real plane)."""
    d = int(round(tau / dt))
    N = int(round(t_end / dt)) + 1
    tr = lorenz_trajectory(dt, t_end + d * dt)
    x = np.zeros((4, N))
    s = np.zeros((4, N))
    s[1:] = tr[d:d + N].T
    x[1:] = tr[0:N].T + noise * normal(seed, 3 * N).reshape(3, N)
    return x, s


# ------------------------------------------- preconditioned Krylov systems

def reservoir_matrix(nx: int = 14, ny: int = 17, seed: int = 20, log_sd: float = 2.0, drift: float = 0.3,
                     storage: float = 1e-7) -> np.ndarray:
    """Real nonsymmetric (nx ny) x (nx ny) matrix standing in for saylr1
    (238 x 238, a 14 x 17 reservoir-simulation grid): 5-point finite-volume
    pressure operator with log-normal cell permeabilities (log standard
    deviation log_sd, stream `seed`), harmonic-mean transmissibilities T,
    an upwind drift term drift * T along x (the nonsymmetric part), and a
    small storage term storage * mean(k) on the diagonal (without it the
    no-flow operator is singular)."""
    n = nx * ny
    k = np.exp(log_sd * normal(seed, n))
    A = np.zeros((n, n))
    for iy in range(ny):
        for ix in range(nx):
            p = iy * nx + ix
            for q, along_x in ((p + 1, True) if ix + 1 < nx else (None, True), (p + nx, False) if iy + 1 < ny
                               else (None, False)):
                if q is None:
                    continue
                T = 2.0 * k[p] * k[q] / (k[p] + k[q])
                A[p, p] += T
                A[q, q] += T
                A[p, q] -= T
                A[q, p] -= T
                if along_x:  # upwind transport from p into q
                    A[q, p] -= drift * T
                    A[p, p] += drift * T
    A[np.arange(n), np.arange(n)] += storage * k.mean()
    return A


def krylov_system(m: int = 3, nx: int = 14, ny: int = 17, seed: int = 20):
    """The quaternion system of the preconditioning example: A = A_s + A_x i +
    A_y j + A_z k with A_x = -A_s, A_y = 2 A_s, A_z = 1.5 A_s (A_s from
    reservoir_matrix), and B (n x m) with every component uniform in [0, 1)
    (stream seed + 1).  Returns (A, B) as planes."""
    As = reservoir_matrix(nx, ny, seed)
    n = As.shape[0]
    A = np.stack([As, -As, 2.0 * As, 1.5 * As])
    B = uniform(seed + 1, 4 * n * m).reshape(4, n, m)
    return A, B
