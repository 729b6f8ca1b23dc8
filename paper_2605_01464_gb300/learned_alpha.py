"""Dataset, labels and evaluation for the learned initial scaling alpha.

The network itself (features, forward, backward, Adam) runs in libqpinv's
kernels; this module only builds training matrices with known spectra from
the seeded generators, computes labels, and drives the C ABI.

Families (the workloads' generators at smaller sizes):
  dense      -- Gaussian quaternion m x n (spectrum from LAPACK on the
                complex representation, used for the label only);
  logspaced  -- U diag(sigma) V^H, sigma log-spaced from 1 to 10^-u;
  geometric  -- rank r < min(m, n), sigma geometric from 1 to 10^-u;
  clustered  -- sigma drawn around 2-4 cluster centres (held-out mix).
Label: y = log(alpha* theta_1), alpha* = 2 / (sigma_1^2 + sigma_r^2) the
minimiser of Thm. 1's max |1 - alpha sigma_i^2|, theta_1 the features'
Lanczos estimate of sigma_1^2 (so alpha = exp(y) / theta_1), scaled down by
1.1 so that most predictions clear the solver's contraction check.
"""
import math

import numpy as np

from . import inputs

MARGIN = 1.1
TRAIN_FAMILIES = ("dense", "logspaced", "geometric")
HELDOUT_FAMILIES = ("logspaced", "geometric", "clustered")


def _spectrum(family, r, rng):
    u = rng.uniform(1.0, 8.0)
    if family == "logspaced":
        return np.logspace(0.0, -u, r)
    if family == "geometric":
        return np.geomspace(1.0, 10.0 ** -u, r)
    centres = 10.0 ** -rng.uniform(0.0, u, size=rng.integers(2, 5))
    centres[0] = 1.0
    s = centres[rng.integers(0, len(centres), size=r)] * np.exp(rng.normal(0.0, 0.05, size=r))
    return np.sort(s)[::-1] / s.max()


def sample_matrix(family, m, n, seed, device="cpu"):
    """(A planes (4, m, n), nonzero singular values descending)."""
    rng = np.random.default_rng(seed)
    if family == "dense":
        # singular values from the Hermitian eigenvalues of chi(A)^H chi(A) on
        # the smaller side (each quaternion singular value appears twice)
        A = inputs.gaussian_quaternion(m, n, seed)
        C = inputs.chi(A)
        G = C.conj().T @ C if n <= m else C @ C.conj().T
        ev = np.sort(np.linalg.eigvalsh(G))[::-1][::2]
        return A, np.sqrt(np.maximum(ev, 0.0))
    k = min(m, n)
    r = k if family != "geometric" else int(rng.integers(max(1, k // 4), max(2, k // 2) + 1))
    sigma = _spectrum(family, r, rng) * 10.0 ** rng.uniform(-2, 2)
    U = inputs.orthonormal_columns(m, r, 2 * seed + 1, device)
    V = inputs.orthonormal_columns(n, r, 2 * seed + 2, device)
    return inputs.with_spectrum(U, sigma, V, device), sigma


def heldout_matrix(family, m, n, seed, device="cpu", umax=5.0):
    """Full-rank held-out matrix (4, m, n) and its singular values: kappa =
    10^u, u ~ U[1, umax]; sigma log-uniform random draws ("logspaced"),
    geometric, or clustered around 2-4 centres; overall scale 10^U[-2, 2]."""
    rng = np.random.default_rng(seed)
    k = min(m, n)
    u = rng.uniform(1.0, umax)
    if family == "logspaced":
        sigma = np.sort(10.0 ** -rng.uniform(0.0, u, size=k))[::-1]
        sigma[0], sigma[-1] = 1.0, 10.0 ** -u
    elif family == "geometric":
        sigma = np.geomspace(1.0, 10.0 ** -u, k)
    else:
        centres = 10.0 ** -rng.uniform(0.0, u, size=rng.integers(2, 5))
        centres[0], centres[-1] = 1.0, 10.0 ** -u
        sigma = np.sort(centres[rng.integers(0, len(centres), size=k)] * np.exp(rng.normal(0.0, 0.05, size=k)))[::-1]
        sigma[0] = max(sigma[0], 1.0)
    sigma = sigma * 10.0 ** rng.uniform(-2, 2)
    U = inputs.orthonormal_columns(m, k, 2 * seed + 1, device)
    V = inputs.orthonormal_columns(n, k, 2 * seed + 2, device)
    return inputs.with_spectrum(U, sigma, V, device), sigma


def optimal_alpha(sigma):
    s = np.asarray(sigma, dtype=np.float64)
    s = s[s > 0]
    return 2.0 / (s.max() ** 2 + s.min() ** 2)


def make_dataset(ctx, count, lo, hi, seed, families=TRAIN_FAMILIES, device="cpu", to_device=None):
    """Features (count x 32), labels (count) and per-sample (family, m, n, theta_1)."""
    rng = np.random.default_rng(seed)
    feats, labels, meta = [], [], []
    for t in range(count):
        fam = families[t % len(families)]
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1)) if rng.uniform() < 0.5 else m
        A, sigma = sample_matrix(fam, m, n, seed * 100003 + t, device)
        Ad = to_device(A) if to_device else A
        f, theta1 = ctx.alpha_features(Ad)
        feats.append(f)
        labels.append(math.log(optimal_alpha(sigma) * theta1 / MARGIN))
        meta.append((fam, m, n, theta1))
    return np.array(feats, dtype=np.float32), np.array(labels, dtype=np.float32), meta


def compare_iterations(ctx, mats, method="qhpi19", tol=1e-12, to_device=None):
    """Solves every matrix with the safe and the learned alpha; returns a list
    of (iters_safe, iters_learned, E1rel_safe, E1rel_learned, alpha_source,
    precision_safe, precision_learned)."""
    out = []
    for A in mats:
        Ad = to_device(A) if to_device else A
        ctx.configure(alpha="safe")
        _, s = ctx.solve(Ad, method, tol=tol)
        ctx.configure(alpha="learned")
        _, l = ctx.solve(Ad, method, tol=tol)
        out.append((s["iters"], l["iters"], s["E_rel"][0], l["E_rel"][0], l["alpha_source"], s["precision"],
                    l["precision"]))
    ctx.configure(alpha="safe")
    return out


# ------------------------------------------------- GPU batch generator (training sets)
# Training sets of tens of thousands of matrices are drawn in groups of one
# shape on the GPU (torch's seeded generator, complex64 chi form): Haar-like
# orthonormal factors by CholeskyQR2, A = U diag(sigma) V^H.  Their spectra
# are exact to FP32 (about 1e-6 relative), ample for labels whose target is
# alpha to a few per cent; the held-out matrices keep the seeded FP64
# generators above.

def _chi_t(torch, Q):
    """(b, 4, m, n) real planes -> (b, 2m, 2n) complex chi form."""
    s, x, y, z = Q.unbind(1)
    b, m, n = s.shape
    C = torch.empty((b, 2 * m, 2 * n), dtype=torch.complex64, device=Q.device)
    C[:, 0::2, 0::2] = torch.complex(s, x)
    C[:, 0::2, 1::2] = torch.complex(y, z)
    C[:, 1::2, 0::2] = torch.complex(-y, z)
    C[:, 1::2, 1::2] = torch.complex(s, -x)
    return C


def _unchi_t(torch, C):
    a, b = C[:, 0::2, 0::2], C[:, 0::2, 1::2]
    return torch.stack([a.real, a.imag, b.real, b.imag], dim=1)


def _orth_t(torch, b, m, r, gen):
    """Orthonormal columns by shifted CholeskyQR3 in FP32: the first Gram gets
    a small diagonal shift (a square Gaussian factor is occasionally too
    ill-conditioned for an FP32 Cholesky; the shift keeps the chi structure),
    two unshifted passes restore orthonormality."""
    C = _chi_t(torch, torch.randn((b, 4, m, r), generator=gen, device=gen.device, dtype=torch.float32))
    for it in range(3):
        H = C.mH @ C
        H = 0.5 * (H + H.mH)
        if it == 0:
            d = H.diagonal(dim1=-2, dim2=-1).real.mean(-1)
            H = H + (1e-4 * d)[:, None, None] * torch.eye(H.shape[-1], dtype=H.dtype, device=H.device)
        L = torch.linalg.cholesky(H)
        C = torch.linalg.solve_triangular(L, C.mH, upper=False).mH
    return C


def sample_group_gpu(torch, family, m, n, count, gen):
    """`count` matrices of one shape: ((count, 4, m, n) float64 planes on the
    GPU, list of nonzero singular values per matrix, descending)."""
    import numpy as np
    k = min(m, n)
    if family == "dense":
        A = torch.randn((count, 4, m, n), generator=gen, device=gen.device, dtype=torch.float32)
        C = _chi_t(torch, A)
        G = C.mH @ C if n <= m else C @ C.mH
        ev = torch.linalg.eigvalsh(0.5 * (G + G.mH)).flip(-1)[:, ::2].clamp_min(0).sqrt()
        return A.double(), [e.cpu().numpy().astype(np.float64) for e in ev]
    rng = np.random.default_rng(int(torch.randint(0, 2 ** 31 - 1, (1,), generator=gen, device=gen.device).item()))
    r = k if family != "geometric" else int(rng.integers(max(1, k // 4), max(2, k // 2) + 1))
    sig = np.stack([_spectrum(family, r, rng) * 10.0 ** rng.uniform(-2, 2) for _ in range(count)])
    U = _orth_t(torch, count, m, r, gen)
    V = _orth_t(torch, count, n, r, gen)
    s2 = torch.as_tensor(np.repeat(sig, 2, axis=1), dtype=torch.float32, device=gen.device)
    A = _unchi_t(torch, (U * s2[:, None, :].to(torch.complex64)) @ V.mH)
    return A.double(), list(sig)


def make_dataset_gpu(ctx, torch, count, lo, hi, seed, families=TRAIN_FAMILIES, group=32):
    """Features (count x 32), labels (count) and per-sample (family, m, n,
    theta_1) for `count` matrices in groups of one shape; features by the
    library's kernels, labels as make_dataset."""
    import numpy as np
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    feats, labels, meta = [], [], []
    g = 0
    while len(feats) < count:
        fam = families[g % len(families)]
        g += 1
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1)) if rng.uniform() < 0.5 else m
        if fam == "dense":  # spectra from a Gram eigensolve: kept to the smaller sizes
            m, n = min(m, 256), min(n, 256)
        cnt = min(group, count - len(feats))
        A, sigs = sample_group_gpu(torch, fam, m, n, cnt, gen)
        for b in range(cnt):
            f, theta1 = ctx.alpha_features(A[b].contiguous())
            feats.append(f)
            labels.append(math.log(optimal_alpha(sigs[b]) * theta1 / MARGIN))
            meta.append((fam, m, n, theta1))
    return np.array(feats, dtype=np.float32), np.array(labels, dtype=np.float32), meta
