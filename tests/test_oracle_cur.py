"""Pins of the CUR image-completion oracle (Sec. 5.1) against facts that do
not come from it: the projection identity of CUR on exact low-rank
matrices, the fixed point of the impute-reconstruct loop, data
consistency, recovery of a low-rank image from half its pixels, and the
Gaussian filter against scipy's and its closed form.  Planted mistakes show
the pins bite."""
import math

import numpy as np
import pytest

import oracle
from oracle import cur
from paper_2605_01464_gb300 import inputs as I


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def low_rank(m, n, k, seed):
    return oracle.matmul(I.gaussian_quaternion(m, k, seed), I.gaussian_quaternion(k, n, seed + 1))


def check_weights():
    e = math.exp(-2.0)
    assert np.allclose(cur.gaussian_weights(0.5), np.array([e, 1.0, e]) / (1.0 + 2.0 * e), rtol=1e-15, atol=0)
    g = cur.gaussian_weights(1.0)
    assert g.size == 5 and abs(g.sum() - 1.0) <= 1e-15


def check_filter_scipy(sigma):
    ndimage = pytest.importorskip("scipy.ndimage")
    X = I.gaussian_quaternion(23, 31, 5)
    got = cur.gaussian_filter(X, sigma)
    # scipy: radius int(truncate * sigma + 0.5) = ceil(2 sigma) for these
    # sigmas with truncate = 2; 'nearest' replicates the border
    want = np.stack([ndimage.gaussian_filter(X[p], sigma, mode="nearest", truncate=2.0) for p in range(4)])
    assert np.max(np.abs(got - want)) <= 1e-14


def check_exact_rank(r, k, cross=False, tol=1e-11):
    A = low_rank(30, 44, k, 7)
    Is, Js = I.cur_index_sets(30, 44, r, 1, 8)
    X, infos = cur.cur_reconstruct(A, Is[0], Js[0], tol=1e-14, max_iter=300, cross=cross)
    assert rel(X, A) <= tol, rel(X, A)


def test_gaussian_weights_closed_form():
    check_weights()


@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.5])
def test_gaussian_filter_matches_scipy(sigma):
    check_filter_scipy(sigma)


def test_gaussian_filter_keeps_constant_planes():
    X = np.ones((4, 9, 13)) * np.array([0.0, 0.2, 0.5, 0.9])[:, None, None]
    assert np.allclose(cur.gaussian_filter(X, 0.5), X, rtol=0, atol=1e-15)


@pytest.mark.parametrize("r,k", [(3, 3), (5, 3)])
def test_exact_low_rank_reproduced(r, k):
    # C_J C_J^dagger A R_I^dagger R_I = A when C_J spans A's columns and R_I
    # its rows (r >= rank); with r > rank the pseudoinverses are of
    # rank-deficient matrices (plateau stop), accurate to about kappa^2 eps
    check_exact_rank(r, k, tol=1e-11 if r == k else 1e-8)


def test_cross_form_exact_low_rank():
    # A = C_J W^dagger R_I for rank(W) = rank(A) (the cross approximation)
    check_exact_rank(4, 4, cross=True)


def test_low_rank_image_is_a_fixed_point():
    A = low_rank(24, 36, 3, 11)
    mask = I.completion_mask(24, 36, 0.4, 12)
    Is, Js = I.cur_index_sets(24, 36, 5, 2, 13)
    C, _ = cur.cur_complete(A, mask, Is, Js, sigma=0.0, tol=1e-14, max_iter=300, x_init=A)
    assert rel(C, A) <= 1e-8


def test_observed_pixels_kept_exactly():
    A = I.synthetic_rgb_image(32, 48, 16)
    mask = I.completion_mask(32, 48, 0.3, 17)
    M = A.copy()
    M[:, mask == 0] = 7.0  # values at unobserved pixels are ignored
    Is, Js = I.cur_index_sets(32, 48, 6, 3, 18)
    C, hist = cur.cur_complete(M, mask, Is, Js, sigma=0.5)
    assert np.array_equal(C[:, mask != 0], A[:, mask != 0])
    assert len(hist) == 3 and all(h["status"] in ("converged", "plateau") for hs in hist for h in hs)


def test_half_observed_low_rank_image_is_recovered():
    A = low_rank(40, 56, 2, 1)
    mask = I.completion_mask(40, 56, 0.5, 3)
    miss = mask == 0
    errs = []
    for T in (30, 60):
        Is, Js = I.cur_index_sets(40, 56, 4, T, 4)
        C, _ = cur.cur_complete(A, mask, Is, Js, sigma=0.0)
        errs.append(np.linalg.norm((C - A)[:, miss]) / np.linalg.norm(A[:, miss]))
    assert errs[1] < 0.1 * errs[0] and errs[1] <= 1e-4, errs


def test_psnr_definition():
    A = np.zeros((4, 4, 4))
    B = A.copy()
    B[1:] += 0.1
    assert abs(cur.psnr(B, A) - 20.0) <= 1e-12
    assert cur.psnr(A, A) == math.inf


def test_planted_mistakes_are_caught(monkeypatch):
    # unnormalised filter weights: the scipy pin fails
    raw = cur.gaussian_weights
    monkeypatch.setattr(cur, "gaussian_weights", lambda s: raw(s) * 1.01)
    with pytest.raises(AssertionError):
        check_filter_scipy(0.5)
    monkeypatch.setattr(cur, "gaussian_weights", raw)
    # the adjoint in place of the pseudoinverse: the low-rank pin fails
    monkeypatch.setattr(cur, "pinv", lambda A, *a: (oracle.adjoint(A), {}))
    with pytest.raises(AssertionError):
        check_exact_rank(3, 3)


def test_optimal_form_improves_and_cross_form_diverges_on_smooth_image():
    # The evidence behind using U = C_J^+ C R_I^+ for completion: with index
    # sets drawn uniformly at random, the cross form's W^+ amplifies the
    # missing-pixel error every iteration, while the optimal form (a pair of
    # projections) improves on the masked image
    A = I.synthetic_rgb_image(64, 96, 16)
    mask = I.completion_mask(64, 96, 0.3, 17)
    Is, Js = I.cur_index_sets(64, 96, 10, 8, 18)
    M = A * mask
    Cx, _ = cur.cur_complete(M, mask, Is, Js, sigma=0.0, cross=True)
    Co, _ = cur.cur_complete(M, mask, Is, Js, sigma=0.0, cross=False)
    assert cur.psnr(Co, A) > cur.psnr(M, A) + 10.0
    assert cur.psnr(Cx, A) < cur.psnr(M, A)


def test_full_index_sets_reproduce_the_filled_matrix():
    # r = min(m, n) with every column chosen: C_J C_J^+ C R_I^+ R_I = C when
    # R_I has full column rank, so the loop returns its starting matrix
    A = I.synthetic_rgb_image(12, 8, 16)
    mask = I.completion_mask(12, 8, 0.5, 17)
    Is = np.array([[0, 2, 3, 5, 6, 8, 9, 11]] * 3, dtype=np.int32)
    Js = np.array([list(range(8))] * 3, dtype=np.int32)
    C, _ = cur.cur_complete(A * mask, mask, Is, Js, sigma=0.0, tol=1e-14, max_iter=500)
    assert rel(C, A * mask) <= 1e-10
