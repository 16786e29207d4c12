"""Pins of the one-shot (sFFT-DT) oracle against facts that do not come from it: Theorem 1
(Eq. 11) written from the sparse truth, the closed-form singular values of a one-tone
bucket, the quadratic formula for the roots of P(z) (Eq. 12, method 1) of a two-tone
bucket, and exact recovery of the generator's truth on exactly sparse inputs.  The bins
come from the oracle's naive DFT bucketization, itself pinned in test_oracle_pins.py.
CPU only."""
import collections

import numpy as np
import pytest

import synth
from oracle import oneshot as dt

N, L = 4096, 16
B = N // L


def problem(K, seed, a_m=3, P=7, snr_db=None, support=None, values=None):
    rng = np.random.default_rng(seed)
    dl = synth.oneshot_delays(N, a_m, P, rng)
    p = synth.make_problem(N, (L,), K, seed=seed + 100, delays=dl, mag=(1.0, 10.0),
                           snr_db=snr_db, support=support, values=values)
    return p, dl


def test_hankel_identity_eq11(oracle_mod):
    """M_{a_m} = sum_j p_j zhat_j zhat_j^T with zhat_j = [z_j^0 .. z_j^{a_m-1}] (Theorem 1),
    exactly for an exactly sparse signal: checks the delay slots and the moment scale."""
    a_m = 3
    p, dl = problem(60, 1, a_m=a_m)
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    m = dt.moments(Y, B, a_m)
    for i in range(B):
        ref = np.zeros((a_m, a_m), dtype=np.complex128)
        for f, v in zip(p.support, p.values):
            if f % B == i:
                z = np.exp(2j * np.pi * f / N) ** np.arange(a_m)
                ref += v * np.outer(z, z)
        np.testing.assert_allclose(dt.hankel(m[i], a_m, a_m), ref, rtol=0, atol=1e-9)


def test_one_tone_singular_values(oracle_mod):
    """A bucket holding one tone p: M = p zhat zhat^T has the single nonzero singular value
    |p| ||zhat||^2 = a_m |p|."""
    a_m = 3
    p, dl = problem(1, 2, a_m=a_m, support=[1234], values=[3.0 - 4.0j])
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    sv = dt.singular_values(dt.moments(Y, B, a_m), a_m)
    i = 1234 % B
    np.testing.assert_allclose(sv[i], [a_m * 5.0, 0.0, 0.0], rtol=0, atol=1e-9)
    others = np.delete(sv, i, axis=0)
    assert np.max(others) < 1e-9


def test_two_tone_prony_roots_quadratic(oracle_mod):
    """For a = 2, P(z) = z^2 + c_1 z + c_0 has the roots (-c_1 -+ sqrt(c_1^2 - 4 c_0)) / 2
    (Sec. 3.1, method 1): they must be the two tones' z = e^{2 pi i f / N}, and the
    enumeration over the bucket's candidates must return the two frequencies."""
    f0, f1 = 77 + 3 * B, 77 + 11 * B
    p, dl = problem(2, 3, support=[f0, f1], values=[2.0 + 1.0j, -1.5 + 0.5j])
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    m = dt.moments(Y, B, 3)
    c = dt.prony_coefficients(m[77], 3, 2)
    disc = np.sqrt(c[1] ** 2 - 4 * c[0] + 0j)
    roots = sorted([(-c[1] - disc) / 2, (-c[1] + disc) / 2], key=np.angle)
    want = sorted([np.exp(2j * np.pi * f0 / N), np.exp(2j * np.pi * f1 / N)], key=np.angle)
    np.testing.assert_allclose(roots, want, rtol=0, atol=1e-9)
    np.testing.assert_array_equal(dt.enumerate_positions(N, B, 77, c), [f0, f1])


def test_subspace_pursuit_moves_position_by_b(oracle_mod):
    """Step 3's dictionary {f, f + B, f - B}: started from the wrong neighbour f + B, the
    pursuit returns the true frequency and value."""
    f = 500 + 5 * B
    p, dl = problem(1, 4, support=[f], values=[1.0 - 2.0j])
    Y = oracle_mod.bucketize(N, [L], dl, p.x).reshape(-1, B)
    y = Y[9:, f % B] / B
    fs, vs = dt.subspace_pursuit(N, B, [f + B], y, dl[0, 9:], tol2=1e-20, max_iter=8)
    np.testing.assert_array_equal(fs, [f])
    np.testing.assert_allclose(vs, [1.0 - 2.0j], rtol=0, atol=1e-9)


@pytest.mark.parametrize("a_m,P", [(2, 6), (3, 7)])
def test_exact_recovery_of_truth(oracle_mod, a_m, P):
    """Exactly sparse, at most a_m tones per bucket: the decoder returns the generator's
    support, values within FP64 rounding, and the vote gives each bucket its tone count."""
    K = 60
    for seed in range(10, 40):
        p, dl = problem(K, seed, a_m=a_m, P=P)
        if max(collections.Counter((p.support % B).tolist()).values()) <= a_m:
            break
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    res = dt.decode(N, B, K, dl, Y, dt.OneShotOpts(a_m=a_m))
    assert res.status == 0
    np.testing.assert_array_equal(res.idx, p.support)
    np.testing.assert_allclose(res.val, p.values, rtol=0, atol=1e-9)
    want = np.bincount(p.support % B, minlength=B)
    np.testing.assert_array_equal(res.counts, want)


def test_noisy_recovery_of_truth(oracle_mod):
    """30 dB: the support is the truth's and the values are within the noise level."""
    K = 40
    p, dl = problem(K, 51, snr_db=30.0)
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    res = dt.decode(N, B, K, dl, Y, dt.OneShotOpts(noise_var=p.noise_var))
    np.testing.assert_array_equal(res.idx, p.support)
    err = np.linalg.norm(res.val - p.values) / np.linalg.norm(p.values)
    assert err < 0.05, err


def test_delay_structure_is_checked():
    with pytest.raises(ValueError):
        dt.check_delays(N, 3, [0, 1, 2, 3, 4, 5, 6, 7, 8, 100, 200, 300, 400, 500, 600])
    rng = np.random.default_rng(0)
    with pytest.raises(ValueError):  # fewer than 2 a_m random delays
        dt.check_delays(N, 3, synth.oneshot_delays(N, 3, 5, rng))


# ---------------------------------------------------------------- Step 2, methods 1 and 3
def three_tone_bucket(seed):
    i = 77
    fs = [i + 2 * B, i + 7 * B, i + 12 * B]
    vals = [2.0 + 1.0j, -1.5 + 0.5j, 0.7 - 1.1j]
    p, dl = problem(3, seed, support=fs, values=vals)
    return p, dl, i, fs


@pytest.mark.parametrize("a", [1, 2, 3])
def test_method1_roots_are_the_tones(oracle_mod, a):
    """Method 1: in the exactly sparse case the a roots of P(z) = 0 (Eq. 12) are the bucket's
    z_j = e^{2 pi i f_j / N}, written here from the generator's support."""
    p, dl, i, fs = three_tone_bucket(5)
    if a < 3:
        p, dl = problem(a, 5, support=fs[:a], values=[2.0 + 1.0j, -1.5 + 0.5j][:a])
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    m = dt.moments(Y, B, 3)
    roots = dt.polynomial_roots(dt.prony_coefficients(m[i], 3, a))
    want = np.exp(2j * np.pi * np.array(fs[:a]) / N)
    np.testing.assert_allclose(sorted(roots, key=np.angle), sorted(want, key=np.angle),
                               rtol=0, atol=1e-9)
    np.testing.assert_array_equal(dt.snap_positions(N, B, i, roots), fs[:a])


@pytest.mark.parametrize("a", [2, 3])
def test_pencil_eigenvalues_theorem3(oracle_mod, a):
    """Method 3: the generalized eigenvalues of Y_2 - lambda Y_1 (Eq. 15-17) are conj(z_j),
    by the Vandermonde factors of Theorem 3.  Checked with scipy's QZ on the square top
    rows of the pencil, against the generator's z_j, and through the oracle's Y_1^+ Y_2."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    p, dl, i, fs = three_tone_bucket(6)
    if a < 3:
        p, dl = problem(a, 6, support=fs[:a], values=[2.0 + 1.0j, -1.5 + 0.5j][:a])
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    m = dt.moments(Y, B, 3)
    Y1, Y2 = dt.pencil(m[i], 3, a)
    assert Y1.shape == (a + 1, a) and Y2.shape == (a + 1, a)
    lam = scipy_linalg.eig(Y2[:a], Y1[:a], right=False)
    z = np.exp(2j * np.pi * np.array(fs[:a]) / N)
    np.testing.assert_allclose(sorted(lam, key=np.angle), sorted(z.conj(), key=np.angle),
                               rtol=0, atol=1e-9)
    pts = dt.pencil_points(m[i], 3, a)
    np.testing.assert_allclose(sorted(pts, key=np.angle), sorted(z, key=np.angle),
                               rtol=0, atol=1e-9)


@pytest.mark.parametrize("a", [1, 2, 3])
def test_pencil_svd_points_are_the_tones(oracle_mod, a):
    """Method 3 as sFFT-DT3.0 runs it (Sec. 4.1): the eigenvalues of V_1^+ V_2 from the right
    singular vectors of Eq. 15's Y are the generator's z_j (not their conjugates), and Y
    itself is U diag(p) U^H with U[r][j] = z_j^r, written here from the truth."""
    p, dl, i, fs = three_tone_bucket(7)
    vals = [2.0 + 1.0j, -1.5 + 0.5j, 0.7 - 1.1j][:a]
    if a < 3:
        p, dl = problem(a, 7, support=fs[:a], values=vals)
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    m = dt.moments(Y, B, 3)
    z = np.exp(2j * np.pi * np.array(fs[:a]) / N)
    U = np.stack([z ** r for r in range(a + 1)])
    np.testing.assert_allclose(dt.toeplitz_y(m[i], 3, a), U @ np.diag(vals) @ U.conj().T,
                               rtol=0, atol=1e-9)
    pts = dt.pencil_svd_points(m[i], 3, a)
    np.testing.assert_allclose(sorted(pts, key=np.angle), sorted(z, key=np.angle),
                               rtol=0, atol=1e-9)


def test_snap_positions_rule():
    """Points take candidates most confident first; a taken candidate sends the point to
    the nearest free one on its own side, and the index wraps modulo L."""
    i, Lc = 77, N // B

    def pt(u):
        return np.exp(2j * np.pi * (i + u * B) / N)

    got = dt.snap_positions(N, B, i, np.array([pt(5.3), pt(5.0), pt(4.6)]))
    np.testing.assert_array_equal(got, [i + 4 * B, i + 5 * B, i + 6 * B])
    got = dt.snap_positions(N, B, i, np.array([pt(Lc - 0.3)]))
    np.testing.assert_array_equal(got, [i])


@pytest.mark.parametrize("method", [1, 3])
@pytest.mark.parametrize("a_m,P", [(2, 6), (3, 7)])
def test_exact_recovery_methods_1_and_3(oracle_mod, method, a_m, P):
    """Methods 1 and 3 recover the generator's truth on exactly sparse inputs, like
    method 2."""
    K = 60
    for seed in range(10, 40):
        p, dl = problem(K, seed, a_m=a_m, P=P)
        if max(collections.Counter((p.support % B).tolist()).values()) <= a_m:
            break
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    res = dt.decode(N, B, K, dl, Y, dt.OneShotOpts(a_m=a_m, method=method))
    assert res.status == 0
    np.testing.assert_array_equal(res.idx, p.support)
    np.testing.assert_allclose(res.val, p.values, rtol=0, atol=1e-9)


@pytest.mark.parametrize("method", [1, 3])
def test_noisy_recovery_methods_1_and_3(oracle_mod, method):
    """30 dB: the support is the truth's for methods 1 and 3 too."""
    K = 40
    p, dl = problem(K, 51, snr_db=30.0)
    Y = oracle_mod.bucketize(N, [L], dl, p.x)
    res = dt.decode(N, B, K, dl, Y, dt.OneShotOpts(noise_var=p.noise_var, method=method))
    np.testing.assert_array_equal(res.idx, p.support)
