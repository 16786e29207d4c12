"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself:
numpy's FFT (a library routine for the special case B = N), closed forms (the aliasing
identity of Eq. 6 built straight from the sparse truth, Parseval), brute force, and the
paper's own N = 20 worked example (Sec. 3.2, Fig. 3-4).  CPU only."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def aliasing_bins(N, f, delays, support, values):
    """Eq. 6 / Eq. 19 written from the sparse truth with no DFT at all:
    Y_{d,r}[j] = B_d * sum_{k in supp, k = j mod B_d} xhat_k e^{+2 pi i k tau_r / N}."""
    out = []
    delays = np.asarray(delays).reshape(len(f), -1)
    for d, L in enumerate(f):
        B = N // L
        for tau in delays[d]:
            Y = np.zeros(B, dtype=np.complex128)
            for k, v in zip(support, values):
                ph = 2 * np.pi * ((int(k) * int(tau)) % N) / N
                Y[int(k) % B] += B * v * np.exp(1j * ph)
            out.append(Y)
    return np.concatenate(out)


# ---------------------------------------------------------------------------- dense DFT
@pytest.mark.parametrize("N", [1, 7, 20, 64, 255])
def test_dense_dft_matches_numpy(oracle_mod, N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    np.testing.assert_allclose(oracle_mod.dense_dft(x), np.fft.fft(x) / N, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,K", [(20, 5), (60, 4)])
def test_dense_dft_recovers_sparse_truth(oracle_mod, N, K):
    p = synth.make_problem(N, (N // 4, 4), K, seed=3)
    xhat = oracle_mod.dense_dft(p.x)
    want = np.zeros(N, dtype=np.complex128)
    want[p.support] = p.values
    np.testing.assert_allclose(xhat, want, atol=1e-12)


# ---------------------------------------------------------------------------- bucketization
@pytest.mark.parametrize("case", [
    dict(N=20, f=(5, 4), K=5, R=3, delays="ffast"),
    dict(N=60, f=(3, 4, 5), K=4, R=4, delays="random"),
    dict(N=9660, f=(20, 21, 23), K=50, R=3, delays="ffast"),
    dict(N=9660, f=(20, 21, 23), K=30, R=6, delays="random"),
])
def test_aliasing_identity(oracle_mod, case):
    p = synth.make_problem(case["N"], case["f"], case["K"], seed=11, R=case["R"],
                           delays=case["delays"])
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    want = aliasing_bins(p.N, p.f, p.delays, p.support, p.values)
    scale = np.abs(want).max()
    np.testing.assert_allclose(Y, want, rtol=0, atol=1e-12 * scale)


def test_aliasing_identity_discriminates_sign(oracle_mod):
    """The pin above fails for the paper's delay sign (phase e^{-2 pi i k tau/N}): it
    distinguishes the advance/delay conventions and cannot pass by accident."""
    p = synth.make_problem(60, (3, 4, 5), 4, seed=5, R=4, delays="random")
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    wrong = aliasing_bins(p.N, p.f, (-p.delays) % p.N, p.support, p.values)
    assert np.abs(Y - wrong).max() > 1e-3 * np.abs(wrong).max()


def test_bucketize_full_dft_special_case(oracle_mod):
    """One stage with L = 1 (B = N): bucketization is the unnormalised DFT of the advanced
    signal, i.e. numpy.fft.fft(roll(x, -tau))."""
    rng = np.random.default_rng(2)
    N = 96
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    delays = np.array([[0, 1, 5, 77]])
    Y = oracle_mod.bucketize(N, (1,), delays, x).reshape(4, N)
    for r, tau in enumerate(delays[0]):
        np.testing.assert_allclose(Y[r], np.fft.fft(np.roll(x, -tau)), atol=1e-11)


def test_bucketize_parseval(oracle_mod):
    """sum_j |Y_j|^2 = B sum_m |y_m|^2 for every (stage, delay), on a dense random signal."""
    rng = np.random.default_rng(4)
    N, f = 630, (9, 10, 7)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    delays = np.array([[0, 1, 17], [0, 1, 400], [0, 1, 629]])
    Y = oracle_mod.bucketize(N, f, delays, x)
    off = 0
    for d, L in enumerate(f):
        B = N // L
        for tau in delays[d]:
            y = x[(np.arange(B) * L + tau) % N]
            e = np.sum(np.abs(Y[off:off + B]) ** 2)
            assert e == pytest.approx(B * np.sum(np.abs(y) ** 2), rel=1e-12)
            off += B


def test_bin_value_matches_bucketize(oracle_mod):
    p = synth.make_problem(9660, (20, 21, 23), 20, seed=8, R=3, delays="random")
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    off = 0
    for d, L in enumerate(p.f):
        B = p.N // L
        for r, tau in enumerate(p.delays[d]):
            for j in (0, 1, B // 2, B - 1):
                v = oracle_mod.bin_value(p.N, L, int(tau), j, p.x)
                assert abs(v - Y[off + j]) <= 1e-9 * max(1.0, abs(Y[off + j]))
            off += B


# ---------------------------------------------------------------------------- decoding
def test_paper_worked_example_n20(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "ffast_n20_example.json")))
    rng = np.random.default_rng(20)
    vals = np.exp(1j * rng.uniform(0, 2 * np.pi, len(g["support"])))
    p = synth.make_problem(g["N"], g["f"], 0, seed=0, R=3, delays="ffast",
                           support=g["support"], values=vals)
    assert p.B == tuple(g["B"])
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    res = oracle_mod.decode(p.N, p.f, p.delays, Y, K=5,
                            opts=oracle_mod.OracleOpts(locate=0))
    log = res["round_log"]
    assert int(log["n_zero"][0]) == g["round1_classes"]["zero"]
    assert int(log["n_single"][0]) == g["round1_classes"]["single"]
    assert int(log["n_multi"][0]) == g["round1_classes"]["multi"]
    assert list(map(int, log["idents"])) == g["identifications_per_round"]
    assert res["idents"] == g["identifications_total"]
    assert res["rounds"] == 3 and res["status"] == 0
    assert list(res["idx"]) == g["support"]
    np.testing.assert_allclose(res["val"], vals, atol=1e-12)


@pytest.mark.parametrize("locate", [0, 1])
def test_ffast_exact_recovery_9660(oracle_mod, locate):
    """Config ffast_exact_9660 (N = 20*21*23, K = 50, delays {0,1,2}): exact recovery of
    the generator's truth, values to 1e-12, with both locate rules."""
    p = synth.config_problem("ffast_exact_9660", seed=1)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    res = oracle_mod.decode(p.N, p.f, p.delays, Y, K=p.K,
                            opts=oracle_mod.OracleOpts(locate=locate))
    assert res["status"] == 0
    np.testing.assert_array_equal(res["idx"], p.support)
    np.testing.assert_allclose(res["val"], p.values, rtol=0, atol=1e-12)


def test_random_delay_ml_exact_recovery(oracle_mod):
    """R-FFAST shape (random delays, ML locate) on an exactly sparse signal."""
    p = synth.make_problem(124950, (49, 50, 51), 100, seed=9, R=6, delays="random",
                           mag=(1.0, 10.0))
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    res = oracle_mod.decode(p.N, p.f, p.delays, Y, K=p.K,
                            opts=oracle_mod.OracleOpts(locate=1))
    assert res["status"] == 0
    np.testing.assert_array_equal(res["idx"], p.support)
    np.testing.assert_allclose(res["val"], p.values, rtol=0, atol=1e-11)


def test_ml_locate_is_brute_force_over_candidates(oracle_mod):
    """A single tone anywhere in [0, N): ML locate returns its frequency.  N = 504 has
    L = 7, 8, 9 candidates per bin; every frequency of a stride is tried."""
    N, f = 504, (7, 8, 9)
    rng = np.random.default_rng(12)
    delays = synth.draw_delays(N, 3, 5, rng)
    for k in range(0, N, 37):
        v = 2.0 * np.exp(1j * rng.uniform(0, 2 * np.pi))
        x = synth.time_signal(N, [k], [v])
        Y = oracle_mod.bucketize(N, f, delays, x)
        res = oracle_mod.decode(N, f, delays, Y, K=1, opts=oracle_mod.OracleOpts(locate=1))
        assert list(res["idx"]) == [k]
        assert abs(res["val"][0] - v) < 1e-12


def test_kay_locate_every_frequency(oracle_mod):
    """KAY locate (Sec. 3.2 subproblem 2, Eq. 21-22) on structured delays r_c + t 2^c: a
    single tone at every frequency of N = 504 (L = 7, 8, 9; C = 4 iterations) is located
    exactly, for m = 2 and for m = 4 (where Eq. 22's weights must sum to one for the
    averaged phase to land on the tone's).  The L = 8 stage's last iteration (2^3 = 8) is
    the uninformative case whose bit comes from the bin index."""
    N, f = 504, (7, 8, 9)
    rng = np.random.default_rng(13)
    for m in (2, 4):
        delays = synth.kay_delays(N, 3, 4, m, rng)
        for k in range(N):
            v = 1.5 * np.exp(1j * rng.uniform(0, 2 * np.pi))
            x = synth.time_signal(N, [k], [v])
            Y = oracle_mod.bucketize(N, f, delays, x)
            res = oracle_mod.decode(N, f, delays, Y, K=1,
                                    opts=oracle_mod.OracleOpts(locate=2, kay_m=m))
            assert list(res["idx"]) == [k], (m, k)
            assert abs(res["val"][0] - v) < 1e-12


def test_kay_exact_recovery_124950(oracle_mod):
    """Exactly sparse, N = 49*50*51 with C = 6 iterations of m = 3 delays per stage: the
    peeling decoder with KAY locate returns the truth."""
    N, f = 124950, (49, 50, 51)
    dl = synth.kay_delays(N, 3, 6, 3, np.random.default_rng(3))
    p = synth.make_problem(N, f, 60, seed=4, delays=dl, mag=(1.0, 10.0))
    Y = oracle_mod.bucketize(N, f, dl, p.x)
    res = oracle_mod.decode(N, f, dl, Y, K=60, opts=oracle_mod.OracleOpts(locate=2, kay_m=3))
    assert res["status"] == 0
    np.testing.assert_array_equal(res["idx"], p.support)
    np.testing.assert_allclose(res["val"], p.values, rtol=0, atol=1e-11)


def test_kay_needs_enough_iterations(oracle_mod):
    """2^C must reach L: C = 5 iterations cannot tell L = 51 candidates apart."""
    N, f = 124950, (49, 50, 51)
    dl = synth.kay_delays(N, 3, 5, 2, np.random.default_rng(3))
    p = synth.make_problem(N, f, 10, seed=4, delays=dl)
    Y = oracle_mod.bucketize(N, f, dl, p.x)
    with pytest.raises(ValueError):
        oracle_mod.decode(N, f, dl, Y, K=10, opts=oracle_mod.OracleOpts(locate=2, kay_m=2))


def test_noisy_rffast_recovers_truth(oracle_mod):
    """General sparse case at 30 dB: every true frequency found, values within noise."""
    p = synth.make_problem(124950, (49, 50, 51), 60, seed=21, R=8, delays="random",
                           mag=(1.0, 10.0), snr_db=30.0)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    res = oracle_mod.decode(p.N, p.f, p.delays, Y, K=p.K,
                            opts=oracle_mod.OracleOpts(noise_var=p.noise_var, eta=1e-6,
                                                       locate=1))
    np.testing.assert_array_equal(res["idx"], p.support)
    err = np.linalg.norm(res["val"] - p.values) / np.linalg.norm(p.values)
    assert err < 0.05


def test_output_keeps_k_largest_sorted(oracle_mod):
    """Output rule (Sec. 2.1): the K largest recovered coefficients, sorted by frequency."""
    N, f = 9660, (20, 21, 23)
    rng = np.random.default_rng(30)
    support = np.sort(rng.choice(N, 12, replace=False))
    mags = np.arange(1, 13, dtype=float)
    rng.shuffle(mags)
    vals = mags * np.exp(1j * rng.uniform(0, 2 * np.pi, 12))
    p = synth.make_problem(N, f, 0, seed=0, R=3, support=support, values=vals)
    Y = oracle_mod.bucketize(N, f, p.delays, p.x)
    res = oracle_mod.decode(N, f, p.delays, Y, K=5, opts=oracle_mod.OracleOpts())
    keep = np.sort(support[np.argsort(-np.abs(vals))[:5]])
    np.testing.assert_array_equal(res["idx"], keep)
    assert len(res["rec_f"]) == 12


def test_same_frequency_in_two_stages_taken_once(oracle_mod):
    """A lone tone is a singleton in every stage in round 1; it is recovered once."""
    N, f = 9660, (20, 21, 23)
    p = synth.make_problem(N, f, 0, seed=0, R=3, support=[1234], values=[3 - 1j])
    Y = oracle_mod.bucketize(N, f, p.delays, p.x)
    res = oracle_mod.decode(N, f, p.delays, Y, K=4, opts=oracle_mod.OracleOpts())
    assert list(res["rec_f"]) == [1234]
    assert res["round_log"]["n_single"][0] == 3
    assert res["round_log"]["n_accepted"][0] == 1


def test_zero_signal_gives_empty_output(oracle_mod):
    N, f = 9660, (20, 21, 23)
    delays = np.tile(np.arange(3), (3, 1))
    Y = oracle_mod.bucketize(N, f, delays, np.zeros(N, dtype=np.complex128))
    res = oracle_mod.decode(N, f, delays, Y, K=10, opts=oracle_mod.OracleOpts())
    assert res["idx"].size == 0 and res["status"] == 0 and res["rounds"] == 1


# ------------------------------------------------------------- noise-variance estimate
def test_gamma_median_matches_library(oracle_mod):
    """The Gamma(R, 1) median the estimate divides by, against scipy's inverse of the
    regularised incomplete gamma function."""
    special = pytest.importorskip("scipy.special")
    for R in range(1, 17):
        assert abs(oracle_mod.gamma_median(R) - special.gammaincinv(R, 0.5)) < 1e-12


def test_noise_estimate_on_pure_noise(oracle_mod):
    """White noise of known sigma^2 at N = 49*50*51: every bin is a zero-ton, and the median
    estimate is within 2 % of sigma^2 (the median of 7500 Gamma draws has a relative
    spread near 0.6 %)."""
    N, f, R = 124950, (49, 50, 51), 8
    rng = np.random.default_rng(17)
    delays = synth.draw_delays(N, 3, R, rng)
    for var in (0.5, 3.0):
        x = synth.awgn(N, var, rng)
        Y = oracle_mod.bucketize(N, f, delays, x)
        est = oracle_mod.noise_estimate(N, f, R, Y)
        assert abs(est / var - 1.0) < 0.02, (var, est)


def test_noise_auto_decoding_recovers_truth(oracle_mod):
    """20 dB at N = 49*50*51 (K = 60 in 7500 bins): decoding with the estimated sigma^2
    returns the truth's support, like decoding with the true one."""
    p = synth.make_problem(124950, (49, 50, 51), 60, seed=23, R=8, delays="random",
                           mag=(1.0, 10.0), snr_db=20.0)
    Y = oracle_mod.bucketize(p.N, p.f, p.delays, p.x)
    res = oracle_mod.decode(p.N, p.f, p.delays, Y, K=p.K,
                            opts=oracle_mod.OracleOpts(locate=1, noise_auto=1))
    np.testing.assert_array_equal(res["idx"], p.support)
    assert abs(res["noise_var"] / p.noise_var - 1.0) < 0.1, (res["noise_var"], p.noise_var)


# ---------------------------------------------------------------------------- DSFFT
def test_dsfft_paper_worked_example(oracle_mod):
    """Sec. 3.3, Fig. 6: N = 64, tones at 1, 6, 13, 20, 59.  Starting from the root, the
    layers hold m_d = 1, 2, 4, 5 efficient nodes; the search stops at d = 3 with one
    frequency per node and returns the five tones."""
    from oracle import dsfft
    g = json.load(open(os.path.join(GOLDEN, "dsfft_n64_example.json")))
    N = g["N"]
    vals = np.exp(2j * np.pi * np.arange(5) / 5) * (1.0 + np.arange(5))
    x = synth.time_signal(N, g["support"], vals)
    res = dsfft.decode(N, 5, x, start_layer=0)
    assert res.layer_counts == g["layer_counts"]
    assert res.stop_layer == g["stop_layer"]
    assert res.status == 0
    np.testing.assert_array_equal(res.idx, g["support"])
    np.testing.assert_allclose(res.val, vals, rtol=0, atol=1e-12)
    Y = dsfft.layer_bins(x, N, 3)
    nodes = np.nonzero(np.abs(Y[:8]) > 1e-9)[0].tolist()
    assert nodes == g["efficient_nodes_of_stop_layer"]


def test_dsfft_layer_bins_are_aliasing_sums(oracle_mod):
    """Layer d's tau = 0 node i is B times the sum of xhat over f = i mod 2^d (Eq. 23), and
    its tau = 1 node carries e^{2 pi i f / N} per frequency (Eq. 6)."""
    from oracle import dsfft
    N, K, d = 1024, 9, 5
    p = synth.make_problem(N, (N >> d,), K, seed=41, delays=np.array([[0, 1]]), mag=(1.0, 3.0))
    Y = dsfft.layer_bins(p.x, N, d)
    np.testing.assert_allclose(Y, aliasing_bins(N, (N >> d,), [[0, 1]], p.support, p.values),
                               rtol=0, atol=1e-9)


def test_dsfft_exact_recovery(oracle_mod):
    """N = 2^16, K = 8 exactly sparse, starting at layer ceil(log2 K): the truth."""
    from oracle import dsfft
    N, K = 1 << 16, 8
    p = synth.make_problem(N, (1,), K, seed=43, delays=np.array([[0, 1]]), mag=(1.0, 10.0))
    res = dsfft.decode(N, K, p.x, start_layer=3)
    assert res.status == 0
    np.testing.assert_array_equal(res.idx, p.support)
    np.testing.assert_allclose(res.val, p.values, rtol=0, atol=1e-10)
    assert res.layer_counts[-1] == K
