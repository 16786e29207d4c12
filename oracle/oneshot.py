"""sFFT-DT one-shot decoder (Sec. 3.1, Eq. 7-18; Sec. 4.1, Stage 2), plain FP64 numpy.

TEST INFRASTRUCTURE ONLY: the CUDA library never imports this module; tests, smoke() and
the benchmark's CPU baseline do.  Library primitives serve as single steps (numpy's SVD
for the singular values of Step 1, its linear solve for Eq. 14, its least squares for the
fits of Step 3); everything else is written out in the paper's order.

One stage of B buckets (L = N / B candidates per bucket).  Delay slots:
  r = 0 .. 3 a_m - 1      tau = r - a_m (mod N): the consecutive set {-a_m, ..., 2 a_m - 1}
  r = 3 a_m .. R - 1      the P random delays of Step 3 (P = R - 3 a_m)
The bins Y[r][i] of bucket i (any bucketization, e.g. oracle.bucketize) give the moments
m_k = Y[k + a_m][i] / B = sum_{f = i mod B} xhat_f z_f^k with z_f = e^{2 pi i f / N} (Eq. 7-8).

Per bucket, in the paper's order:
  Step 1  singular values of the a_m x a_m Hankel matrix M_{a_m} = [m_{r+c}] (Eq. 10-11);
          all B a_m of them vote: the K largest (above a noise floor) give each bucket its
          count a of significant frequencies.
  Step 2  the a positions, by one of the paper's three methods:
          method 1 (polynomial): C = M_a^{-1} M_s (Eq. 13-14); the a roots of
            P(z) = z^a + sum c_t z^t (Eq. 12) are the z_j;
          method 2 (enumeration, the default): P(z) evaluated at every candidate
            z = e^{2 pi i (i + q B) / N}, q < L; the a smallest |P(z)| give the positions;
          method 3 (matrix pencil, as sFFT-DT3.0 runs it in Sec. 4.1): the SVD
            Y = U S V^H of the (a + 1) x (a + 1) Toeplitz matrix of Eq. 15; with V_s the
            right singular vectors of the a largest singular values, V_1 = V_s without its
            last row and V_2 = V_s without its first row, the eigenvalues of V_1^+ V_2 are
            the z_j (the matrix pencil of Hua and Sarkar on the signal subspace: Y =
            U_{a+1} diag(p) U_{a+1}^H, so V_s spans the Vandermonde columns).  The direct
            pencil of Theorem 3, Y_2 - lambda Y_1 (Eq. 16-17), has eigenvalues
            conj(z_j) = 1 / z_j (pencil_points, pinned but not used by decode).
          Methods 1 and 3 give points z; each becomes a position by its angle, snapped to
          the nearest candidate i + q B (snap_positions).
  Step 3  values by subspace pursuit on Eq. 18 with the P random-delay measurements: the
          dictionary holds, for each position f, the atoms f, f + B and f - B; each pass
          adds the a atoms most correlated with the residual, fits the union by least
          squares, keeps the a largest coefficients and refits; it stops when the residual
          is within the noise tolerance, stops shrinking, or after max_iter passes.
Readings where the paper is silent (also listed in the design notes): the vote keeps the
K largest singular values that exceed sigma_floor = a_m sqrt(c0 B sigma^2 + (eta B a_min)^2)
/ B (the per-delay zero-ton level of a bucket, in moment units, times the largest singular
value a single tone of that level gives); ties at the K-th value all pass; the residual
tolerance of Step 3 is P (c1 sigma^2 / B + (eta a_min)^2); at most 8 passes.  Methods 1 and
3 snap the roots most confident first (smallest distance to a candidate); a root whose
candidate is taken moves to the nearest free one, on its own side first.

Parity pins (tests/test_oracle_pins.py): the Hankel identity of Eq. 11 on exact bins, the
closed-form singular values of a one-tone bucket, the quadratic roots of P(z) for a two-tone
bucket, subspace pursuit moving a position off by B back to the true one, and exact
recovery (support and values against the generator's truth) on exactly sparse inputs.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class OneShotOpts:
    a_m: int = 3
    noise_var: float = 0.0
    a_min: float = 1.0
    eta: float = 1e-6
    c0: float = 4.0
    c1: float = 2.0
    max_iter: int = 8
    method: int = 2      # Step 2: 1 polynomial roots, 2 enumeration, 3 matrix pencil (SVD)


def check_delays(N: int, a_m: int, delays) -> None:
    """The delay slots must start with {-a_m, ..., 2 a_m - 1} mod N (Sec. 4.1, Stage 1) and
    hold at least 2 a_m random delays after them (Step 3 fits up to 2 a atoms)."""
    d = [int(t) for t in np.asarray(delays).ravel()]
    if d[:3 * a_m] != [(k - a_m) % N for k in range(3 * a_m)]:
        raise ValueError("delay slots 0 .. 3 a_m - 1 must be -a_m .. 2 a_m - 1 mod N")
    if len(d) - 3 * a_m < 2 * a_m or len(set(d)) != len(d):
        raise ValueError("need at least 2 a_m distinct random delays")


def moments(Y: np.ndarray, B: int, a_m: int) -> np.ndarray:
    """m[i, k + a_m] = Y[k + a_m][i] / B for k = -a_m .. 2 a_m - 1 (Eq. 7-8)."""
    R = Y.size // B
    Yr = Y.reshape(R, B)
    return (Yr[:3 * a_m] / B).T.copy()


def hankel(m_row: np.ndarray, a_m: int, a: int) -> np.ndarray:
    """[m_{r+c}]_{r,c<a} of one bucket (Eq. 10 with a = a_m, Eq. 13 with a < a_m); m_row is
    indexed k + a_m."""
    return np.array([[m_row[r + c + a_m] for c in range(a)] for r in range(a)])


def singular_values(m: np.ndarray, a_m: int) -> np.ndarray:
    """Step 1: the a_m singular values of every bucket's M_{a_m}, descending [B, a_m]."""
    H = np.stack([hankel(m[i], a_m, a_m) for i in range(m.shape[0])])
    return np.linalg.svd(H, compute_uv=False)


def sv_floor(N: int, B: int, opts: OneShotOpts) -> float:
    s2 = opts.c0 * B * opts.noise_var + (opts.eta * B * opts.a_min) ** 2
    return opts.a_m * np.sqrt(s2) / B


def vote(sv: np.ndarray, K: int, floor: float) -> np.ndarray:
    """Counts a_i: the bucket's singular values among the K largest of all buckets that
    exceed floor (values equal to the K-th largest all pass)."""
    flat = sv.ravel()
    ok = flat > floor
    if not np.any(ok):
        return np.zeros(sv.shape[0], dtype=np.int64)
    vals = np.sort(flat[ok])[::-1]
    theta = vals[min(K, vals.size) - 1]
    sel = (sv >= theta) & (sv > floor)
    return sel.sum(axis=1).astype(np.int64)


def prony_coefficients(m_row: np.ndarray, a_m: int, a: int) -> np.ndarray:
    """Eq. 14: C = M_a^{-1} M_s with M_s = -[m_a, ..., m_{2a-1}]; returns c_0 .. c_{a-1}."""
    Ma = hankel(m_row, a_m, a)
    Ms = -np.array([m_row[a + t + a_m] for t in range(a)])
    return np.linalg.solve(Ma, Ms)


def poly_abs(c: np.ndarray, z: np.ndarray) -> np.ndarray:
    """|P(z)| of Eq. 12 with P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0."""
    a = c.size
    p = np.ones_like(z)
    for t in range(a - 1, -1, -1):
        p = p * z + c[t]
    return np.abs(p)


def enumerate_positions(N: int, B: int, i: int, c: np.ndarray) -> np.ndarray:
    """Step 2, method 2: the a candidates f = i + q B with the smallest |P(e^{2 pi i f/N})|
    (lower q first on ties)."""
    L = N // B
    f = i + B * np.arange(L, dtype=np.int64)
    z = np.exp(2j * np.pi * f / N)
    v = poly_abs(c, z)
    order = np.lexsort((np.arange(L), v))
    return np.sort(f[order[:c.size]])


def polynomial_roots(c: np.ndarray) -> np.ndarray:
    """Step 2, method 1: the a roots of P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0 (Eq. 12)."""
    return np.roots(np.concatenate(([1.0 + 0j], c[::-1])))


def pencil(m_row: np.ndarray, a_m: int, a: int):
    """Y_1 and Y_2 of Eq. 16-17, (a + 1) x a: Y_1[r][c] = m_{r-c}, Y_2[r][c] = m_{r-c-1};
    m_row is indexed k + a_m."""
    Y1 = np.array([[m_row[r - c + a_m] for c in range(a)] for r in range(a + 1)])
    Y2 = np.array([[m_row[r - c - 1 + a_m] for c in range(a)] for r in range(a + 1)])
    return Y1, Y2


def pencil_points(m_row: np.ndarray, a_m: int, a: int) -> np.ndarray:
    """Step 2, method 3: the eigenvalues lambda_j of Y_1^+ Y_2 (Theorem 3, rank a) are
    1 / z_j; returns the z_j."""
    Y1, Y2 = pencil(m_row, a_m, a)
    lam = np.linalg.eigvals(np.linalg.pinv(Y1) @ Y2)
    lam = np.where(lam == 0, 1.0 + 0j, lam)  # a zero eigenvalue carries no angle: take z = 1
    return 1.0 / lam


def toeplitz_y(m_row: np.ndarray, a_m: int, a: int) -> np.ndarray:
    """Y of Eq. 15, (a + 1) x (a + 1): Y[r][c] = m_{r-c}; m_row is indexed k + a_m."""
    return np.array([[m_row[r - c + a_m] for c in range(a + 1)] for r in range(a + 1)])


def pencil_svd_points(m_row: np.ndarray, a_m: int, a: int) -> np.ndarray:
    """Step 2, method 3 as Sec. 4.1 runs it: V_s = the right singular vectors of the a
    largest singular values of Y (Eq. 15); the eigenvalues of V_1^+ V_2 (V_1: V_s without
    its last row, V_2: without its first) are the z_j."""
    _, _, vh = np.linalg.svd(toeplitz_y(m_row, a_m, a))
    vs = vh.conj().T[:, :a]
    return np.linalg.eigvals(np.linalg.pinv(vs[:-1]) @ vs[1:])


def snap_positions(N: int, B: int, i: int, z: np.ndarray) -> np.ndarray:
    """Positions of the points z (methods 1 and 3): u = ((arg z) N / (2 pi) - i) / B mod L
    is the fractional candidate index; the points take candidates in order of increasing
    |u - round(u)|, each the nearest q not yet taken (round(u), then alternately one step
    further on u's side and on the other side).  Returns the positions ascending."""
    L = N // B
    u = ((np.angle(z) * N / (2 * np.pi) - i) / B) % L
    q0 = np.floor(u + 0.5)
    err = np.abs(u - q0)
    taken = []
    for t in np.argsort(err, kind="stable"):
        side = 1 if u[t] >= q0[t] else -1
        q = int(q0[t]) % L
        k = 0
        while q in taken and k < 2 * L - 1:  # (the bound only matters when L < a)
            k += 1
            step = (k + 1) // 2 * (side if k % 2 == 1 else -side)
            q = (int(q0[t]) + step) % L
        taken.append(q)
    return np.sort(i + B * np.array(taken, dtype=np.int64))


def atoms(N: int, freqs, taus) -> np.ndarray:
    """Columns e^{2 pi i (f tau mod N) / N} over the measurement delays (Eq. 18)."""
    taus = np.asarray(taus, dtype=np.int64)
    cols = [np.exp(2j * np.pi * ((int(f) * taus) % N) / N) for f in freqs]
    return np.stack(cols, axis=1) if cols else np.zeros((taus.size, 0), dtype=np.complex128)


def subspace_pursuit(N: int, B: int, pos, y: np.ndarray, taus, tol2: float, max_iter: int):
    """Step 3: values of the a positions by subspace pursuit over the 3a-atom dictionary
    {f, f + B, f - B}.  Returns (frequencies, values) of the final support."""
    a = len(pos)
    dic = []
    for f in pos:
        for s in (0, B, -B):
            g = (int(f) + s) % N
            if g not in dic:
                dic.append(g)
    Dm = atoms(N, dic, taus)

    def fit(sup):
        A = Dm[:, sup]
        p, *_ = np.linalg.lstsq(A, y, rcond=None)
        r = y - A @ p
        return p, float(np.vdot(r, r).real), r

    S = [dic.index(int(f)) for f in pos]
    p, res, r = fit(S)
    for _ in range(max_iter):
        if res <= tol2:
            break
        corr = np.abs(Dm.conj().T @ r)
        extra = [k for k in np.lexsort((np.arange(len(dic)), -corr)) if k not in S][:a]
        T = S + extra
        pT, _, _ = fit(T)
        keep = np.lexsort((np.arange(len(T)), -np.abs(pT)))[:a]
        S2 = [T[k] for k in sorted(keep)]
        p2, res2, r2 = fit(S2)
        if res2 >= res:
            break
        S, p, res, r = S2, p2, res2, r2
    return np.array([dic[k] for k in S], dtype=np.int64), p


@dataclasses.dataclass
class OneShotResult:
    idx: np.ndarray
    val: np.ndarray
    counts: np.ndarray   # a_i per bucket (Step 1)
    status: int          # 0, or 2 when a voted bucket's Eq. 14 was singular (methods 1, 2)
    n_recovered: int


def decode(N: int, B: int, K: int, delays, Y: np.ndarray, opts: OneShotOpts) -> OneShotResult:
    """The whole Stage 2 of the one-shot framework on one stage's bins Y [R][B] (natural
    order), then the output rule of Sec. 2.1 (sorted, the K largest)."""
    a_m = opts.a_m
    delays = np.asarray(delays, dtype=np.int64).ravel()
    check_delays(N, a_m, delays)
    R = delays.size
    Pn = R - 3 * a_m
    m = moments(Y, B, a_m)
    sv = singular_values(m, a_m)
    counts = vote(sv, K, sv_floor(N, B, opts))
    Yr = Y.reshape(R, B)
    taus = delays[3 * a_m:]
    tol2 = Pn * (opts.c1 * opts.noise_var / B + (opts.eta * opts.a_min) ** 2)
    fs, vs, status = [], [], 0
    for i in np.nonzero(counts)[0]:
        a = int(counts[i])
        if opts.method == 3:
            pos = snap_positions(N, B, int(i), pencil_svd_points(m[i], a_m, a))
        else:
            try:
                c = prony_coefficients(m[i], a_m, a)
            except np.linalg.LinAlgError:
                status = 2
                continue
            if opts.method == 1:
                pos = snap_positions(N, B, int(i), polynomial_roots(c))
            else:
                pos = enumerate_positions(N, B, int(i), c)
        y = Yr[3 * a_m:, i] / B
        f, p = subspace_pursuit(N, B, pos, y, taus, tol2, opts.max_iter)
        fs.extend(f.tolist())
        vs.extend(p.tolist())
    fs = np.array(fs, dtype=np.int64)
    vs = np.array(vs, dtype=np.complex128)
    n = fs.size
    if n > K:
        order = np.lexsort((fs, -np.abs(vs)))[:K]
        fs, vs = fs[order], vs[order]
    o = np.argsort(fs, kind="stable")
    return OneShotResult(idx=fs[o], val=vs[o], counts=counts, status=status, n_recovered=n)
