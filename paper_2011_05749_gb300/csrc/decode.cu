// decode.cu -- peeling decoder (Sec. 3.2, subproblems 1-3, Eq. 20) and output compaction.
//
// Round 1 examines every bin of every signal and is embarrassingly parallel, so it runs as
// one grid-wide launch (classify_kernel): tiles of bins, energies with all R loads in
// flight, then locate/fit of the tile's non-zero bins.  The later rounds touch O(K) bins and
// run in peel_kernel, one group of G CTAs per signal:
//   P   every candidate frequency f not already taken (earlier round, or a lower stage in
//       this round): recorded, and the subtraction of B_e v a_r(f) from bin f mod B_e of
//       every stage e and delay r where that bin is still open (resolved bins are never
//       read again) appended to that bin's list; the bins that change are queued;
//   D1  every queued bin: its listed subtractions applied in increasing order of f, each
//       delay's sum compensated (TwoSum), so the result does not depend on the order in
//       which the candidates were accepted; then the energy sum_r |Y_r|^2 against T0 ->
//       zero-ton, else non-zero.  (peel_atomic plans subtract in P instead, with unordered
//       float atomics on the bins.)
//   D2  every non-zero bin: location (ARG phase or ML candidate search), least-squares
//       value v and residual rho; rho <= T1 -> single-ton candidate (the bin is resolved).
// Phases are separated by a group barrier (a bounded spin when G > 1, so a lost CTA turns
// into SFFT_ETIMEDOUT instead of a hang).
//
// Arithmetic: the delay phasors a_r(f) = e^{2 pi i (f tau_r mod N) / N} come from the exact
// integer residue (f tau_r) mod N, looked up in a two-level table of N-th roots of unity
// made in FP64 (FP32 path: error about 1e-7).  The ML search of a bin j factors a_r(j + q B) = a_r(j) e^{2 pi i q tau_r / L},
// so its L candidates are scored against a table of the L-th roots of unity indexed by
// (q (tau_r mod L)) mod L.  The ARG location takes the angle and the snap to the bin's
// candidates in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "sfft_internal.cuh"

namespace sfft {

constexpr int64_t kFMask = (1ll << 40) - 1;
constexpr int kClassifyThreads = 256;

__device__ __forceinline__ int ldv(const int32_t* p) { return *(const volatile int32_t*)p; }

// Barrier of the G CTAs decoding one signal; returns false when the wait ran out (or any
// CTA of the group saw it run out), in which case the error word is set.
__device__ bool group_barrier(int32_t* ctr, int G, long long spin_limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = ldv(ctr + kCtrErr) == 0;
        if (G > 1 && good) {
            const int gen = ldv(ctr + kCtrBarGen);
            __threadfence();
            if (atomicAdd(ctr + kCtrBarCount, 1) == G - 1) {
                atomicExch(ctr + kCtrBarCount, 0);
                __threadfence();
                atomicAdd(ctr + kCtrBarGen, 1);
            } else {
                long long it = 0;
                while (ldv(ctr + kCtrBarGen) == gen) {
                    if (++it > spin_limit || ldv(ctr + kCtrErr) != 0) {
                        atomicExch(ctr + kCtrErr, 1);
                        good = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        } else if (G == 1) {
            __threadfence_block();
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int stage_of(const PlanDesc& pd, int b)
{
    int d = 0;
    while (d + 1 < pd.D && b >= pd.st[d + 1].bin_base) ++d;
    return d;
}

// (a b) mod N for 0 <= a, b < N < 2^30 by Barrett reduction with mu = floor((2^64-1)/N):
// the estimated quotient is at most two below the true one, so two corrections suffice
__device__ __forceinline__ int64_t mulmod(int64_t a, int64_t b, const PlanDesc& pd)
{
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    const uint64_t q = __umul64hi(p, pd.mu);
    uint64_t r = p - q * (uint64_t)pd.N;
    if (r >= (uint64_t)pd.N) r -= pd.N;
    if (r >= (uint64_t)pd.N) r -= pd.N;
    return (int64_t)r;
}

// threshold test in the path's arithmetic type
__device__ __forceinline__ bool below(float v, float tf, double) { return v <= tf; }
__device__ __forceinline__ bool below(double v, float, double td) { return v <= td; }

// v mod L for 0 <= v < 2^20, with a float reciprocal and one correction each way
__device__ __forceinline__ int small_mod(int v, int L, float invL)
{
    int r = v - (int)((float)v * invL) * L;
    if (r < 0) r += L;
    if (r >= L) r -= L;
    return r;
}

// a_r(f) = e^{2 pi i ((f tau) mod N) / N} from the plan's two-level root table (two loads
// that stay in L1/L2 and one complex product)
template <typename T>
__device__ __forceinline__ typename C2<T>::t delay_phasor(const DecodeArgs& a, int64_t f, int32_t tau)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int64_t m = mulmod(f, tau, pd);
    const V* tw = reinterpret_cast<const V*>(a.roots);
    const V hi = __ldg(tw + pd.ph_hi_off + (int)(m >> pd.ph_shift));
    const V lo = __ldg(tw + pd.ph_lo_off + (int)(m & ((1 << pd.ph_shift) - 1)));
    return V{fma(hi.x, lo.x, -(hi.y * lo.y)), fma(hi.x, lo.y, hi.y * lo.x)};
}

// bin b's single-ton f, v: its state and candidate word, and entry k of the round's list
template <typename T>
__device__ __forceinline__ void record_at(const DecodeWs& w, int round, int b, int64_t f,
                                          typename C2<T>::t v, int k)
{
    using V = typename C2<T>::t;
    __stcg(w.state + b, (uint8_t)2);
    __stcg((long long*)w.cand + b, (long long)(((int64_t)round << 40) | f));
    __stcg(w.cbin + k, b);
    __stcg((long long*)w.cf + k, (long long)f);
    reinterpret_cast<V*>(w.cv)[k] = v;
}

template <typename T>
__device__ __forceinline__ void record_candidate(int32_t* ctr, const DecodeWs& w, int round, int b,
                                                 int64_t f, typename C2<T>::t v)
{
    record_at<T>(w, round, b, f, v, atomicAdd(ctr + kCtrRoundBase + 3 * round + 2, 1));
    atomicAdd(ctr + kCtrResolved, 1);
}

// The fit of non-zero bin b (stage d, bin j, Z_r in zx / zy, RM >= R slots) at candidate
// bq: v = sum_r Z_r conj(W[r][bq]) / (R B) and rho = sum_r |Z_r - B v W[r][bq]|^2;
// rho <= T1 records f = j + bq B as a single-ton.
template <typename T, int RM>
__device__ __forceinline__ void ml_fit(int32_t* ctr, const DecodeWs& w, const typename C2<T>::t* W,
                                       int L, int B, int R, const T* zx, const T* zy, int j, int bq,
                                       int d, int b, int round, const Thr* thr)
{
    using V = typename C2<T>::t;
    T cx = 0, cy = 0;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        if (r < R) {
            const V e = W[r * L + bq];
            cx = fma(zx[r], e.x, fma(zy[r], e.y, cx));
            cy = fma(zy[r], e.x, fma(-zx[r], e.y, cy));
        }
    }
    const int64_t f = (int64_t)j + (int64_t)bq * B;
    const T sc = (T)1 / ((T)R * (T)B);
    const V v = {cx * sc, cy * sc};
    T e2 = 0;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        if (r < R) {
            const V e = W[r * L + bq];
            const T ex = zx[r] - (T)B * (v.x * e.x - v.y * e.y);
            const T ey = zy[r] - (T)B * (v.x * e.y + v.y * e.x);
            e2 += ex * ex + ey * ey;
        }
    }
    if (below(e2, thr[d].T1f, thr[d].T1)) record_candidate<T>(ctr, w, round, b, f, v);
}

// D2, ML locate for non-zero bin j of stage d, by a group of G lanes (G a power of two
// <= 32, groups aligned within the warp; every lane of the warp calls this in lockstep).
// Groups without a bin of their own pass valid = false and some other bin of the same
// tile as b, whose stage's table is within wtab, and record nothing.  Z_r = Y_r conj(a_r(j)); the L
// candidates q are scored by |sum_r Z_r conj(W[r][q])|^2 with the stage's phasor table
// W[r][q] = e^{2 pi i (q tauL_r mod L) / L} (a candidate f = j + q B has
// a_r(f) = a_r(j) W[r][q]); the lanes of the group split the candidates (consecutive q on
// consecutive lanes, so the table reads are conflict-free), then a group argmax (lowest q
// on ties).  The best q gives v = sum_r Z_r conj(W[r][q]) / (R B) and
// rho = sum_r |Z_r - B v W[r][q]|^2; lane 0 of the group records a single-ton.
// RT > 0: the number of delays as a compile-time constant (R = RT); RT = 0: R = pd.R.
// wtab holds the tables from plan-table offset wtab_base on.
template <typename T, int RT>
__device__ void locate_ml_group(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                                const typename C2<T>::t* Y, const typename C2<T>::t* wtab,
                                int32_t wtab_base, int round, int b, bool valid, int G,
                                const Thr* thr)
{
    using V = typename C2<T>::t;
    constexpr int RM = RT > 0 ? RT : kMaxDelays;  // delay slots the loops unroll over
    const PlanDesc& pd = a.pd;
    const int li = threadIdx.x & (G - 1);
    const int d = stage_of(pd, b);
    const StageDesc& st = pd.st[d];
    const int R = RT > 0 ? RT : pd.R;
    const int B = st.B, L = st.L;
    const int j = __ldg(a.pbin + b);
    const V* Yb = Y + st.y_off + (b - st.bin_base);
    T zx[RM], zy[RM];
    if (G >= R) {
        // lane r of the group forms Z_r, the group shares them
        V z = {0, 0};
        if (li < R) {
            const V y = __ldcg(Yb + (int64_t)li * B);
            const V aj = delay_phasor<T>(a, j, st.tau[li]);
            z = V{y.x * aj.x + y.y * aj.y, y.y * aj.x - y.x * aj.y};
        }
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            zx[r] = 0;
            zy[r] = 0;
            if (r < R) {
                zx[r] = __shfl_sync(0xffffffffu, z.x, r, G);
                zy[r] = __shfl_sync(0xffffffffu, z.y, r, G);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            zx[r] = 0;
            zy[r] = 0;
            if (r < R) {
                const V y = __ldcg(Yb + (int64_t)r * B);
                const V aj = delay_phasor<T>(a, j, st.tau[r]);
                zx[r] = y.x * aj.x + y.y * aj.y;
                zy[r] = y.y * aj.x - y.x * aj.y;
            }
        }
    }
    const V* W = wtab + (st.wtab_off - wtab_base);
    T best = (T)-1;
    int bq = 0;
    // the score of candidate q: the sum over delays in two interleaved halves (even and odd
    // r), as before; two candidates (q, q + G) per trip so that their FMA chains interleave
    auto score = [&](int q) {
        T cx0 = 0, cy0 = 0, cx1 = 0, cy1 = 0;
#pragma unroll
        for (int r = 0; r < RM; r += 2) {
            if (r < R) {
                // Z_r conj(w): (zx wx + zy wy, zy wx - zx wy), as fused multiply-adds
                const V w0 = W[r * L + q];
                cx0 = fma(zx[r], w0.x, fma(zy[r], w0.y, cx0));
                cy0 = fma(zy[r], w0.x, fma(-zx[r], w0.y, cy0));
            }
            if (r + 1 < R) {
                const V w1 = W[(r + 1) * L + q];
                cx1 = fma(zx[r + 1], w1.x, fma(zy[r + 1], w1.y, cx1));
                cy1 = fma(zy[r + 1], w1.x, fma(-zx[r + 1], w1.y, cy1));
            }
        }
        const T cx = cx0 + cx1, cy = cy0 + cy1;
        return cx * cx + cy * cy;
    };
    int q = li;
    for (; q + G < L; q += 2 * G) {
        const T s0 = score(q), s1 = score(q + G);
        if (s0 > best) {
            best = s0;
            bq = q;
        }
        if (s1 > best) {
            best = s1;
            bq = q + G;
        }
    }
    if (q < L) {
        const T s0 = score(q);
        if (s0 > best) {
            best = s0;
            bq = q;
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o, G);
        const int oq = __shfl_xor_sync(0xffffffffu, bq, o, G);
        if (ob > best || (ob == best && oq < bq)) {
            best = ob;
            bq = oq;
        }
    }
    if (!valid || li != 0) return;
    ml_fit<T, RM>(ctr, w, W, L, B, R, zx, zy, j, bq, d, b, round, thr);
}

// D2 on the tensor cores (FP32, ML, the first round): the scores of up to 8 NT bins of one
// stage (bl[0 .. nb)) against all L candidates as the product A Z of the stage's fragment
// table (the candidate matrix, split into high and low parts) with the bins' [Re Z; Im Z],
// Z_r = Y_r conj(a_r(j)) -- n-tile u's column g is bin 8 u + g -- keeping three partial
// products (hi hi + hi lo + lo hi, FP32-level scores) as the tensor-core DFT axes do.
// Two forms, which differ only in the MMA shape and so in which delays a lane holds:
//   split TF32 (locate_ml_tc, ml_tc_tf32 = 1): m16n8k8 MMAs, the table of ml_tc_word, lane
//     slot i holds delay t + 4 i (k-tiles of 4 delays);
//   split FP16 (locate_ml_tc16, the default): m16n8k16 MMAs, the table of ml_tc16_word, lane
//     slot i holds delay 8 (i / 2) + 2 t + i % 2 (k-tiles of 8 delays, so R <= 8 is one
//     k-tile and a candidate tile takes half the MMAs and fragment loads), with a
//     power-of-two scale per bin -- its largest Z component mapped into [2^13, 2^14) -- which
//     all of its candidates share, so its argmax is that of the unscaled scores.
// Each A fragment serves the NT n-tiles.  Lane (g, t) keeps the best of candidates 8 mt + g
// for bins 2 t and 2 t + 1 of each n-tile; the eight lanes sharing t reduce them (lowest q
// on ties).  The fit of bin 8 u + g then runs on lanes (g, 0..3), which hold its Z:
// v = sum_r Z_r conj(W[r][bq]) / (R B) and the residual, each a sum of per-lane parts.
// Every lane of the warp calls these in lockstep.
template <bool F16>
__device__ __forceinline__ int ml_tc_delay(int i, int t)
{
    return F16 ? 8 * (i >> 1) + 2 * t + (i & 1) : t + 4 * i;
}

// Z of bin 8 u + g at the lane's delays: every load in flight at once (bins, then their
// samples and phasors)
template <int NZ, int NT, bool F16>
__device__ __forceinline__ void ml_tc_form_z(const DecodeArgs& a, const StageDesc& st, const float2* Y,
                                             const int* bl, int nb, float (&zx)[NT][NZ], float (&zy)[NT][NZ])
{
    using V = float2;
    const int lane = (int)(threadIdx.x & 31), g = lane >> 2, t = lane & 3;
    const int R = a.pd.R, B = st.B;
    int jg[NT];
    V y[NT][NZ];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        const int i8 = 8 * u + g;
        const int bg = bl[i8 < nb ? i8 : 0];
        jg[u] = __ldg(a.pbin + bg);
        const V* Yg = Y + st.y_off + (bg - st.bin_base);
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            const int r = ml_tc_delay<F16>(i, t);
            y[u][i] = r < R && i8 < nb ? __ldcg(Yg + (int64_t)r * B) : V{0.0f, 0.0f};
        }
    }
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            const int r = ml_tc_delay<F16>(i, t);
            const V aj = delay_phasor<float>(a, jg[u], st.tau[r < R ? r : 0]);
            zx[u][i] = y[u][i].x * aj.x + y[u][i].y * aj.y;
            zy[u][i] = y[u][i].y * aj.x - y[u][i].x * aj.y;
        }
}

// One candidate tile's accumulators into the lane's running best: rows g / g + 8 are Re / Im
// c of candidate q = 8 mt + g; columns 2 t, 2 t + 1 the bins
template <int NT>
__device__ __forceinline__ void ml_tc_score(const float (&c)[NT][4], const float (&e)[NT][4],
                                            const float (&f)[NT][4], int q, int L,
                                            float (&best)[NT][2], int (&bq)[NT][2])
{
    if (q >= L) return;
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float cx = c[u][h] + (e[u][h] + f[u][h]);
            const float cy = c[u][2 + h] + (e[u][2 + h] + f[u][2 + h]);
            const float sc = cx * cx + cy * cy;
            if (sc > best[u][h]) {
                best[u][h] = sc;
                bq[u][h] = q;
            }
        }
}

// The argmax over the lanes sharing t, the fit of each bin on the four lanes that hold its
// Z, and the warp's single-tons recorded with one list reservation
template <int NZ, int NT, bool F16>
__device__ __forceinline__ void ml_tc_finish(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                                             const float2* wtab, int32_t wtab_base, int round,
                                             const int* bl, int nb, const Thr* thr, int d,
                                             const StageDesc& st, const float (&zx)[NT][NZ],
                                             const float (&zy)[NT][NZ], float (&best)[NT][2],
                                             int (&bq)[NT][2])
{
    using V = float2;
    const int lane = (int)(threadIdx.x & 31), g = lane >> 2, t = lane & 3;
    const int R = a.pd.R, B = st.B, L = st.L;
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best[u][h], o);
                const int oq = __shfl_xor_sync(0xffffffffu, bq[u][h], o);
                if (ob > best[u][h] || (ob == best[u][h] && oq < bq[u][h])) {
                    best[u][h] = ob;
                    bq[u][h] = oq;
                }
            }
    // the fit of bin 8 u + g on lanes (g, 0..3); its best candidate is held by lane g / 2
    const V* W = wtab + (st.wtab_off - wtab_base);
    const float scl = 1.0f / ((float)R * (float)B);
    bool ok[NT];
    V vv[NT];
    int qq[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        const int i8 = 8 * u + g;
        const int q0 = __shfl_sync(0xffffffffu, bq[u][0], g >> 1);
        const int q1 = __shfl_sync(0xffffffffu, bq[u][1], g >> 1);
        const int qb = (g & 1) ? q1 : q0;
        float cx = 0.0f, cy = 0.0f;
        V wr[NZ];
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            const int r = ml_tc_delay<F16>(i, t);
            wr[i] = r < R ? W[r * L + qb] : V{0.0f, 0.0f};
            cx = fma(zx[u][i], wr[i].x, fma(zy[u][i], wr[i].y, cx));
            cy = fma(zy[u][i], wr[i].x, fma(-zx[u][i], wr[i].y, cy));
        }
        cx += __shfl_xor_sync(0xffffffffu, cx, 1);
        cy += __shfl_xor_sync(0xffffffffu, cy, 1);
        cx += __shfl_xor_sync(0xffffffffu, cx, 2);
        cy += __shfl_xor_sync(0xffffffffu, cy, 2);
        const V v = {cx * scl, cy * scl};
        float e2 = 0.0f;
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            if (ml_tc_delay<F16>(i, t) < R) {
                const float ex = zx[u][i] - (float)B * (v.x * wr[i].x - v.y * wr[i].y);
                const float ey = zy[u][i] - (float)B * (v.x * wr[i].y + v.y * wr[i].x);
                e2 += ex * ex + ey * ey;
            }
        }
        e2 += __shfl_xor_sync(0xffffffffu, e2, 1);
        e2 += __shfl_xor_sync(0xffffffffu, e2, 2);
        ok[u] = t == 0 && i8 < nb && below(e2, thr[d].T1f, thr[d].T1);
        vv[u] = v;
        qq[u] = qb;
    }
    // the warp's single-tons: one list reservation for all of them
    unsigned m[NT];
    int n_rec = 0;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        m[u] = __ballot_sync(0xffffffffu, ok[u]);
        n_rec += __popc(m[u]);
    }
    if (n_rec == 0) return;
    int base = 0;
    if (lane == 0) {
        base = atomicAdd(ctr + kCtrRoundBase + 3 * round + 2, n_rec);
        atomicAdd(ctr + kCtrResolved, n_rec);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    const unsigned below_me = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        if (ok[u]) {
            const int b = bl[8 * u + g];
            const int64_t f = (int64_t)__ldg(a.pbin + b) + (int64_t)qq[u] * B;
            record_at<float>(w, round, b, f, vv[u], base + __popc(m[u] & below_me));
        }
        base += __popc(m[u]);
    }
}

// Split TF32: NZ = RP / 4 k-tiles of 8 rows (RP = ml_tc_rp(R)); k-tile kt's rows are
// 8 kt + t (slot 0) and 8 kt + t + 4 (slot 1) of [Re Z; Im Z] (row k < RP: Re Z_k, else
// Im Z_{k - RP}); the partial products in separate accumulators, chains of KT MMAs
template <int NZ, int NT>
__device__ __noinline__ void locate_ml_tc(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                                          const float2* Y, const float2* wtab, int32_t wtab_base,
                                          int round, const int* bl, int nb, const Thr* thr)
{
    constexpr int RP = 4 * NZ, KT = NZ;
    const int lane = (int)(threadIdx.x & 31);
    const int d = stage_of(a.pd, bl[0]);
    const StageDesc& st = a.pd.st[d];
    float zx[NT][NZ], zy[NT][NZ];          // Z_{t + 4 i} of bin 8 u + g
    uint32_t bh[NT][KT][2], bo[NT][KT][2];  // its B fragments: high and low parts
    ml_tc_form_z<NZ, NT, false>(a, st, Y, bl, nb, zx, zy);
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int kt = 0; kt < KT; ++kt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 8 * kt + 4 * h;
                const float v = k < RP ? zx[u][(k % RP) >> 2] : zy[u][(k % RP) >> 2];
                tf32_split_bits(__float_as_uint(v), &bh[u][kt][h], &bo[u][kt][h]);
            }
    const uint4* fr = a.mltc + (size_t)st.mltc_off * 64 + lane;
    const int MT = (st.L + 7) >> 3;
    float best[NT][2];
    int bq[NT][2];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        best[u][0] = best[u][1] = -1.0f;
        bq[u][0] = bq[u][1] = 0;
    }
    for (int mt = 0; mt < MT; ++mt) {
        float c[NT][4], e[NT][4], f[NT][4];
#pragma unroll
        for (int u = 0; u < NT; ++u)
#pragma unroll
            for (int x = 0; x < 4; ++x) c[u][x] = e[u][x] = f[u][x] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            const uint4 ah = __ldg(fr + (mt * KT + kt) * 64), al = __ldg(fr + (mt * KT + kt) * 64 + 32);
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                mma_tf32(e[u], al, bh[u][kt][0], bh[u][kt][1]);
                mma_tf32(f[u], ah, bo[u][kt][0], bo[u][kt][1]);
                mma_tf32(c[u], ah, bh[u][kt][0], bh[u][kt][1]);
            }
        }
        ml_tc_score<NT>(c, e, f, 8 * mt + (lane >> 2), st.L, best, bq);
    }
    ml_tc_finish<NZ, NT, false>(a, ctr, w, wtab, wtab_base, round, bl, nb, thr, d, st, zx, zy, best, bq);
}

// Split FP16: KK k-tiles of 16 rows; lane (g, t)'s B fragment of k-tile kk is rows 2 t,
// 2 t + 1 (register 0: Re Z_{8 kk + 2 t + j}) and 2 t + 8, 2 t + 9 (register 1: the Im
// parts) of column g.  With one k-tile the next candidate tile's fragments are loaded while
// the current one's MMAs run.
template <int KK, int NT>
__device__ __noinline__ void locate_ml_tc16(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                                            const float2* Y, const float2* wtab, int32_t wtab_base,
                                            int round, const int* bl, int nb, const Thr* thr)
{
    constexpr int NZ = 2 * KK;  // Z per lane and bin
    const int lane = (int)(threadIdx.x & 31);
    const int d = stage_of(a.pd, bl[0]);
    const StageDesc& st = a.pd.st[d];
    float zx[NT][NZ], zy[NT][NZ];
    uint32_t bh[NT][KK][2], bo[NT][KK][2];  // B fragments: high and low parts
    ml_tc_form_z<NZ, NT, true>(a, st, Y, bl, nb, zx, zy);
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        // the bin's scale: its largest component over the four lanes that hold its Z
        float mx = 0.0f;
#pragma unroll
        for (int i = 0; i < NZ; ++i) mx = fmaxf(mx, fmaxf(fabsf(zx[u][i]), fabsf(zy[u][i])));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        const float sc = ldexpf(1.0f, 13 - (mx > 0.0f ? max(ilogbf(mx), -100) : 0));
#pragma unroll
        for (int kk = 0; kk < KK; ++kk) {
            f16_split2(zx[u][2 * kk] * sc, zx[u][2 * kk + 1] * sc, bh[u][kk][0], bo[u][kk][0]);
            f16_split2(zy[u][2 * kk] * sc, zy[u][2 * kk + 1] * sc, bh[u][kk][1], bo[u][kk][1]);
        }
    }
    const uint4* fr = a.mltc + (size_t)st.mltc_off * 64 + lane;
    const int MT = (st.L + 7) >> 3;
    float best[NT][2];
    int bq[NT][2];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        best[u][0] = best[u][1] = -1.0f;
        bq[u][0] = bq[u][1] = 0;
    }
    // with one k-tile the registers allow the next candidate tile's fragments in flight
    constexpr bool kAhead = KK == 1;
    uint4 nh[KK], nl[KK];
    if constexpr (kAhead) {
        nh[0] = __ldg(fr);
        nl[0] = __ldg(fr + 32);
    }
    for (int mt = 0; mt < MT; ++mt) {
        uint4 ah[KK], al[KK];
        if constexpr (kAhead) {
            ah[0] = nh[0];
            al[0] = nl[0];
            // the next tile's fragments (the last tile's again at the end: in bounds, unused)
            const int mn = min(mt + 1, MT - 1);
            nh[0] = __ldg(fr + mn * 64);
            nl[0] = __ldg(fr + mn * 64 + 32);
        } else {
#pragma unroll
            for (int kk = 0; kk < KK; ++kk) {
                ah[kk] = __ldg(fr + (mt * KK + kk) * 64);
                al[kk] = __ldg(fr + (mt * KK + kk) * 64 + 32);
            }
        }
        float c[NT][4], e[NT][4], f[NT][4];
#pragma unroll
        for (int u = 0; u < NT; ++u)
#pragma unroll
            for (int x = 0; x < 4; ++x) c[u][x] = e[u][x] = f[u][x] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < KK; ++kk)
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                mma_f16(e[u], al[kk], bh[u][kk][0], bh[u][kk][1]);
                mma_f16(f[u], ah[kk], bo[u][kk][0], bo[u][kk][1]);
                mma_f16(c[u], ah[kk], bh[u][kk][0], bh[u][kk][1]);
            }
        ml_tc_score<NT>(c, e, f, 8 * mt + (lane >> 2), st.L, best, bq);
    }
    ml_tc_finish<NZ, NT, true>(a, ctr, w, wtab, wtab_base, round, bl, nb, thr, d, st, zx, zy, best, bq);
}

// Lanes per bin for the ML search of n bins with at most Lmax candidates by nt threads:
// the G that minimises (bins per lane) x (work per bin and lane), where a bin costs every
// lane of its group ~4 R FMAs per candidate it scans, forming Z (shared when G >= R) and
// the log2 G reduction steps.
__device__ __forceinline__ int ml_group_size(int n, int Lmax, int R, int nt)
{
    int best_g = 1, best = 0x7fffffff;
    for (int g = 1, lg = 0; g <= 32; g <<= 1, ++lg) {
        const int per = nt / g;
        const int rounds = (n + per - 1) / per;
        const int cost = rounds * (((Lmax + g - 1) / g) * 4 * R + (g >= R ? 40 : 20 * R) + 12 * lg);
        if (cost < best) {
            best = cost;
            best_g = g;
        }
    }
    return best_g;
}

// D2, phase locate, one thread per bin: ARG (FFAST, Sec. 3.2 subproblem 2, exact case): f
// from the phase of Y(1) conj(Y(0)) in FP64; KAY (general sparse case, Eq. 21-22): one bit
// of f / N per iteration of structured delays, in FP64.  Either estimate is snapped to the
// bin's candidate set {j + q B}; then the least-squares value and the residual test.
template <typename T>
__device__ void locate_phase_thread(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                                    const typename C2<T>::t* Y, int round, int b, const Thr* thr)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int d = stage_of(pd, b);
    const StageDesc& st = pd.st[d];
    const int R = pd.R;
    const int B = st.B, L = st.L, N = pd.N;
    const int j = __ldg(a.pbin + b);
    const V* Yb = Y + st.y_off + (b - st.bin_base);
    constexpr double kTwoPi = 6.283185307179586476925286766559;
    V ar[kMaxDelays], yv[kMaxDelays];
#pragma unroll
    for (int r = 0; r < kMaxDelays; ++r)
        if (r < R) yv[r] = __ldcg(Yb + (int64_t)r * B);
    double fe;  // estimated position on the circle of N frequencies
    if (pd.locate == 2) {
        // KAY (general sparse case, Eq. 21-22): slots c m + t hold r_c + t 2^c; iteration c
        // averages the phase differences arg(y_{c,t+1} conj(y_{c,t})) with Kay's weights into
        // the angle of omega^{2^c f} and reads one bit of f / N from it (binary search); the
        // C bits leave f / N in [k / 2^C, (k + 1) / 2^C), whose centre is fe / N
        const int m = pd.kay_m;
        int64_t k = 0;
        double th = 0.0;
        V yp = yv[0];
#pragma unroll 1
        for (int r = 1; r < R; ++r) {
            const int t1 = r % m;  // t + 1 of this difference, 0 at an iteration's first slot
            const V yr = __ldcg(Yb + (int64_t)r * B);
            if (t1 != 0) {
                const double rx = (double)yr.x * yp.x + (double)yr.y * yp.y;
                const double ry = (double)yr.y * yp.x - (double)yr.x * yp.y;
                const double u = (2.0 * (t1 - 1) - m + 2.0) / (2.0 * m);
                th += 3.0 * m / (2.0 * ((double)m * m - 1.0)) * (1.0 - 4.0 * u * u) * atan2(ry, rx);
            }
            if (t1 == m - 1) {
                // iteration c complete.  The weights are positive and sum to one, so th lies
                // in (-pi, pi]; its angle mod 2 pi is in [pi, 2 pi) (upper half) iff th < 0 or
                // th = pi.  When L divides 2^c the iteration carries no information (every
                // candidate gives 2^c f / N = 2^c j / N mod 1, possibly exactly on the
                // boundary): the bit comes from j, floor(2^{c+1} j / N) mod 2.
                const int c = r / m;
                if (((1ll << c) % L) == 0)
                    k = 2 * k + ((((int64_t)j << (c + 1)) / N) & 1);
                else
                    k = 2 * k + ((th < 0.0 || th >= kTwoPi / 2) ? 1 : 0);
                th = 0.0;
            }
            yp = yr;
        }
        fe = ((double)k + 0.5) * (double)N / (double)(1ll << (R / m));
    } else {
        // ARG (FFAST phase encoding): angle of y(1) conj(y(0)) times N / 2 pi
        const V u0 = __ldcg(Yb + (int64_t)st.r0 * B), u1 = __ldcg(Yb + (int64_t)st.r1 * B);
        if (pd.arg_mode & 1) {
            // angle and scaling in FP32 (a precision experiment, not the library's path)
            const float rxf = (float)u1.x * (float)u0.x + (float)u1.y * (float)u0.y;
            const float ryf = (float)u1.y * (float)u0.x - (float)u1.x * (float)u0.y;
            fe = (double)(atan2f(ryf, rxf) * ((float)N / 6.28318531f));
        } else {
            const double rx = (double)u1.x * u0.x + (double)u1.y * u0.y;
            const double ry = (double)u1.y * u0.x - (double)u1.x * u0.y;
            fe = atan2(ry, rx) * (double)N / kTwoPi;
        }
    }
    int64_t f;
    if (pd.locate == 0 && (pd.arg_mode & 2)) {
        // no residue snap (a precision experiment): the integer nearest the estimate, which
        // the single-ton test rejects unless it is the bin's frequency
        f = (int64_t)floor(fe + 0.5) % N;
        if (f < 0) f += N;
    } else {
        // the bin's candidate j + q B nearest fe
        const double qd = floor((fe - (double)j) / (double)B + 0.5);
        int64_t q = (int64_t)qd % L;
        if (q < 0) q += L;
        f = (int64_t)j + q * B;
    }
#pragma unroll
    for (int r = 0; r < kMaxDelays; ++r)
        if (r < R) ar[r] = delay_phasor<T>(a, f, st.tau[r]);
    V c = {0, 0};
#pragma unroll
    for (int r = 0; r < kMaxDelays; ++r) {
        if (r < R) {
            c.x += yv[r].x * ar[r].x + yv[r].y * ar[r].y;
            c.y += yv[r].y * ar[r].x - yv[r].x * ar[r].y;
        }
    }
    const T sc = (T)1 / ((T)R * (T)B);
    const V v = {c.x * sc, c.y * sc};
    T e2 = 0;
#pragma unroll
    for (int r = 0; r < kMaxDelays; ++r) {
        if (r < R) {
            const T ex = yv[r].x - (T)B * (v.x * ar[r].x - v.y * ar[r].y);
            const T ey = yv[r].y - (T)B * (v.x * ar[r].y + v.y * ar[r].x);
            e2 += ex * ex + ey * ey;
        }
    }
    if (below(e2, thr[d].T1f, thr[d].T1)) record_candidate<T>(ctr, w, round, b, f, v);
}

__device__ __forceinline__ void atomic_sub_c(float2* p, float2 d)
{
    atomicAdd(p, float2{-d.x, -d.y});  // one 8-byte vector atomic (global memory, sm_90+)
}
__device__ __forceinline__ void atomic_sub_c(double2* p, double2 d)
{
    atomicAdd(&p->x, -d.x);
    atomicAdd(&p->y, -d.y);
}

// P: accept candidate c and peel it from every stage (Eq. 20).  The per-stage loads,
// checks and atomics are independent, so they are issued together (stage loops unrolled)
// rather than one round trip after another.
template <typename T>
__device__ void peel_candidate(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                               typename C2<T>::t* Y, int round, int c)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int D = pd.D;
    const int b = __ldcg(w.cbin + c);
    const int64_t f = (int64_t)__ldcg((const long long*)w.cf + c);
    const V v = __ldcg(reinterpret_cast<const V*>(w.cv) + c);
    const int d = stage_of(pd, b);
    int be[kMaxStages];
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e) {
        be[e] = 0;
        if (e < D) {
            const StageDesc& se = pd.st[e];
            const int je = (int)((uint32_t)f % (uint32_t)se.B);
            be[e] = se.bin_base + __ldg(a.bpos + se.bin_base + je);
        }
    }
    int64_t cw[kMaxStages];
    uint8_t open[kMaxStages];
    uint8_t stt[kMaxStages];
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e) stt[e] = e < D ? __ldcg(w.state + be[e]) : (uint8_t)1;
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e) {
        // a bin's candidate word is written with its single-ton state and only read then
        cw[e] = (e < D && e != d && stt[e] == 2) ? (int64_t)__ldcg((const long long*)w.cand + be[e]) : -1;
        open[e] = stt[e] == 0;
    }
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e) {
        if (e < D && e != d && cw[e] >= 0 && (cw[e] & kFMask) == f) {
            const int rd = (int)(cw[e] >> 40);
            if (rd < round || (rd == round && e < d)) return;
        }
    }
    const int k = atomicAdd(ctr + kCtrRec, 1);
    __stcg((long long*)w.rec_f + k, (long long)f);
    reinterpret_cast<V*>(w.rec_v)[k] = v;
    const int R = pd.R;
    // only open bins are updated: a resolved bin (zero-ton, or single-ton -- f's own bin
    // among them) is never read again, so its value no longer matters
    if (!pd.peel_atomic) {
        // the subtraction is queued on the bin's list and applied in D1 (at most D entries
        // per accepted candidate, each bin a candidate at most once: D sumB entries)
        const int cap = D * pd.sumB;
#pragma unroll
        for (int e = 0; e < kMaxStages; ++e) {
            if (e >= D || !open[e]) continue;
            const int sl = atomicAdd(ctr + kCtrSub, 1);
            if (sl >= cap) {
                atomicExch(ctr + kCtrErr, 1);
                continue;
            }
            const int prev = atomicExch(w.sub_head + be[e], sl);
            __stcg(w.sub_ent + sl, int2{c, prev});
            // the bin's first entry this round queues it for the next round
            if (prev < 0) __stcg(((round & 1) ? w.list1 : w.list0) + atomicAdd(ctr + kCtrRoundBase + 3 * round + 0, 1), be[e]);
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e) {
        if (e >= D || !open[e] || !pd.peel_atomic) continue;
        const StageDesc& se = pd.st[e];
        const T Bv = (T)se.B;
        V* Yb = Y + se.y_off + (be[e] - se.bin_base);
        // all R phasor lookups in flight first, then the atomics (a table load placed after
        // an atomic could not be hoisted above it)
        V ar[kMaxDelays];
#pragma unroll
        for (int r = 0; r < kMaxDelays; ++r)
            if (r < R) ar[r] = delay_phasor<T>(a, f, se.tau[r]);
#pragma unroll
        for (int r = 0; r < kMaxDelays; ++r) {
            if (r < R) {
                const V dlt = {Bv * (v.x * ar[r].x - v.y * ar[r].y), Bv * (v.x * ar[r].y + v.y * ar[r].x)};
                atomic_sub_c(Yb + (int64_t)r * se.B, dlt);
            }
        }
    }
    // unordered atomics: the dirty flag's first setter queues the bin
    uint32_t was[kMaxStages];
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e) was[e] = (e < D && open[e]) ? atomicExch(w.dirty + be[e], 1u) : 1u;
    int32_t* nl = (round & 1) ? w.list1 : w.list0;
#pragma unroll
    for (int e = 0; e < kMaxStages; ++e)
        if (was[e] == 0u) __stcg(nl + atomicAdd(ctr + kCtrRoundBase + 3 * round + 0, 1), be[e]);
}

// D1 of one bin: energy over the R delays (all loads in flight)
template <typename T>
__device__ __forceinline__ bool bin_is_zero(const PlanDesc& pd, const typename C2<T>::t* Y, int b,
                                            const Thr* thr)
{
    using V = typename C2<T>::t;
    const int d = stage_of(pd, b);
    const StageDesc& st = pd.st[d];
    const V* Yb = Y + st.y_off + (b - st.bin_base);
    V y[kMaxDelays];
#pragma unroll
    for (int r = 0; r < kMaxDelays; ++r)
        if (r < pd.R) y[r] = __ldcg(Yb + (int64_t)r * st.B);
    T E = 0;
#pragma unroll
    for (int r = 0; r < kMaxDelays; ++r)
        if (r < pd.R) E += y[r].x * y[r].x + y[r].y * y[r].y;
    return below(E, thr[d].T0f, thr[d].T0);
}

// D1 of NB bins b, b + stride, ... (those at or past b1 count as zero) with a compile-time
// delay count: all NB RT loads in flight before the energies (the same sums as bin_is_zero)
template <typename T, int RT, int NB>
__device__ __forceinline__ void bins_are_zero(const PlanDesc& pd, const typename C2<T>::t* Y, int b,
                                              int stride, int b1, const Thr* thr, bool* z)
{
    using V = typename C2<T>::t;
    V y[NB][RT];
    int dd[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int bu = b + u * stride < b1 ? b + u * stride : b;
        const int d = stage_of(pd, bu);
        dd[u] = d;
        const StageDesc& st = pd.st[d];
        const V* Yb = Y + st.y_off + (bu - st.bin_base);
#pragma unroll
        for (int r = 0; r < RT; ++r) y[u][r] = __ldcg(Yb + (int64_t)r * st.B);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        T E = 0;
#pragma unroll
        for (int r = 0; r < RT; ++r) E += y[u][r].x * y[u][r].x + y[u][r].y * y[u][r].y;
        z[u] = b + u * stride >= b1 || below(E, thr[dd[u]].T0f, thr[dd[u]].T0);
    }
}

// s = a + b and the rounding error e of that sum, a + b = s + e exactly (Knuth's TwoSum)
template <typename T>
__device__ __forceinline__ T two_sum(T a, T b, T* e)
{
    const T s = a + b;
    const T bb = s - a;
    *e = (a - (s - bb)) + (b - bb);
    return s;
}

// D1 of one bin with ordered peeling: apply the bin's listed subtractions (Eq. 20) in
// increasing order of frequency f -- each delay's y_r - sum_f B v_f a_r(f) summed with
// TwoSum and its error terms added back at the end -- store the bin, clear its list, and
// test its energy against T0.  The order and the arithmetic depend only on the set of
// listed frequencies, so the bits do not depend on which CTA accepted what first.
template <typename T, int RT>
__device__ bool apply_and_test_r(const DecodeArgs& a, const DecodeWs& w, typename C2<T>::t* Y,
                                 int b, const Thr* thr)
{
    using V = typename C2<T>::t;
    constexpr int RM = RT > 0 ? RT : kMaxDelays;  // delay slots the loops unroll over
    const PlanDesc& pd = a.pd;
    const int R = RT > 0 ? RT : pd.R;
    const int d = stage_of(pd, b);
    const StageDesc& st = pd.st[d];
    V* Yb = Y + st.y_off + (b - st.bin_base);
    V y[RM], cmp[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        cmp[r] = V{0, 0};
        if (r < R) y[r] = __ldcg(Yb + (int64_t)r * st.B);
    }
    const int head = __ldcg(w.sub_head + b);
    if (head >= 0) {
        __stcg(w.sub_head + b, -1);
        const T Bv = (T)st.B;
        const V* cv = reinterpret_cast<const V*>(w.cv);
        int64_t last = -1;
        while (true) {
            // the listed subtraction with the smallest frequency above the last one applied
            int64_t fmin = INT64_MAX;
            int cmin = -1;
            for (int e = head; e >= 0;) {
                const int2 en = __ldcg(w.sub_ent + e);
                const int64_t f = (int64_t)__ldcg((const long long*)w.cf + en.x);
                if (f > last && f < fmin) {
                    fmin = f;
                    cmin = en.x;
                }
                e = en.y;
            }
            if (cmin < 0) break;
            last = fmin;
            const V v = __ldcg(cv + cmin);
            V ar[RM];
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) ar[r] = delay_phasor<T>(a, fmin, st.tau[r]);
#pragma unroll
            for (int r = 0; r < RM; ++r) {
                if (r < R) {
                    const T tx = Bv * (v.x * ar[r].x - v.y * ar[r].y);
                    const T ty = Bv * (v.x * ar[r].y + v.y * ar[r].x);
                    T ex, ey;
                    y[r].x = two_sum<T>(y[r].x, -tx, &ex);
                    y[r].y = two_sum<T>(y[r].y, -ty, &ey);
                    cmp[r].x += ex;
                    cmp[r].y += ey;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (r < R) {
                y[r] = V{y[r].x + cmp[r].x, y[r].y + cmp[r].y};
                __stcg(Yb + (int64_t)r * st.B, y[r]);
            }
        }
    }
    T E = 0;
#pragma unroll
    for (int r = 0; r < RM; ++r)
        if (r < R) E += y[r].x * y[r].x + y[r].y * y[r].y;
    return below(E, thr[d].T0f, thr[d].T0);
}

// apply_and_test_r with the delay count as a constant for the common R
template <typename T>
__device__ __forceinline__ bool apply_and_test(const DecodeArgs& a, const DecodeWs& w,
                                               typename C2<T>::t* Y, int b, const Thr* thr)
{
    switch (a.pd.R) {
    case 6: return apply_and_test_r<T, 6>(a, w, Y, b, thr);
    case 8: return apply_and_test_r<T, 8>(a, w, Y, b, thr);
    case 10: return apply_and_test_r<T, 10>(a, w, Y, b, thr);
    default: return apply_and_test_r<T, 0>(a, w, Y, b, thr);
    }
}

template <typename T>
__device__ __forceinline__ DecodeWs slot_ws(const DecodeArgs& a, int sig)
{
    using V = typename C2<T>::t;
    DecodeWs w = a.ws;
    const int64_t so = (int64_t)sig * a.pd.sumB;
    w.state += so;
    w.dirty += so;
    w.cand += so;
    w.list0 += so;
    w.list1 += so;
    w.nzl += so;
    w.cbin += so;
    w.cf += so;
    w.cv = reinterpret_cast<V*>(w.cv) + so;
    w.rec_f += so;
    w.rec_v = reinterpret_cast<V*>(w.rec_v) + so;
    w.ctr += (int64_t)sig * a.ctr_stride;
    if (w.sub_head) {
        w.sub_head += so;
        w.sub_ent += so * a.pd.D;
    }
    return w;
}

// locate_ml_group with the delay count as a constant for the common R
template <typename T>
__device__ __forceinline__ void locate_ml(const DecodeArgs& a, int32_t* ctr, const DecodeWs& w,
                                          const typename C2<T>::t* Y, const typename C2<T>::t* wtab,
                                          int32_t wtab_base, int round, int b, bool valid, int G,
                                          const Thr* thr)
{
    switch (a.pd.R) {
    case 6: locate_ml_group<T, 6>(a, ctr, w, Y, wtab, wtab_base, round, b, valid, G, thr); break;
    case 8: locate_ml_group<T, 8>(a, ctr, w, Y, wtab, wtab_base, round, b, valid, G, thr); break;
    case 10: locate_ml_group<T, 10>(a, ctr, w, Y, wtab, wtab_base, round, b, valid, G, thr); break;
    default: locate_ml_group<T, 0>(a, ctr, w, Y, wtab, wtab_base, round, b, valid, G, thr); break;
    }
}

// The stages' thresholds for signal sig into thr[0 .. D): the plan's, or from the signal's
// estimated sigma^2 (noise_auto).  Called by one thread.
__device__ __forceinline__ void signal_thresholds(const DecodeArgs& a, int sig, Thr* thr)
{
    const PlanDesc& pd = a.pd;
    const double s2 = pd.noise_auto ? __ldcg(a.ws.sig2 + sig) : 0.0;
    for (int d = 0; d < pd.D; ++d) {
        const StageDesc& st = pd.st[d];
        if (pd.noise_auto) {
            thr[d].T0 = st.T0a * s2 + st.Tb;
            thr[d].T1 = st.T1a * s2 + st.Tb;
        } else {
            thr[d].T0 = st.T0;
            thr[d].T1 = st.T1;
        }
        thr[d].T0f = (float)thr[d].T0;
        thr[d].T1f = (float)thr[d].T1;
    }
}

// Round 1: classify every bin.  One CTA per tile of kClassifyTile bins of one signal.
// FP32: three CTAs per SM (85 registers).  With the split-FP16 tensor-core search, decode
// takes 0.411 ms per 256 signals of N = 127 * 128 * 129 against 0.427 with four CTAs (64
// registers), and tiles of 2048 bins beat 1024 (0.482), 3072 (0.445) and 4096 (0.429); with
// the split-TF32 search three CTAs also won (0.462 against 0.468 with four, 0.490 with two);
// with the FMA search four had been best (0.67 against 0.77 with two), and five or six
// spill too much.
template <typename T>
__global__ void __launch_bounds__(kClassifyThreads, sizeof(T) == 4 ? 3 : 2)
    classify_kernel(const __grid_constant__ DecodeArgs a)
{
    using V = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_nz[kClassifyTile];  // non-zero bins: the first stage's from the front,
    __shared__ int s_cnt, s_hi;          // the second's from the back (tiles within two stages)
    const PlanDesc& pd = a.pd;
    const int tiles = (pd.sumB + kClassifyTile - 1) / kClassifyTile;
    const int sig = blockIdx.x / tiles;
    const int tile = blockIdx.x - sig * tiles;
    const DecodeWs w = slot_ws<T>(a, sig);
    V* Y = reinterpret_cast<V*>(a.bins) + (int64_t)sig * pd.y_per_sig;
    const int b0 = tile * kClassifyTile;
    const int b1 = min(pd.sumB, b0 + kClassifyTile);
    // the ML phasor tables of the tile's stages (consecutive in the plan table), in shared
    // memory when the launch gave room for them
    const V* wtab = reinterpret_cast<const V*>(a.roots);
    int32_t wtab_base = 0;
    if (pd.locate == 1 && a.wtab_smem) {
        const int d0 = stage_of(pd, b0), d1 = stage_of(pd, b1 - 1);
        wtab_base = pd.st[d0].wtab_off;
        const int n = pd.st[d1].wtab_off + pd.R * pd.st[d1].L - wtab_base;
        V* ws = reinterpret_cast<V*>(smem_raw);
        // asynchronous copies, all in flight at once
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(ws + i);
            if constexpr (sizeof(V) == 16)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(wtab + wtab_base + i) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(wtab + wtab_base + i) : "memory");
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        wtab = ws;
    }
    __shared__ Thr s_thr[kMaxStages];
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_hi = 0;
        signal_thresholds(a, sig, s_thr);
    }
    __syncthreads();
    const int dlo = stage_of(pd, b0), dhi = stage_of(pd, b1 - 1);
    const int bsplit = dhi == dlo + 1 ? pd.st[dhi].bin_base : b1;
    // D1: the zero-ton test of every bin, NB bins per thread with all their loads in flight
    // (a compile-time delay count for the common R)
    constexpr int NB = 4;
    for (int b = b0 + threadIdx.x; b < b1; b += NB * blockDim.x) {
        bool z[NB];
        if (pd.R == 8) {
            bins_are_zero<T, 8, 2>(pd, Y, b, blockDim.x, b1, s_thr, z);
            bins_are_zero<T, 8, 2>(pd, Y, b + 2 * blockDim.x, blockDim.x, b1, s_thr, z + 2);
        } else if (pd.R == 6) {
            bins_are_zero<T, 6, 2>(pd, Y, b, blockDim.x, b1, s_thr, z);
            bins_are_zero<T, 6, 2>(pd, Y, b + 2 * blockDim.x, blockDim.x, b1, s_thr, z + 2);
        } else {
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int bu = b + u * blockDim.x;
                z[u] = bu < b1 ? bin_is_zero<T>(pd, Y, bu, s_thr) : true;
            }
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int bu = b + u * blockDim.x;
            if (bu >= b1) continue;
            // per-bin decode state: the state of every bin; the subtraction list head (ordered
            // peeling) or the dirty flag (atomic peeling) of the bins that can stay open; the
            // candidate word is written only with a single-ton state
            __stcg(w.state + bu, (uint8_t)(z[u] ? 1 : 0));
            if (!z[u]) {
                if (bu < bsplit)
                    s_nz[atomicAdd(&s_cnt, 1)] = bu;
                else
                    s_nz[kClassifyTile - 1 - atomicAdd(&s_hi, 1)] = bu;
                if (pd.peel_atomic)
                    __stcg(w.dirty + bu, 0u);
                else
                    __stcg(w.sub_head + bu, -1);
            }
        }
    }
    __syncthreads();
    const int n_lo = s_cnt, n_hi = s_hi, n_nz = n_lo + n_hi;
    const int* nz_hi = s_nz + kClassifyTile - n_hi;
    auto nz_at = [&](int i) { return i < n_lo ? s_nz[i] : nz_hi[i - n_lo]; };
    bool tc_done = false;
    if (pd.locate == 1) {
        if constexpr (sizeof(T) == 4) {
            if (a.mltc && a.lanes == 0 && dhi - dlo <= 1 && pd.R <= 16) {
                // the tensor-core search: warps take groups of 8 bins of one stage
                constexpr int NB = 16;  // bins per warp task (two n-tiles)
                const int t_lo = (n_lo + NB - 1) / NB, t_all = t_lo + (n_hi + NB - 1) / NB;
                const int nw = (int)(blockDim.x >> 5);
                for (int k = (int)(threadIdx.x >> 5); k < t_all; k += nw) {
                    const int* bl = k < t_lo ? s_nz + NB * k : nz_hi + NB * (k - t_lo);
                    const int nb = min(NB, k < t_lo ? n_lo - NB * k : n_hi - NB * (k - t_lo));
                    if (!a.ml_tf32) {
                        if (pd.R <= 8)
                            locate_ml_tc16<1, 2>(a, w.ctr, w, Y, wtab, wtab_base, 1, bl, nb, s_thr);
                        else
                            locate_ml_tc16<2, 2>(a, w.ctr, w, Y, wtab, wtab_base, 1, bl, nb, s_thr);
                        continue;
                    }
                    switch ((pd.R + 3) >> 2) {
                        case 1: locate_ml_tc<1, 2>(a, w.ctr, w, Y, wtab, wtab_base, 1, bl, nb, s_thr); break;
                        case 2: locate_ml_tc<2, 2>(a, w.ctr, w, Y, wtab, wtab_base, 1, bl, nb, s_thr); break;
                        case 3: locate_ml_tc<3, 2>(a, w.ctr, w, Y, wtab, wtab_base, 1, bl, nb, s_thr); break;
                        default: locate_ml_tc<4, 2>(a, w.ctr, w, Y, wtab, wtab_base, 1, bl, nb, s_thr); break;
                    }
                }
                tc_done = true;
            }
        }
    }
    if (pd.locate == 1 && !tc_done) {
        int Lmax = 0;
        for (int d = 0; d < pd.D; ++d) Lmax = max(Lmax, pd.st[d].L);
        const int G = a.lanes > 0 ? a.lanes : ml_group_size(n_nz, Lmax, pd.R, blockDim.x);
        const int per = blockDim.x / G;
        for (int k = 0; k < (n_nz + per - 1) / per; ++k) {
            const int i = k * per + threadIdx.x / G;
            locate_ml<T>(a, w.ctr, w, Y, wtab, wtab_base, 1, nz_at(i < n_nz ? i : 0), i < n_nz, G, s_thr);
        }
    } else if (pd.locate != 1) {
        for (int i = threadIdx.x; i < n_nz; i += blockDim.x)
            locate_phase_thread<T>(a, w.ctr, w, Y, 1, nz_at(i), s_thr);
    }
    if (threadIdx.x == 0) {
        atomicAdd(w.ctr + kCtrResolved, b1 - b0 - n_nz);  // the zero-tons
        atomicAdd(w.ctr + kCtrIdents, b1 - b0);
    }
}

// Rounds 1 (peel) .. last: one group of G CTAs per signal.  FP32: two CTAs of 512 threads per
// SM (64 registers): a 256-signal batch fits one wave, which outweighs the spills
// (decode 0.54 against 0.59 ms per 256 signals at 128 registers).
template <typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) peel_kernel(const __grid_constant__ DecodeArgs a)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int G = a.G;
    const int sig = blockIdx.x / G;
    const int gi = blockIdx.x - sig * G;
    if (sig >= a.n_sig) return;
    const DecodeWs w = slot_ws<T>(a, sig);
    int32_t* ctr = w.ctr;
    V* Y = reinterpret_cast<V*>(a.bins) + (int64_t)sig * pd.y_per_sig;
    if (a.fault == 1 && G > 1 && gi == G - 1) return;  // injected loss of a CTA (testing)
    const int wt = gi * blockDim.x + threadIdx.x;
    const int nw = G * blockDim.x;
    __shared__ Thr s_thr[kMaxStages];
    if (threadIdx.x == 0) signal_thresholds(a, sig, s_thr);
    __syncthreads();

    int round = 1;
    while (true) {
        // P: accept and peel this round's single-tons
        const int n_c = ldv(ctr + kCtrRoundBase + 3 * round + 2);
        for (int i = wt; i < n_c; i += nw) peel_candidate<T>(a, ctr, w, Y, round, i);
        if (!group_barrier(ctr, G, a.spin_limit)) break;
        const int n_next = ldv(ctr + kCtrRoundBase + 3 * round + 0);
        if (n_next == 0 || round >= pd.max_rounds) break;
        ++round;
        // D1: energies of the queued bins
        const int32_t* act = ((round - 1) & 1) ? w.list1 : w.list0;
        for (int i = wt; i < n_next; i += nw) {
            const int b = __ldcg(act + i);
            if (pd.peel_atomic) __stcg(w.dirty + b, 0u);
            const bool zero = pd.peel_atomic ? bin_is_zero<T>(pd, Y, b, s_thr)
                                             : apply_and_test<T>(a, w, Y, b, s_thr);
            if (zero) {
                __stcg(w.state + b, (uint8_t)1);
                atomicAdd(ctr + kCtrResolved, 1);
            } else {
                __stcg(w.nzl + atomicAdd(ctr + kCtrRoundBase + 3 * round + 1, 1), b);
            }
        }
        if (wt == 0) atomicAdd(ctr + kCtrIdents, n_next);
        if (!group_barrier(ctr, G, a.spin_limit)) break;
        // D2: locate, fit, singleton test
        const int n_nz = ldv(ctr + kCtrRoundBase + 3 * round + 1);
        if (pd.locate == 1) {
            const int gw = wt >> 5, nwarps = nw >> 5;
            const V* wtab = reinterpret_cast<const V*>(a.roots);
            for (int i = gw; i < n_nz; i += nwarps)
                locate_ml<T>(a, ctr, w, Y, wtab, 0, round, __ldcg(w.nzl + i), true, 32, s_thr);
        } else {
            for (int i = wt; i < n_nz; i += nw)
                locate_phase_thread<T>(a, ctr, w, Y, round, __ldcg(w.nzl + i), s_thr);
        }
        if (!group_barrier(ctr, G, a.spin_limit)) break;
    }
    if (gi == 0 && threadIdx.x == 0) ctr[kCtrRounds] = round;
}

// ---------------------------------------------------------------------------------------
// Output (Sec. 2.1): the K largest recovered coefficients, sorted by frequency.  One CTA
// per signal; bitonic sorts in shared memory (or in the slot's global sort buffer when the
// recovered list is larger than the shared-memory capacity).

__device__ void bitonic_sort(uint64_t* key, int n_pad)
{
    for (int k = 2; k <= n_pad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            // pair q: i has bit j clear, partner i + j
            for (int q = threadIdx.x; q < (n_pad >> 1); q += blockDim.x) {
                const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                const int ixj = i + j;
                const uint64_t x = key[i], y = key[ixj];
                const bool up = (i & k) == 0;
                if ((x > y) == up) {
                    key[i] = y;
                    key[ixj] = x;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ uint32_t mag_key(float2 v)
{
    return __float_as_uint(v.x * v.x + v.y * v.y);
}
__device__ __forceinline__ uint32_t mag_key(double2 v)
{
    return (uint32_t)(__double_as_longlong(v.x * v.x + v.y * v.y) >> 32);
}

template <typename T, typename XS>
__global__ void __launch_bounds__(1024) compact_kernel(const __grid_constant__ CompactArgs a)
{
    using V = typename C2<T>::t;
    using XV = typename C2<XS>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sig = blockIdx.x;
    const PlanDesc& pd = a.pd;
    const int nb = pd.sumB;
    const int32_t* ctr = a.ws.ctr + (int64_t)sig * a.ctr_stride;
    const int64_t* rec_f = a.ws.rec_f + (int64_t)sig * nb;
    const V* rec_v = reinterpret_cast<const V*>(a.ws.rec_v) + (int64_t)sig * nb;
    const int n = ldv(ctr + kCtrRec);
    const int K = pd.K;
    int n_pad = 1;
    while (n_pad < n) n_pad <<= 1;
    // keys in shared memory where they fit (smem_cap keys), else in the slot's sort buffer
    uint64_t* const kg = a.sortbuf + (int64_t)sig * 2 * a.sort_cap;
    uint64_t* const ks = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* k1 = n_pad <= a.smem_cap ? ks : kg;
    uint64_t* k2 = 2 * n_pad <= a.smem_cap ? ks + n_pad : kg + a.sort_cap;
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x)
        k1[i] = i < n ? (((uint64_t)__ldcg((const long long*)rec_f + i) << 32) | (uint32_t)i)
                      : ~0ull;
    __syncthreads();
    bitonic_sort(k1, n_pad);
    int cnt = n;
    const uint64_t* order = k1;  // entries [0, cnt) in frequency order
    if (n > K) {
        // rank by magnitude (larger first, lower frequency on ties), keep K, re-sort ranks
        for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
            uint64_t kk = ~0ull;
            if (i < n) {
                const uint32_t idx = (uint32_t)(k1[i] & 0xffffffffu);
                kk = ((uint64_t)(~mag_key(__ldcg(rec_v + idx))) << 32) | (uint32_t)i;
            }
            k2[i] = kk;
        }
        __syncthreads();
        bitonic_sort(k2, n_pad);
        for (int i = threadIdx.x; i < n_pad; i += blockDim.x)
            k2[i] = i < K ? (k2[i] & 0xffffffffu) : ~0ull;
        __syncthreads();
        bitonic_sort(k2, n_pad);
        cnt = K;
    }
    int64_t* oi = a.out_idx ? a.out_idx[sig] : a.idx0;
    XV* ov = reinterpret_cast<XV*>(a.out_val ? a.out_val[sig] : a.val0);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint64_t e = n > K ? order[k2[i]] : order[i];
        const uint32_t idx = (uint32_t)(e & 0xffffffffu);
        oi[i] = (int64_t)(e >> 32);
        const V v = __ldcg(rec_v + idx);
        ov[i] = XV{(XS)v.x, (XS)v.y};
    }
    if (threadIdx.x == 0) {
        int32_t* info = a.info_rows ? a.info_rows[sig] : a.infos + 4 * sig;
        const int err = ldv(ctr + kCtrErr);
        const int resolved = ldv(ctr + kCtrResolved);
        info[0] = cnt;
        info[1] = err ? -4 : (resolved < nb ? 2 : 0);
        info[2] = ldv(ctr + kCtrRounds);
        info[3] = ldv(ctr + kCtrIdents);
    }
    // leave the slot's counters zeroed for the next execution (every thread has read
    // what it needs above: rec count at the start, the rest by thread 0)
    __syncthreads();
    int32_t* wctr = const_cast<int32_t*>(ctr);
    for (int i = threadIdx.x; i < a.ctr_stride; i += blockDim.x) wctr[i] = 0;
}

// Noise-variance estimate (thresholds without a given sigma^2): a bin holding only noise
// has R delays of CN(0, B sigma^2) values, so e = sum_r |Y_r|^2 / B is sigma^2 times a
// Gamma(R, 1) variable; sigma^2 = (lower median of e over the signal's bins) / median of
// Gamma(R, 1).  NE1: one thread per (signal, bin) writes e (FP32) into the slot's cf array,
// which the decode only uses later.
template <typename T>
__global__ void noise_energy_kernel(const __grid_constant__ DecodeArgs a)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)a.n_sig * pd.sumB) return;
    const int sig = (int)(gid / pd.sumB), b = (int)(gid - (int64_t)sig * pd.sumB);
    const V* Y = reinterpret_cast<const V*>(a.bins) + (int64_t)sig * pd.y_per_sig;
    const int d = stage_of(pd, b);
    const StageDesc& st = pd.st[d];
    const V* Yb = Y + st.y_off + (b - st.bin_base);
    T E = 0;
    for (int r = 0; r < pd.R; ++r) {
        const V y = __ldcg(Yb + (int64_t)r * st.B);
        E += y.x * y.x + y.y * y.y;
    }
    reinterpret_cast<float*>(a.ws.cf)[(int64_t)sig * pd.sumB * 2 + b] = (float)(E / (T)st.B);
}

// NE2: one CTA per signal; the lower median (rank floor((n - 1) / 2) from the smallest) of
// the n = sumB energies by an 8-bit radix select on their FP32 bit patterns, then sigma^2.
__global__ void __launch_bounds__(1024) noise_median_kernel(const __grid_constant__ DecodeArgs a)
{
    const PlanDesc& pd = a.pd;
    const int sig = blockIdx.x;
    const int n = pd.sumB;
    const uint32_t* e = reinterpret_cast<const uint32_t*>(a.ws.cf) + (int64_t)sig * n * 2;
    __shared__ unsigned int hist[256];
    __shared__ uint32_t s_prefix;
    __shared__ int s_need;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_need = (n - 1) / 2 + 1;  // 1-based rank from the smallest
    }
    uint32_t mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t u = __ldcg(e + i);
            if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cum = 0;
            const int need = s_need;
            for (int dg = 0; dg < 256; ++dg) {
                if (cum + (int)hist[dg] >= need) {
                    s_prefix = prefix | ((uint32_t)dg << shift);
                    s_need = need - cum;
                    break;
                }
                cum += (int)hist[dg];
            }
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.ws.sig2[sig] = (double)__uint_as_float(s_prefix) / pd.gmed;
}

cudaError_t launch_noise_estimate(const DecodeArgs& a, int precision, cudaStream_t st)
{
    if (a.n_sig == 0) return cudaSuccess;
    const int64_t n = (int64_t)a.n_sig * a.pd.sumB;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (precision == 1)
        noise_energy_kernel<float><<<g, 256, 0, st>>>(a);
    else
        noise_energy_kernel<double><<<g, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    noise_median_kernel<<<(unsigned)a.n_sig, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_classify(const DecodeArgs& a, int precision, cudaStream_t st)
{
    const int tiles = (a.pd.sumB + kClassifyTile - 1) / kClassifyTile;
    const unsigned grid = (unsigned)a.n_sig * (unsigned)tiles;
    if (grid == 0) return cudaSuccess;
    const size_t smem = a.wtab_smem ? (size_t)a.wtab_elems * (precision == 1 ? 8 : 16) : 0;
    if (precision == 1)
        classify_kernel<float><<<grid, kClassifyThreads, smem, st>>>(a);
    else
        classify_kernel<double><<<grid, kClassifyThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_decode(const DecodeArgs& a, int precision, int threads, bool cooperative,
                          cudaStream_t st)
{
    const unsigned grid = (unsigned)a.n_sig * (unsigned)a.G;
    if (grid == 0) return cudaSuccess;
    void* fn = precision == 1 ? (void*)peel_kernel<float> : (void*)peel_kernel<double>;
    if (cooperative) {
        void* args[] = {(void*)&a};
        return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, 0, st);
    }
    if (precision == 1)
        peel_kernel<float><<<grid, threads, 0, st>>>(a);
    else
        peel_kernel<double><<<grid, threads, 0, st>>>(a);
    return cudaGetLastError();
}

int decode_occupancy(int precision, int threads)
{
    int nb = 0;
    void* fn = precision == 1 ? (void*)peel_kernel<float> : (void*)peel_kernel<double>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_compact(const CompactArgs& a, int precision, int xdouble, int threads,
                           size_t smem, cudaStream_t st)
{
    const unsigned grid = (unsigned)a.n_sig;
    if (grid == 0) return cudaSuccess;
    if (precision == 1) {
        if (xdouble)
            compact_kernel<float, double><<<grid, threads, smem, st>>>(a);
        else
            compact_kernel<float, float><<<grid, threads, smem, st>>>(a);
    } else {
        if (xdouble)
            compact_kernel<double, double><<<grid, threads, smem, st>>>(a);
        else
            compact_kernel<double, float><<<grid, threads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t set_classify_smem_limit(int max_smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(classify_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  max_smem)))
        return e;
    return cudaFuncSetAttribute(classify_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem);
}

cudaError_t set_compact_smem_limit(int max_smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(compact_kernel<float, float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(compact_kernel<float, double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(compact_kernel<double, float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    return cudaFuncSetAttribute(compact_kernel<double, double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

}  // namespace sfft
