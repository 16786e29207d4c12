// dft.cu -- bucketization kernels: strided delayed gather (Eq. 5, with the shift of
// Eq. 3-4) fused with the B-point DFTs of Eq. 6 / Eq. 19.
//
// Each B_d-point DFT is split by the prime-factor (Good-Thomas) map into co-prime
// prime-power axes, so no twiddles are needed between axes: odd axes are done as direct
// DFTs with the conjugate-pair symmetry (a 2P-real-FMA inner product per output pair),
// power-of-two axes as in-place radix-2 decimation-in-time FFTs.  A tile of the stage
// array lives in shared memory for a whole pass.  When B_d fits in shared memory the stage
// is one pass straight from x to the bins; otherwise the outer axes run first (from x into
// scratch) and the inner axes second (scratch to bins).  The direct odd-axis DFTs are dense
// contractions (a cosine and a sine matrix applied to every sub-DFT): in FP32 stages those
// with 17 <= P <= 127 run on the tensor cores (3-term split FP16 MMAs with FP32
// accumulation, FP32-level accuracy),
// the rest on the FMA pipes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "sfft_internal.cuh"

namespace sfft {

// x / d and x % d for 0 <= x < 2^22 through a float reciprocal, corrected by one step
__device__ __forceinline__ int fdivmod(int x, int d, float inv, int* rem)
{
    int q = (int)((float)x * inv);
    int r = x - q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
    *rem = r;
    return q;
}

// In-place P-point DFTs (P odd) along one axis of a shared-memory tile.
//   sub-DFT m starts at (m % LS) + (m / LS) * LS * P, element n at + n * LS.
// X_k = x_0 + sum_{n=1}^{(P-1)/2} [ (x_n + x_{P-n}) cos(2 pi n k / P)
//                                   - i (x_n - x_{P-n}) sin(2 pi n k / P) ],
// X_{P-k} the same with the sine term negated.  Thread (g, m) computes GP output pairs
// k = g GP + 1 .. g GP + GP of sub-DFT m; the twiddle matrix row n (cos, sin)(2 pi n k / P)
// is read as 16-byte vectors that every lane of a warp shares.
template <typename T, int GP>
__device__ void axis_dft_odd(typename C2<T>::t* s, const typename C2<T>::t* twm, int P, int LS,
                             int TS)
{
    using V = typename C2<T>::t;
    const int M = TS / P;
    const int pairs = (P - 1) >> 1;
    const int KP = odd_row_len(P);  // row length of the twiddle matrix (a multiple of GP)
    const int NG = KP / GP;
    const float invLS = 1.0f / (float)LS;
    // pre-pass: (x_n, x_{P-n}) -> (a_n, b_n) = (x_n + x_{P-n}, x_n - x_{P-n}) in place
    {
        const int items = M * pairs;
        const float invp = 1.0f / (float)pairs;
        for (int w = threadIdx.x; w < items; w += blockDim.x) {
            int n, lo;
            const int m = fdivmod(w, pairs, invp, &n);
            const int hi = fdivmod(m, LS, invLS, &lo);
            const int base = lo + hi * LS * P;
            const int pa = base + (n + 1) * LS, pb = base + (P - 1 - n) * LS;
            const V xa = s[pa], xb = s[pb];
            s[pa] = V{xa.x + xb.x, xa.y + xb.y};
            s[pb] = V{xa.x - xb.x, xa.y - xb.y};
        }
        __syncthreads();
    }
    // column chunks of equal size (at most blockDim / NG columns each)
    const int Mmax = max(1, (int)blockDim.x / NG);
    const int nch = (M + Mmax - 1) / Mmax;
    const int Mc = (M + nch - 1) / nch;
    const int g = threadIdx.x / Mc;
    const int ml = threadIdx.x - g * Mc;
    for (int m0 = 0; m0 < M; m0 += Mc) {
        const int m = m0 + ml;
        const bool act = g < NG && m < M && m < m0 + Mc;
        V acc[GP], sac[GP];
        V x0 = {0, 0}, dc = {0, 0};
        int base = 0;
        if (act) {
            int lo;
            const int hi = fdivmod(m, LS, invLS, &lo);
            base = lo + hi * LS * P;
            x0 = s[base];
            dc = x0;
#pragma unroll
            for (int i = 0; i < GP; ++i) {
                acc[i] = {0, 0};
                sac[i] = {0, 0};
            }
            const V* row = twm + g * GP;
            const V* pa = s + base + LS;
            const V* pb = s + base + (P - 1) * LS;
#pragma unroll 2
            for (int n = 1; n <= pairs; ++n, row += KP, pa += LS, pb -= LS) {
                const V av = *pa;  // x_n + x_{P-n}
                const V bv = *pb;  // x_n - x_{P-n}
                if (g == 0) {
                    dc.x += av.x;
                    dc.y += av.y;
                }
                V w[GP];
                if constexpr (sizeof(V) == 8 && GP >= 2) {
#pragma unroll
                    for (int i = 0; i < GP / 2; ++i) {
                        const float4 q = reinterpret_cast<const float4*>(row)[i];
                        w[2 * i] = V{q.x, q.y};
                        w[2 * i + 1] = V{q.z, q.w};
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < GP; ++i) w[i] = row[i];
                }
#pragma unroll
                for (int i = 0; i < GP; ++i) {
                    acc[i].x = fma(av.x, w[i].x, acc[i].x);
                    acc[i].y = fma(av.y, w[i].x, acc[i].y);
                    sac[i].x = fma(bv.x, w[i].y, sac[i].x);
                    sac[i].y = fma(bv.y, w[i].y, sac[i].y);
                }
            }
        }
        __syncthreads();
        if (act) {
            if (g == 0) s[base] = dc;
#pragma unroll
            for (int i = 0; i < GP; ++i) {
                const int k = g * GP + 1 + i;
                if (k > pairs) continue;
                const V c = {x0.x + acc[i].x, x0.y + acc[i].y};
                s[base + k * LS] = V{c.x + sac[i].y, c.y - sac[i].x};
                s[base + (P - k) * LS] = V{c.x - sac[i].y, c.y + sac[i].x};
            }
        }
        __syncthreads();
    }
}

// In-place decimation-in-time FFTs of length P = 2^log2P along one axis; the input is
// stored bit-reversed along the axis, the output comes out in natural order.  Up to three
// radix-2 stages run per pass in registers (a radix-8 group of elements i h, i < 8, of a
// block), so the tile makes ceil(log2P / 3) trips through shared memory.
// tw[t] = (cos, sin)(2 pi t / P), t < P / 2; the butterfly of the stage with half-size H
// multiplies by W_P^{(p mod H) P / (2 H)}.
// nst < log2P runs only the first nst stages (the caller does the rest); lh0 > 0 starts at
// stage lh0 (the first lh0 done already).
template <typename T>
__device__ void axis_fft_pow2(typename C2<T>::t* s, const typename C2<T>::t* tw, int P,
                              int log2P, int LS, int TS, int nst, int lh0 = 0)
{
    using V = typename C2<T>::t;
    const int M = TS / P;
    for (int lh = lh0; lh < nst;) {
        const int c = min(3, nst - lh);
        const int G8 = 1 << c;
        const int h = 1 << lh;
        const int ngrp = P >> c;
        const int nw = M * ngrp;
        const float invM = 1.0f / (float)M, invLS = 1.0f / (float)LS;
        const int lg = log2P - c;  // ngrp = 2^lg
        for (int w = threadIdx.x; w < nw; w += blockDim.x) {
            int gi, m;
            if (LS == 1) {
                gi = w & (ngrp - 1);
                m = w >> lg;
            } else {
                gi = fdivmod(w, M, invM, &m);
            }
            const int ii = gi & (h - 1), blk = gi >> lh;
            int lo;
            const int hi = LS == 1 ? m : fdivmod(m, LS, invLS, &lo);
            const int base = LS == 1 ? m * P : lo + hi * LS * P;
            const int p0 = base + (blk * (G8 * h) + ii) * LS;
            const int st = h * LS;
            V v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < G8) v[i] = s[p0 + i * st];
#pragma unroll
            for (int sg = 0; sg < 3; ++sg) {
                if (sg >= c) break;
                const int hs = 1 << sg;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (i >= G8 || (i & hs)) continue;
                    const int t = (ii + (i & (hs - 1)) * h) << (log2P - 1 - lh - sg);
                    const V wv = tw[t];
                    const V u = v[i], x = v[i + hs];
                    const V xt = {fma(x.x, wv.x, x.y * wv.y), fma(x.y, wv.x, -(x.x * wv.y))};
                    v[i] = V{u.x + xt.x, u.y + xt.y};
                    v[i + hs] = V{u.x - xt.x, u.y - xt.y};
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < G8) s[p0 + i * st] = v[i];
        }
        __syncthreads();
        lh += c;
    }
}

// Odd-axis DFT on columns [c0, c1), each thread computing GP output pairs of CM columns
// (m and m + Mc, so the lanes of a warp touch consecutive columns).  Expects the
// (a_n, b_n) pre-pass done.  A chunk holds every group of its columns, so the in-place
// writes after the barrier cannot clobber inputs another thread still reads.
// With GP = 8 a thread does 32 FMAs per 2 shared loads of data and 4 (broadcast) of
// twiddles.  Kept out of line so that each variant gets its own register allocation.
template <typename T, int GP, int CM>
__device__ __noinline__ void odd_dft_cols(typename C2<T>::t* s, const typename C2<T>::t* twm, int P, int LS,
                             int c0, int c1)
{
    using V = typename C2<T>::t;
    const int pairs = (P - 1) >> 1;
    const int KP = odd_row_len(P);
    const int NG = KP / GP;
    const int Mc = max(1, (int)blockDim.x / NG);
    const int span = Mc * CM;
    const int g = threadIdx.x / Mc;
    const int ml = threadIdx.x - g * Mc;
    const float invLS = 1.0f / (float)LS;
    for (int m0 = c0; m0 < c1; m0 += span) {
        const int lim = min(c1, m0 + span);
        bool act[CM];
        int base[CM];
        V x0[CM], dc[CM], acc[CM][GP], sac[CM][GP];
#pragma unroll
        for (int c = 0; c < CM; ++c) {
            const int m = m0 + ml + c * Mc;
            act[c] = g < NG && m < lim;
            int lo;
            const int hi = fdivmod(act[c] ? m : m0, LS, invLS, &lo);
            base[c] = lo + hi * LS * P;
        }
        if (act[0]) {
#pragma unroll
            for (int c = 0; c < CM; ++c) {
                x0[c] = s[base[c]];
                dc[c] = x0[c];
#pragma unroll
                for (int i = 0; i < GP; ++i) {
                    acc[c][i] = {0, 0};
                    sac[c][i] = {0, 0};
                }
            }
            const V* row = twm + g * GP;
#pragma unroll 2
            for (int n = 1; n <= pairs; ++n, row += KP) {
                V w[GP];
                if constexpr (sizeof(V) == 8 && GP >= 2) {
#pragma unroll
                    for (int i = 0; i < GP / 2; ++i) {
                        const float4 q = reinterpret_cast<const float4*>(row)[i];
                        w[2 * i] = V{q.x, q.y};
                        w[2 * i + 1] = V{q.z, q.w};
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < GP; ++i) w[i] = row[i];
                }
#pragma unroll
                for (int c = 0; c < CM; ++c) {
                    const V av = s[base[c] + n * LS];        // x_n + x_{P-n}
                    const V bv = s[base[c] + (P - n) * LS];  // x_n - x_{P-n}
                    if (g == 0) {
                        dc[c].x += av.x;
                        dc[c].y += av.y;
                    }
#pragma unroll
                    for (int i = 0; i < GP; ++i) {
                        acc[c][i].x = fma(av.x, w[i].x, acc[c][i].x);
                        acc[c][i].y = fma(av.y, w[i].x, acc[c][i].y);
                        sac[c][i].x = fma(bv.x, w[i].y, sac[c][i].x);
                        sac[c][i].y = fma(bv.y, w[i].y, sac[c][i].y);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CM; ++c) {
            if (!act[c]) continue;
            if (g == 0) s[base[c]] = dc[c];
#pragma unroll
            for (int i = 0; i < GP; ++i) {
                const int k = g * GP + 1 + i;
                if (k > pairs) continue;
                const V cc = {x0[c].x + acc[c][i].x, x0[c].y + acc[c][i].y};
                s[base[c] + k * LS] = V{cc.x + sac[c][i].y, cc.y - sac[c][i].x};
                s[base[c] + (P - k) * LS] = V{cc.x - sac[c][i].y, cc.y + sac[c][i].x};
            }
        }
        __syncthreads();
    }
}

// (a_n, b_n) pre-pass of an odd axis: (x_n, x_{P-n}) -> (x_n + x_{P-n}, x_n - x_{P-n})
template <typename T>
__device__ void odd_prepass(typename C2<T>::t* s, int P, int LS, int TS)
{
    using V = typename C2<T>::t;
    const int M = TS / P, pairs = (P - 1) >> 1;
    const float invLS = 1.0f / (float)LS, invp = 1.0f / (float)pairs;
    for (int w = threadIdx.x; w < M * pairs; w += blockDim.x) {
        int n, lo;
        const int m = fdivmod(w, pairs, invp, &n);
        const int hi = fdivmod(m, LS, invLS, &lo);
        const int base = lo + hi * LS * P;
        const int pa = base + (n + 1) * LS, pb = base + (P - 1 - n) * LS;
        const V xa = s[pa], xb = s[pb];
        s[pa] = V{xa.x + xb.x, xa.y + xb.y};
        s[pb] = V{xa.x - xb.x, xa.y - xb.y};
    }
    __syncthreads();
}

template <typename T, int G2>
__device__ __forceinline__ void odd_tail(typename C2<T>::t* s, const typename C2<T>::t* tw, int P,
                                         int LS, int c0, int c1)
{
    // leftover columns: the smallest GP whose groups x columns fit one chunk
    const int KP = odd_row_len(P), rem = c1 - c0, nt = blockDim.x;
    if ((KP / 1) * rem <= nt)
        odd_dft_cols<T, 1, 1>(s, tw, P, LS, c0, c1);
    else if (G2 >= 2 && (KP / 2) * rem <= nt)
        odd_dft_cols<T, (G2 >= 2 ? 2 : 1), 1>(s, tw, P, LS, c0, c1);
    else if (G2 >= 4 && (KP / 4) * rem <= nt)
        odd_dft_cols<T, (G2 >= 4 ? 4 : 1), 1>(s, tw, P, LS, c0, c1);
    else
        odd_dft_cols<T, G2, 1>(s, tw, P, LS, c0, c1);
}

// Odd axis with P <= 9: one thread per column computes the whole P-point DFT in
// registers (it owns its column, so no barrier is needed until the axis is done).
template <typename T>
__device__ __noinline__ void odd_small(typename C2<T>::t* s, const typename C2<T>::t* twm, int P, int LS, int TS)
{
    using V = typename C2<T>::t;
    const int M = TS / P, pairs = (P - 1) >> 1, KP = odd_row_len(P);
    const float invLS = 1.0f / (float)LS;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int lo;
        const int hi = fdivmod(m, LS, invLS, &lo);
        const int base = lo + hi * LS * P;
        const V x0 = s[base];
        V av[4], bv[4], dc = x0;
#pragma unroll
        for (int n = 1; n <= 4; ++n) {
            if (n > pairs) break;
            const V xa = s[base + n * LS], xb = s[base + (P - n) * LS];
            av[n - 1] = V{xa.x + xb.x, xa.y + xb.y};
            bv[n - 1] = V{xa.x - xb.x, xa.y - xb.y};
            dc.x += av[n - 1].x;
            dc.y += av[n - 1].y;
        }
        s[base] = dc;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            if (k > pairs) break;
            V A = x0, S = {0, 0};
#pragma unroll
            for (int n = 1; n <= 4; ++n) {
                if (n > pairs) break;
                const V w = twm[(n - 1) * KP + (k - 1)];
                A.x = fma(av[n - 1].x, w.x, A.x);
                A.y = fma(av[n - 1].y, w.x, A.y);
                S.x = fma(bv[n - 1].x, w.y, S.x);
                S.y = fma(bv[n - 1].y, w.y, S.y);
            }
            s[base + k * LS] = V{A.x + S.y, A.y - S.x};
            s[base + (P - k) * LS] = V{A.x - S.y, A.y + S.x};
        }
    }
    __syncthreads();
}

// FP32 odd axis: pre-pass, then the bulk of the columns in full chunks of GP = odd_group_
// pairs(P) pairs per thread, then the leftover columns in one small chunk.
template <int G2>
__device__ void odd_axis_f32(float2* s, const float2* tw, int P, int LS, int TS)
{
    const int M = TS / P, KP = odd_row_len(P);
    const int span = max(1, (int)blockDim.x / (KP / G2));
    const int main_end = M / span * span;
    odd_prepass<float>(s, P, LS, TS);
    if (main_end > 0) odd_dft_cols<float, G2, 1>(s, tw, P, LS, 0, main_end);
    if (main_end < M) odd_tail<float, G2>(s, tw, P, LS, main_end, M);
}

// Output pairs per thread for an odd axis: the twiddle matrix rows are padded for
// odd_group_pairs(P); any GP dividing that works.  At most 4 pairs per thread keep the
// 640-thread CTA within its register budget; pick the GP that minimises (balanced column
// chunks) x GP -- the per-thread work of the axis.
template <typename T>
__device__ __forceinline__ void axis_dft_odd_dispatch(typename C2<T>::t* s,
                                                      const typename C2<T>::t* tw, int P,
                                                      int LS, int TS)
{
    const int gmax = odd_group_pairs(P);
    if (gmax < 4) {
        if (gmax == 1)
            axis_dft_odd<T, 1>(s, tw, P, LS, TS);
        else
            axis_dft_odd<T, 2>(s, tw, P, LS, TS);
        return;
    }
    const int KP = odd_row_len(P), M = TS / P, nt = blockDim.x;
    int best_gp = 0, best_cost = 0;
    for (int gp = 4; gp >= 2; gp >>= 1) {
        const int ng = KP / gp;
        const int mc = max(1, nt / ng);
        const int cost = (M + mc - 1) / mc * gp;
        if (best_gp == 0 || cost < best_cost) {
            best_gp = gp;
            best_cost = cost;
        }
    }
    if (best_gp == 4)
        axis_dft_odd<T, 4>(s, tw, P, LS, TS);
    else
        axis_dft_odd<T, 2>(s, tw, P, LS, TS);
}

// ---- odd axes on the tensor cores (FP32 tiles) ------------------------------------------
// With a_n = x_n + x_{P-n} and b_n = x_n - x_{P-n} the P-point DFTs of an odd axis are two
// real matrix products over the H = (P + 1) / 2 inputs n = 0 .. (P - 1) / 2 and outputs
// k = 0 .. (P - 1) / 2:
//   C[k][c] = sum_n cos(2 pi n k / P) A[n][c],   A[n] = x_0 (n = 0), a_n (n >= 1)
//   S[k][c] = sum_n sin(2 pi n k / P) Bs[n][c],  Bs[n] = 0 (n = 0), b_n (n >= 1)
// over the real columns c (the real and imaginary parts of every sub-DFT); then X_0 = C_0,
// X_k = C_k - i S_k and X_{P-k} = C_k + i S_k.  Each product runs as m16n8k16 FP16 MMAs
// with FP32 accumulation and both operands split into FP16 high and low parts, keeping the
// three largest partial products (hi hi + hi lo + lo hi) -- the split-operand scheme of
// Ootomo and Yokota (2022) with FP16 parts: FP16 has TF32's 11-bit significand, so the
// dropped terms are again about 2^-22 of the product and the result keeps FP32-level
// accuracy, while an FP16 MMA covers 16 inputs where a TF32 one covers 8.  FP16's range is
// kept by a power-of-two scale per axis call (the tile's largest component mapped into
// [2^13, 2^14), undone exactly on the accumulators).  The cosine and sine matrices come
// pre-split in fragment order (the axis' twiddle table in global memory, see
// tc_twiddle_word, read through the read-only cache); the data come straight from the tile
// in shared memory, so nothing is staged beside the resident tile.

// WPG warps per column group of 8 sub-DFTs (an n-tile of their real parts and one of their
// imaginary parts), each for MR of the row tiles, so each data fragment is loaded and split
// once per warp and a thread ends up holding C and S, real and imaginary, of the same
// sub-DFT and output row.  With one warp per group (WPG = 1) a warp overwrites only its own
// columns and needs no block barrier until the axis is done; with two, the warps of a chunk
// of groups all read before a barrier and overwrite after it.  Input rows 4 apart in a k-tile
// (tc_row) put the 16 lanes of a half-warp (4 rows x 4 columns) in distinct shared-memory
// banks when the columns are an odd number of elements apart (LS = 1, column stride P) or
// adjacent (odd LS).
template <int MR, int WPG>
__device__ __noinline__ void odd_dft_tc(float2* s, const uint4* frag, int P, int LS, int TS,
                                        float sc, float isc)
{
    const int M = TS / P, pairs = (P - 1) >> 1;
    const int KK = tc_ktiles(P) >> 1;
    const int NG = (M + 7) >> 3;
    const int W = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int GPC = W / WPG;                 // groups per chunk
    const int part = warp % WPG, m0 = part * MR;
    const bool wact = warp < GPC * WPG;
    const int g = lane >> 2, t = lane & 3;
    const float invLS = 1.0f / (float)LS;
    for (int c0 = (WPG == 1 ? warp : 0); c0 < NG; c0 += (WPG == 1 ? W : GPC)) {
        const int grp = WPG == 1 ? c0 : c0 + warp / WPG;
        const bool act = wact && grp < NG;
        float acc[MR][4][4];  // [row tile][C re, C im, S re, S im][fragment]
#pragma unroll
        for (int m = 0; m < MR; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[m][q][e] = 0.0f;
        if (act) {
            const int cc = grp * 8 + g;
            int src = -1;
            if (cc < M) {
                int lo;
                const int hi = fdivmod(cc, LS, invLS, &lo);
                src = lo + hi * LS * P;
            }
            for (int kk = 0; kk < KK; ++kk) {
                // (a_n, b_n) = (x_n + x_{P-n}, x_n - x_{P-n}), scaled, formed as the fragments
                // are loaded (a_0 = x_0, b_0 = 0): slot 2 t + j of the k-tile is row
                // tc_row(2 kk + j, t), slot 2 t + 8 + j row tc_row(2 kk + j, t + 4)
                float2 av[2][2], bv[2][2];  // [t or t + 4][j]
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int n = tc_row(2 * kk + j, t + 4 * p);
                        float2 a = {0.0f, 0.0f}, b = a;
                        if (src >= 0 && n <= pairs) {
                            const float2 u = s[src + n * LS];
                            if (n == 0) {
                                a = u;
                            } else {
                                const float2 v = s[src + (P - n) * LS];
                                a = float2{u.x + v.x, u.y + v.y};
                                b = float2{u.x - v.x, u.y - v.y};
                            }
                        }
                        av[p][j] = float2{a.x * sc, a.y * sc};
                        bv[p][j] = float2{b.x * sc, b.y * sc};
                    }
                uint32_t arh[2], arl[2], aih[2], ail[2], brh[2], brl[2], bih[2], bil[2];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    f16_split2(av[p][0].x, av[p][1].x, arh[p], arl[p]);
                    f16_split2(av[p][0].y, av[p][1].y, aih[p], ail[p]);
                    f16_split2(bv[p][0].x, bv[p][1].x, brh[p], brl[p]);
                    f16_split2(bv[p][0].y, bv[p][1].y, bih[p], bil[p]);
                }
                const uint4* fk = frag + ((size_t)m0 * KK + kk) * 128 + lane;
#pragma unroll
                for (int m = 0; m < MR; ++m) {
                    const uint4* fm = fk + (size_t)m * KK * 128;
                    const uint4 ch = __ldg(fm), cl = __ldg(fm + 32);
                    const uint4 sh = __ldg(fm + 64), sl = __ldg(fm + 96);
                    // the three partial products of the four accumulators, interleaved so
                    // that no MMA waits on the one before it; small terms first
                    mma_f16(acc[m][0], cl, arh[0], arh[1]);
                    mma_f16(acc[m][1], cl, aih[0], aih[1]);
                    mma_f16(acc[m][2], sl, brh[0], brh[1]);
                    mma_f16(acc[m][3], sl, bih[0], bih[1]);
                    mma_f16(acc[m][0], ch, arl[0], arl[1]);
                    mma_f16(acc[m][1], ch, ail[0], ail[1]);
                    mma_f16(acc[m][2], sh, brl[0], brl[1]);
                    mma_f16(acc[m][3], sh, bil[0], bil[1]);
                    mma_f16(acc[m][0], ch, arh[0], arh[1]);
                    mma_f16(acc[m][1], ch, aih[0], aih[1]);
                    mma_f16(acc[m][2], sh, brh[0], brh[1]);
                    mma_f16(acc[m][3], sh, bih[0], bih[1]);
                }
            }
        }
        if constexpr (WPG == 1)
            __syncwarp();
        else
            __syncthreads();
        if (act) {
#pragma unroll
            for (int hc = 0; hc < 2; ++hc) {
                const int cw = grp * 8 + 2 * t + hc;
                if (cw >= M) continue;
                int lo;
                const int hi = fdivmod(cw, LS, invLS, &lo);
                const int base = lo + hi * LS * P;
#pragma unroll
                for (int m = 0; m < MR; ++m)
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int k = (m0 + m) * 16 + g + 8 * r, e = 2 * r + hc;
                        if (k > pairs) continue;
                        const float cr = acc[m][0][e] * isc, ci = acc[m][1][e] * isc;
                        const float sr = acc[m][2][e] * isc, si = acc[m][3][e] * isc;
                        if (k == 0) {
                            s[base] = float2{cr, ci};
                        } else {
                            s[base + k * LS] = float2{cr + si, ci - sr};
                            s[base + (P - k) * LS] = float2{cr - si, ci + sr};
                        }
                    }
            }
        }
        if constexpr (WPG == 1) __syncwarp();
    }
    __syncthreads();
}

// Row tiles per warp: all of them up to three (one warp per column group); four row tiles
// (P > 95) are split over two warps, which keeps the accumulators within the register budget.
__device__ __forceinline__ void odd_axis_tc(float2* s, const float2* tw, int P, int LS, int TS)
{
    const uint4* frag = reinterpret_cast<const uint4*>(tw);
    // the tile's largest component, for the FP16 operands' scale
    __shared__ float red[32];
    float mx = 0.0f;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) {
        const float2 v = s[i];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mx = fmaxf(mx, red[i]);
    __syncthreads();  // red is free again
    // largest component into [2^13, 2^14): a_n = x_n + x_{P-n} stays below 2^15 (tiles of
    // only tiny values, below 2^-100, get the scale of 2^-100: their FP16 parts underflow)
    const int e = mx > 0.0f ? max(ilogbf(mx), -100) : 0;
    const float sc = ldexpf(1.0f, 13 - e), isc = ldexpf(1.0f, e - 13);
    switch (tc_mtiles(P)) {
        case 1: odd_dft_tc<1, 1>(s, frag, P, LS, TS, sc, isc); break;
        case 2: odd_dft_tc<2, 1>(s, frag, P, LS, TS, sc, isc); break;
        case 3: odd_dft_tc<3, 1>(s, frag, P, LS, TS, sc, isc); break;
        default: odd_dft_tc<2, 2>(s, frag, P, LS, TS, sc, isc); break;
    }
}

// The store of a one-pass tile to the bins, with up to two axes done on the way (the axes of
// the prime-factor map commute, so they can run last): the last radix-2 stage of the
// power-of-two axis a2 (half size H = P2 / 2, twiddles tw2) and the whole small odd axis a3
// (3 <= P3 <= 9, conjugate-pair table tw3 as odd_small reads it).  A work item holds the
// 2 P3 (or P3, or 2) elements that differ only in those coordinates: one thread reads them,
// transforms them in registers and writes them to the bins, which saves the trips through
// shared memory (and the barriers) those axes would take on their own.  a2 / a3 = -1: none.
template <typename T, int P3>
__device__ __forceinline__ void store_fused_p(const typename C2<T>::t* s, typename C2<T>::t* dst,
                                              const StageDesc& st, int TS, int a2,
                                              const typename C2<T>::t* tw2, int a3,
                                              const typename C2<T>::t* tw3)
{
    using V = typename C2<T>::t;
    constexpr int pairs = (P3 - 1) / 2;
    const int S3 = a3 >= 0 ? st.ax[a3].S : 0;
    const int H = a2 >= 0 ? st.ax[a2].P >> 1 : 1, HS2 = a2 >= 0 ? H * st.ax[a2].S : 0;
    const int J = a2 >= 0 ? 2 : 1;
    const int KP = odd_row_len(P3);
    const int W = TS / (P3 * J);
    // the item index in mixed radix over the other axes (axis a2 with radix H), innermost
    // first; the last digit needs no division
    // (fully unrolled over the axis slots so that the digits stay in registers)
    int Rr[kMaxAxes], Sr[kMaxAxes];
    float inv[kMaxAxes];
    const int nax = st.n_axes;
#pragma unroll
    for (int ax = 0; ax < kMaxAxes; ++ax) {
        const bool live = ax < nax && ax != a3;
        Rr[ax] = !live ? 1 : ax == a2 ? H : st.ax[ax].P;
        Sr[ax] = live ? st.ax[ax].S : 0;
        inv[ax] = 1.0f / (float)Rr[ax];
    }
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        // position of the item's first element, and its coordinate k < H on axis a2
        int rem = w, base = 0, k = 0;
#pragma unroll
        for (int ax = 0; ax < kMaxAxes; ++ax) {
            if (ax >= nax) break;
            int c;
            rem = fdivmod(rem, Rr[ax], inv[ax], &c);
            if (ax == a2) k = c;
            base += c * Sr[ax];
        }
        V v[2][P3];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < P3; ++i)
                if (j < J) v[j][i] = s[base + i * S3 + j * HS2];
        if (a2 >= 0) {
            const V wv = tw2[k];
#pragma unroll
            for (int i = 0; i < P3; ++i) {
                const V u = v[0][i], x = v[1][i];
                const V xt = {fma(x.x, wv.x, x.y * wv.y), fma(x.y, wv.x, -(x.x * wv.y))};
                v[0][i] = V{u.x + xt.x, u.y + xt.y};
                v[1][i] = V{u.x - xt.x, u.y - xt.y};
            }
        }
        if constexpr (P3 > 1) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (j >= J) break;
                const V x0 = v[j][0];
                V av[pairs], bv[pairs], dc = x0;
#pragma unroll
                for (int n = 1; n <= pairs; ++n) {
                    const V xa = v[j][n], xb = v[j][P3 - n];
                    av[n - 1] = V{xa.x + xb.x, xa.y + xb.y};
                    bv[n - 1] = V{xa.x - xb.x, xa.y - xb.y};
                    dc.x += av[n - 1].x;
                    dc.y += av[n - 1].y;
                }
                v[j][0] = dc;
#pragma unroll
                for (int kk = 1; kk <= pairs; ++kk) {
                    V A = x0, S = {0, 0};
#pragma unroll
                    for (int n = 1; n <= pairs; ++n) {
                        const V c = tw3[(n - 1) * KP + (kk - 1)];
                        A.x = fma(av[n - 1].x, c.x, A.x);
                        A.y = fma(av[n - 1].y, c.x, A.y);
                        S.x = fma(bv[n - 1].x, c.y, S.x);
                        S.y = fma(bv[n - 1].y, c.y, S.y);
                    }
                    v[j][kk] = V{A.x + S.y, A.y - S.x};
                    v[j][P3 - kk] = V{A.x - S.y, A.y + S.x};
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < P3; ++i)
                if (j < J) __stcg(dst + base + i * S3 + j * HS2, v[j][i]);
    }
}

template <typename T>
__device__ __noinline__ void store_fused(const typename C2<T>::t* s, typename C2<T>::t* dst,
                                         const StageDesc& st, int TS, int a2,
                                         const typename C2<T>::t* tw2, int a3,
                                         const typename C2<T>::t* tw3)
{
    switch (a3 >= 0 ? st.ax[a3].P : 1) {
        case 3: store_fused_p<T, 3>(s, dst, st, TS, a2, tw2, a3, tw3); break;
        case 5: store_fused_p<T, 5>(s, dst, st, TS, a2, tw2, a3, tw3); break;
        case 7: store_fused_p<T, 7>(s, dst, st, TS, a2, tw2, a3, tw3); break;
        case 9: store_fused_p<T, 9>(s, dst, st, TS, a2, tw2, a3, tw3); break;
        default: store_fused_p<T, 1>(s, dst, st, TS, a2, tw2, -1, tw3); break;
    }
}

// The tensor-core axes of a one-pass tile (run after its other axes: the axes of the
// prime-factor map commute), then the tile's fused store to the bins (store_fused, with the
// deferred radix-2 stage of axis a2 and the small odd axis a3).  Out of line, so that the
// kernel holds nothing live across the MMA code.
__device__ __noinline__ void tc_axes_store(float2* s, const BucketArgs& a, int d, int64_t slot,
                                           int TS, int a2, const float2* tw2, int a3,
                                           const float2* tw3)
{
    const StageDesc& st = a.pd.st[d];
    const float2* twg = reinterpret_cast<const float2*>(a.tw);
    for (int ax = 0; ax < st.n_axes; ++ax) {
        const AxisDesc& A = st.ax[ax];
        if (A.tc) odd_axis_tc(s, twg + A.tw_off, A.P, A.S, TS);  // one pass: stride A.S
    }
    store_fused<float>(s, reinterpret_cast<float2*>(a.bins) + slot, st, TS, a2, tw2, a3, tw3);
}

__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc, int bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename XS, typename V>
__device__ __forceinline__ V load_sample(const void* x, int32_t i)
{
    using XV = typename C2<XS>::t;
    const XV v = __ldg(reinterpret_cast<const XV*>(x) + i);
    return V{(decltype(V{}.x))v.x, (decltype(V{}.x))v.y};
}

// a sample of a page-locked host signal read in place (plain load, cached in L2 only)
template <typename XS, typename V>
__device__ __forceinline__ V load_sample_host(const void* x, int32_t i)
{
    using XV = typename C2<XS>::t;
    const XV v = __ldcg(reinterpret_cast<const XV*>(x) + i);
    return V{(decltype(V{}.x))v.x, (decltype(V{}.x))v.y};
}

// One block = one tile of one (signal, stage, delay).  Block order within a signal:
// (stage, tile, delay), so the delays of a tile run back to back and share x's sectors.
// TC: the launch holds tensor-core odd axes (FP32 only).  Without them the tensor-core path
// is compiled out, which keeps the register allocation of the other paths free of it.
template <typename T, typename XS, bool TC>
__global__ void __launch_bounds__(512, 1) bucketize_kernel(const __grid_constant__ BucketArgs a)
{
    using V = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);

    const int tps = a.tiles_per_sig;
    const int sig = blockIdx.x / tps;
    int rem = blockIdx.x - sig * tps;
    int d = 0;
    while (rem >= a.tile_prefix[d + 1]) ++d;
    rem -= a.tile_prefix[d];
    const StageDesc& st = a.pd.st[d];
    const PassDesc& ps = a.pass[d];
    const int R = a.pd.R;
    const int tile = rem / R;
    const int r = rem - tile * R;

    const int a0 = ps.a0, a1 = ps.a1;
    const int Sb = st.ax[a0].S;
    int G = 1;
    for (int ax = a0; ax < a1; ++ax) G *= st.ax[ax].P;
    const int Sab = Sb * G;
    const int above = st.B / Sab;
    const int Tb = ps.Tb, Ta = ps.Ta;
    const int nTb = (Sb + Tb - 1) / Tb;
    const int tb0 = (tile % nTb) * Tb;
    const int ta0 = (tile / nTb) * Ta;
    const int TS = ps.tile_elems;
    V* tws = s + ((TS + 1) & ~1);  // 16-byte aligned: twiddle rows are read as 16-byte vectors

    // twiddles of this pass' axes
    {
        const V* twg = reinterpret_cast<const V*>(a.tw);
        int off = 0;
        for (int ax = a0; ax < a1; ++ax) {
            const int n = axis_tw_smem(st.ax[ax].P, st.ax[ax].pow2, st.ax[ax].tc, st.ax[ax].gmem);
            for (int t = threadIdx.x; t < n; t += blockDim.x) tws[off + t] = twg[st.ax[ax].tw_off + t];
            off += (n + 1) & ~1;
        }
    }

    const int64_t slot = (int64_t)sig * a.pd.y_per_sig + st.y_off + (int64_t)r * st.B;
    const void* x = a.xs ? a.xs[sig] : a.x0;
    const int tau = st.tau[r], L = st.L, N = a.pd.N;
    const int32_t* nidx = a.nidx + st.bin_base;
    const V* scr = reinterpret_cast<const V*>(a.scratch);

    // a host signal read in place takes the register loads of the general path below (no
    // asynchronous copies from host memory)
    const bool host_src = a.x_sys && ps.src_gather;
    int pow2_done = 0;  // radix-2 stages of the outermost axis done in the gather
    if constexpr (sizeof(XS) == sizeof(T)) {
        // a whole-stage tile whose outermost axis is a power of two (stored bit-reversed):
        // each work item gathers the 2^c samples of one radix-8 group of that axis into
        // registers and runs the axis' first c radix-2 stages on them before its single
        // store, which saves the axis a trip through shared memory (c <= 3; the rest of the
        // axis runs in axis_fft_pow2 from stage c on, the last stage in the store)
        const int ao = st.n_axes - 1;
        if (ps.src_gather && Tb == 1 && Ta == 1 && !host_src && a0 == 0 && a1 == st.n_axes &&
            ps.dst_bins && st.ax[ao].pow2 && st.ax[ao].log2P >= 2) {
            const AxisDesc& A = st.ax[ao];
            const int P = A.P, S = A.S, lg = A.log2P;
            const int c = min(3, lg - 1), G8 = 1 << c;
            const int nw = S * (P >> c);
            const float invS = 1.0f / (float)S;
            const V* twp = reinterpret_cast<const V*>(a.tw) + A.tw_off;
            const V* xv = reinterpret_cast<const V*>(x);
            constexpr int UI = 2;  // work items per trip: their 16 loads in flight at once
            for (int w0 = threadIdx.x; w0 < nw; w0 += UI * blockDim.x) {
                V v[UI][8];
                int pos[UI];
                bool ok[UI];
#pragma unroll
                for (int k = 0; k < UI; ++k) {
                    int w = w0 + k * blockDim.x;
                    ok[k] = w < nw;
                    if (!ok[k]) w = w0;
                    int m;
                    const int blk = fdivmod(w, S, invS, &m);
                    pos[k] = m + blk * G8 * S;
                    int src[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) src[i] = i < G8 ? __ldg(nidx + pos[k] + i * S) : 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (i >= G8) continue;
                        int xi = src[i] * L + tau;
                        xi = xi >= N ? xi - N : xi;
                        v[k][i] = __ldg(xv + xi);
                    }
                }
#pragma unroll
                for (int k = 0; k < UI; ++k)
#pragma unroll
                    for (int sg = 0; sg < 3; ++sg) {
                        if (sg >= c) break;
                        const int hs = 1 << sg;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (i >= G8 || (i & hs)) continue;
                            const V wv = __ldg(twp + ((i & (hs - 1)) << (lg - 1 - sg)));
                            const V u = v[k][i], xx = v[k][i + hs];
                            const V xt = {fma(xx.x, wv.x, xx.y * wv.y), fma(xx.y, wv.x, -(xx.x * wv.y))};
                            v[k][i] = V{u.x + xt.x, u.y + xt.y};
                            v[k][i + hs] = V{u.x - xt.x, u.y - xt.y};
                        }
                    }
#pragma unroll
                for (int k = 0; k < UI; ++k)
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < G8 && ok[k]) s[pos[k] + i * S] = v[k][i];
            }
            pow2_done = c;
            goto loaded;
        }
        if (ps.src_gather && Tb == 1 && Ta == 1 && !host_src) {
            // whole-stage tile straight from x: sample indices from the table, then
            // asynchronous 8/16-byte copies into shared memory, all in flight at once
            constexpr int U = 8;
            const V* xv = reinterpret_cast<const V*>(x);
            for (int e0 = threadIdx.x; e0 < TS; e0 += U * blockDim.x) {
                int src[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * blockDim.x;
                    src[u] = e < TS ? __ldg(nidx + e) : 0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < TS) {
                        int xi = src[u] * L + tau;
                        xi = xi >= N ? xi - N : xi;
                        cp_async(s + e, xv + xi, (int)sizeof(V));
                    }
                }
            }
            cp_async_wait_all();
            goto loaded;
        }
    }
    {
        // general tile (two-pass stages, or a conversion of the input type): 8 loads in
        // flight per thread
        constexpr int U = 8;
        for (int e0 = threadIdx.x; e0 < TS; e0 += U * blockDim.x) {
            int pos[U];
            int32_t src[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * blockDim.x;
                int p = -1;
                if (e < TS) {
                    if (Tb == 1 && Ta == 1) {
                        p = e;
                    } else {
                        const int tb = e % Tb;
                        const int rest = e / Tb;
                        const int g = rest % G;
                        const int ta = rest / G;
                        const int pb = tb0 + tb, pa = ta0 + ta;
                        if (pb < Sb && pa < above) p = pb + Sb * g + Sab * pa;
                    }
                }
                pos[u] = p;
                src[u] = 0;
                if (p >= 0) {
                    if (ps.src_gather) {
                        const int xi = __ldg(nidx + p) * L + tau;
                        src[u] = xi >= N ? xi - N : xi;
                    } else {
                        src[u] = p;
                    }
                }
            }
            bool done = false;
            if constexpr (sizeof(XS) == sizeof(T)) {
                if (!host_src) {
                    // samples of the arithmetic type: asynchronous copies straight into shared
                    // memory (positions outside the stage are zero)
                    const V* xv = reinterpret_cast<const V*>(x);
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = e0 + u * blockDim.x;
                        if (e >= TS) continue;
                        if (pos[u] < 0)
                            s[e] = V{0, 0};
                        else
                            cp_async(s + e, ps.src_gather ? xv + src[u] : scr + slot + src[u], (int)sizeof(V));
                    }
                    done = true;
                }
            }
            if (!done) {
                V v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    v[u] = V{0, 0};
                    if (pos[u] >= 0) {
                        if (!ps.src_gather)
                            v[u] = __ldcg(scr + slot + src[u]);
                        else if (host_src)
                            v[u] = load_sample_host<XS, V>(x, src[u]);
                        else
                            v[u] = load_sample<XS, V>(x, src[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < TS) s[e] = v[u];
                }
            }
        }
        if constexpr (sizeof(XS) == sizeof(T)) cp_async_wait_all();
    }
loaded:
    __syncthreads();

    bool stage_tc = false;  // stages with tensor-core axes are one-pass (whole stage, to the bins)
    for (int ax = a0; ax < a1; ++ax) stage_tc |= st.ax[ax].tc != 0;
    // a tile holding the whole stage (one pass, straight to the bins) defers the last radix-2
    // stage of its power-of-two axis and its first small odd axis to the fused store
    const bool whole = Tb == 1 && Ta == 1 && a0 == 0 && a1 == st.n_axes && ps.dst_bins;
    int a2 = -1, a3 = -1;
    const V* tw2 = nullptr;
    const V* tw3 = nullptr;
    int off = 0;
    for (int ax = a0; ax < a1; ++ax) {
        const AxisDesc& A = st.ax[ax];
        const int LS = Tb * (A.S / Sb);
        if (A.pow2) {
            const bool defer = whole;
            if (defer) {
                a2 = ax;
                tw2 = tws + off;
            }
            axis_fft_pow2<T>(s, tws + off, A.P, A.log2P, LS, TS, defer ? A.log2P - 1 : A.log2P, pow2_done);
        } else if (A.P > 1) {
            if (A.P <= 9) {
                if (whole && a3 < 0) {
                    a3 = ax;
                    tw3 = tws + off;
                } else {
                    odd_small<T>(s, tws + off, A.P, LS, TS);
                }
            } else {
                // the matrix of a larger odd axis: in shared memory, or read from the plan
                // table in global memory (gmem)
                const V* twa = A.gmem ? reinterpret_cast<const V*>(a.tw) + A.tw_off : tws + off;
                if constexpr (sizeof(T) == 4) {
                    if (!(TC && A.tc)) odd_axis_f32<8>(s, twa, A.P, LS, TS);
                } else
                    axis_dft_odd_dispatch<T>(s, twa, A.P, LS, TS);
            }
        }
        off += (axis_tw_smem(A.P, A.pow2, A.tc, A.gmem) + 1) & ~1;
    }
    if constexpr (TC && sizeof(T) == 4) {
        if (stage_tc) {
            tc_axes_store(reinterpret_cast<float2*>(s), a, d, slot, TS, a2,
                          reinterpret_cast<const float2*>(tw2), a3,
                          reinterpret_cast<const float2*>(tw3));
            return;
        }
    }
    if (whole) {
        store_fused<T>(s, reinterpret_cast<V*>(a.bins) + slot, st, TS, a2, tw2, a3, tw3);
        return;
    }

    V* dst = reinterpret_cast<V*>(ps.dst_bins ? a.bins : a.scratch);
    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
        int p;
        if (Tb == 1 && Ta == 1) {
            p = e;
        } else {
            const int tb = e % Tb;
            const int rest = e / Tb;
            const int g = rest % G;
            const int ta = rest / G;
            const int pb = tb0 + tb, pa = ta0 + ta;
            if (pb >= Sb || pa >= above) continue;
            p = pb + Sb * g + Sab * pa;
        }
        __stcg(dst + slot + p, s[e]);
    }
}

// ---- persistent one-pass bucketization with the next tile's gather overlapped ----------
// When a whole-stage FP32 tile fills more than half of shared memory, one CTA fits an SM
// and, in bucketize_kernel, a tile's scattered gather cannot overlap another tile's DFTs.
// Here one persistent CTA per SM takes the work items (signal, stage, delay) round robin
// and keeps two tile regions at the two ends of shared memory: A = [0, region) and
// B = [off_b, off_b + region), overlapping in the middle when 2 region > smem.  While the
// current item is transformed in one region, the next item's samples that fall outside it
// are already being copied (asynchronous 8-byte copies) into the other; the rest of them
// follow once the current item is stored.

// asynchronous copies of samples [e_lo, e_hi) of the item (sig, d, r) into tile s
__device__ __forceinline__ void gather_issue(float2* s, const BucketArgs& a, int sig, int d, int r,
                                             int e_lo, int e_hi)
{
    const StageDesc& st = a.pd.st[d];
    const float2* xv = reinterpret_cast<const float2*>(a.xs ? a.xs[sig] : a.x0);
    const int tau = st.tau[r], L = st.L, N = a.pd.N;
    const int32_t* nidx = a.nidx + st.bin_base;
    constexpr int U = 8;
    for (int e0 = e_lo + threadIdx.x; e0 < e_hi; e0 += U * blockDim.x) {
        int src[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            src[u] = e < e_hi ? __ldg(nidx + e) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < e_hi) {
                int xi = src[u] * L + tau;
                xi = xi >= N ? xi - N : xi;
                cp_async(s + e, xv + xi, 8);
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void stream_item(const BucketArgs& a, int w, int* sig, int* d, int* r)
{
    *sig = w / a.tiles_per_sig;
    int rem = w - *sig * a.tiles_per_sig;
    int dd = 0;
    while (rem >= a.tile_prefix[dd + 1]) ++dd;
    *d = dd;
    *r = rem - a.tile_prefix[dd];  // one tile per (stage, delay)
}

template <bool TC>
__global__ void __launch_bounds__(512, 1)
    bucketize_stream_kernel(const __grid_constant__ BucketArgs a, int32_t region, int32_t off_b)
{
    using V = float2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* const sm = reinterpret_cast<V*>(smem_raw);
    const int n_items = a.n_sig * a.tiles_per_sig;
    int w = blockIdx.x;
    if (w >= n_items) return;
    int sig, d, r;
    stream_item(a, w, &sig, &d, &r);
    int cur = 0;  // region of the current item: 0 = A, 1 = B
    gather_issue(sm, a, sig, d, r, 0, a.pd.st[d].B);
    for (; w < n_items; w += gridDim.x) {
        V* s = cur ? sm + off_b : sm;
        const StageDesc& st = a.pd.st[d];
        const int TS = st.B;
        V* tws = s + ((TS + 1) & ~1);
        {
            const V* twg = reinterpret_cast<const V*>(a.tw);
            int off = 0;
            for (int ax = 0; ax < st.n_axes; ++ax) {
                const int n = axis_tw_smem(st.ax[ax].P, st.ax[ax].pow2, st.ax[ax].tc, st.ax[ax].gmem);
                for (int t = threadIdx.x; t < n; t += blockDim.x) tws[off + t] = twg[st.ax[ax].tw_off + t];
                off += (n + 1) & ~1;
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        // the next item's samples outside this region, copied while this one is transformed
        const int wn = w + gridDim.x;
        int sn = 0, dn = 0, rn = 0, lo = 0, hi = 0, TSn = 0;
        if (wn < n_items) {
            stream_item(a, wn, &sn, &dn, &rn);
            TSn = a.pd.st[dn].B;
            if (cur == 0) {  // next in B: element e lies outside A when off_b + e >= region
                lo = min(TSn, max(0, region - off_b));
                gather_issue(sm + off_b, a, sn, dn, rn, lo, TSn);
            } else {         // next in A: outside B when e < off_b
                hi = min(TSn, off_b);
                gather_issue(sm, a, sn, dn, rn, 0, hi);
            }
        }
        const int64_t slot = (int64_t)sig * a.pd.y_per_sig + st.y_off + (int64_t)r * st.B;
        bool stage_tc = false;
        for (int ax = 0; ax < st.n_axes; ++ax) stage_tc |= st.ax[ax].tc != 0;
        int a2 = -1, a3 = -1;
        const V* tw2 = nullptr;
        const V* tw3 = nullptr;
        int off = 0;
        for (int ax = 0; ax < st.n_axes; ++ax) {
            const AxisDesc& A = st.ax[ax];
            if (A.pow2) {
                a2 = ax;
                tw2 = tws + off;
                axis_fft_pow2<float>(s, tws + off, A.P, A.log2P, A.S, TS, A.log2P - 1);
            } else if (A.P > 1) {
                if (A.P <= 9) {
                    if (a3 < 0) {
                        a3 = ax;
                        tw3 = tws + off;
                    } else {
                        odd_small<float>(s, tws + off, A.P, A.S, TS);
                    }
                } else if (!(TC && A.tc)) {
                    odd_axis_f32<8>(s, A.gmem ? reinterpret_cast<const V*>(a.tw) + A.tw_off : tws + off,
                                    A.P, A.S, TS);
                }
            }
            off += (axis_tw_smem(A.P, A.pow2, A.tc, A.gmem) + 1) & ~1;
        }
        if (TC && stage_tc)
            tc_axes_store(s, a, d, slot, TS, a2, tw2, a3, tw3);
        else
            store_fused<float>(s, reinterpret_cast<V*>(a.bins) + slot, st, TS, a2, tw2, a3, tw3);
        __syncthreads();  // this region is read for the last time above
        if (wn < n_items) {
            if (cur == 0)
                gather_issue(sm + off_b, a, sn, dn, rn, 0, lo);
            else
                gather_issue(sm, a, sn, dn, rn, hi, TSn);
        }
        sig = sn;
        d = dn;
        r = rn;
        cur ^= 1;
    }
}

template <typename T>
__global__ void twiddle_kernel(typename C2<T>::t* tw, const int32_t* P_of, const int32_t* t_of,
                               int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (sizeof(T) == 4) {
        if (P_of[i] < 0) {  // fragment table of a tensor-core odd axis: -P, entry index
            tw[i] = typename C2<T>::t{__uint_as_float(tc_twiddle_word(-P_of[i], 2 * t_of[i])),
                                      __uint_as_float(tc_twiddle_word(-P_of[i], 2 * t_of[i] + 1))};
            return;
        }
    }
    if (P_of[i] == 0) {  // padding entry
        tw[i] = typename C2<T>::t{(T)0, (T)0};
        return;
    }
    double sv, cv;
    sincospi(2.0 * (double)t_of[i] / (double)P_of[i], &sv, &cv);
    tw[i] = typename C2<T>::t{(T)cv, (T)sv};
}

// bins in storage order <-> natural order [stage][delay][j] for one signal
template <typename T>
__global__ void bins_natural_kernel(const __grid_constant__ PlanDesc pd, const int32_t* pbin,
                                    const typename C2<T>::t* src, typename C2<T>::t* dst,
                                    int to_natural)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.y_per_sig) return;
    int d = 0;
    while (d + 1 < pd.D && i >= pd.st[d + 1].y_off) ++d;
    const StageDesc& st = pd.st[d];
    const int64_t rel = i - st.y_off;
    const int r = (int)(rel / st.B);
    const int p = (int)(rel - (int64_t)r * st.B);
    const int j = pbin[st.bin_base + p];
    const int64_t nat = st.y_off + (int64_t)r * st.B + j;
    if (to_natural)
        dst[nat] = src[i];
    else
        dst[i] = src[nat];
}

// does any stage's pass in this launch hold a tensor-core odd axis (fragment table)
static bool launch_has_tc(const BucketArgs& a)
{
    for (int d = 0; d < a.pd.D; ++d)
        for (int ax = a.pass[d].a0; ax < a.pass[d].a1; ++ax) {
            if (a.pd.st[d].ax[ax].tc) return true;
        }
    return false;
}

cudaError_t launch_bucketize(const BucketArgs& a, int precision, int xdouble, int threads,
                             size_t smem, cudaStream_t st)
{
    const unsigned grid = (unsigned)a.n_sig * (unsigned)a.tiles_per_sig;
    if (grid == 0) return cudaSuccess;
    if (precision == 1) {
        const bool tc = launch_has_tc(a);
        if (xdouble) {
            if (tc)
                bucketize_kernel<float, double, true><<<grid, threads, smem, st>>>(a);
            else
                bucketize_kernel<float, double, false><<<grid, threads, smem, st>>>(a);
        } else {
            if (tc)
                bucketize_kernel<float, float, true><<<grid, threads, smem, st>>>(a);
            else
                bucketize_kernel<float, float, false><<<grid, threads, smem, st>>>(a);
        }
    } else {
        if (xdouble)
            bucketize_kernel<double, double, false><<<grid, threads, smem, st>>>(a);
        else
            bucketize_kernel<double, float, false><<<grid, threads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

// the persistent overlapped variant (FP32 arithmetic and samples, one-pass stages, device
// memory): grid CTAs, all of shared memory (smem bytes), tile regions of `region` elements
cudaError_t launch_bucketize_stream(const BucketArgs& a, int grid, int threads, size_t smem,
                                    int region, cudaStream_t st)
{
    const int n_items = a.n_sig * a.tiles_per_sig;
    if (n_items == 0) return cudaSuccess;
    if (grid > n_items) grid = n_items;
    const int off_b = (int)((smem / 8 - (size_t)region) & ~(size_t)1);
    if (off_b < 0) return cudaErrorInvalidValue;
    if (launch_has_tc(a))
        bucketize_stream_kernel<true><<<grid, threads, smem, st>>>(a, region, off_b);
    else
        bucketize_stream_kernel<false><<<grid, threads, smem, st>>>(a, region, off_b);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(void* tw, const int32_t* P_of, const int32_t* t_of, int64_t n,
                            int precision, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (precision == 1)
        twiddle_kernel<float><<<grid, 256, 0, st>>>((float2*)tw, P_of, t_of, n);
    else
        twiddle_kernel<double><<<grid, 256, 0, st>>>((double2*)tw, P_of, t_of, n);
    return cudaGetLastError();
}

cudaError_t launch_bins_to_natural(const PlanDesc& pd, const int32_t* pbin, const void* src,
                                   void* dst, int precision, int to_natural, cudaStream_t st)
{
    const unsigned grid = (unsigned)((pd.y_per_sig + 255) / 256);
    if (precision == 1)
        bins_natural_kernel<float><<<grid, 256, 0, st>>>(pd, pbin, (const float2*)src, (float2*)dst,
                                                         to_natural);
    else
        bins_natural_kernel<double><<<grid, 256, 0, st>>>(pd, pbin, (const double2*)src,
                                                          (double2*)dst, to_natural);
    return cudaGetLastError();
}

cudaError_t set_bucketize_smem_limit(int max_smem)
{
    const void* fns[] = {(const void*)bucketize_kernel<float, float, false>,
                         (const void*)bucketize_kernel<float, float, true>,
                         (const void*)bucketize_kernel<float, double, false>,
                         (const void*)bucketize_kernel<float, double, true>,
                         (const void*)bucketize_kernel<double, float, false>,
                         (const void*)bucketize_kernel<double, double, false>,
                         (const void*)bucketize_stream_kernel<false>,
                         (const void*)bucketize_stream_kernel<true>};
    for (const void* fn : fns) {
        // the opt-in limit covers static and dynamic shared memory together
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sfft
