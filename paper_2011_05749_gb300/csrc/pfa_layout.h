// pfa_layout.h -- host-side layout of one stage's B-point DFT: prime-power axes, their
// order, the one- or two-pass split and the tiles of each pass (no heap allocation).
#pragma once
#include <stdint.h>

#include "sfft_internal.cuh"

namespace sfft {

inline int64_t pfa_gcd(int64_t a, int64_t b)
{
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

inline int64_t pfa_inv_mod(int64_t a, int64_t m)
{
    if (m == 1) return 0;
    int64_t g = m, x = 0, x1 = 1, b = a % m;
    while (b) {
        const int64_t q = g / b;
        int64_t t = g - q * b;
        g = b;
        b = t;
        t = x - q * x1;
        x = x1;
        x1 = t;
    }
    x %= m;
    return x < 0 ? x + m : x;
}

// even number of elements, so every twiddle block starts on a 16-byte boundary
inline int64_t pfa_even(int64_t n) { return (n + 1) & ~(int64_t)1; }

// Prime-power factors of B: odd ones descending, then the power of two.  -1 if more than cap.
inline int pfa_prime_powers(int64_t B, int32_t* out, int cap)
{
    int n = 0;
    int64_t pw2 = 1;
    while (B % 2 == 0) {
        B /= 2;
        pw2 *= 2;
    }
    for (int64_t p = 3; p * p <= B; p += 2) {
        if (B % p) continue;
        int64_t q = 1;
        while (B % p == 0) {
            B /= p;
            q *= p;
        }
        if (n == cap) return -1;
        out[n++] = (int32_t)q;
    }
    if (B > 1) {
        if (n == cap) return -1;
        out[n++] = (int32_t)B;
    }
    // largest odd factor first (innermost): every other odd axis then has a stride of at
    // least that factor, so the lanes of a warp walk consecutive shared-memory words
    for (int i = 1; i < n; ++i)
        for (int k = i; k > 0 && out[k - 1] < out[k]; --k) {
            const int32_t t = out[k];
            out[k] = out[k - 1];
            out[k - 1] = t;
        }
    if (pw2 > 1) {
        if (n == cap) return -1;
        out[n++] = (int32_t)pw2;
    }
    if (n == 0) out[n++] = 1;
    return n;
}

inline bool pfa_is_pow2(int32_t P) { return P > 1 && (P & (P - 1)) == 0; }

inline int64_t pfa_tw_elems(int32_t P, int tc)
{
    return pfa_even(axis_tw_count(P, pfa_is_pow2(P) ? 1 : 0, tc));
}
inline int64_t pfa_tw_smem(int32_t P, int tc, int gmem)
{
    return pfa_even(axis_tw_smem(P, pfa_is_pow2(P) ? 1 : 0, tc, gmem));
}

struct PassPlan {
    size_t smem = 0;     // dynamic shared memory of the launch
    int64_t tile = 0;    // largest tile of the launch
};

// Lay out stage s (B and L already set).  esz: bytes per complex element; max_smem: the
// device's opt-in shared memory per block.  *tw_cursor advances past this stage's
// twiddles.  allow_tc = false keeps every odd axis on the FMA pipes.  Returns false when an
// axis is not supported or no split fits.
inline bool pfa_layout_stage(StageDesc* s, size_t esz, int max_smem, int64_t tile_target,
                             PassDesc* p1, PassDesc* p2, PassPlan* l1, PassPlan* l2,
                             int32_t* tw_cursor, bool* two_pass, int64_t max_tile = 0,
                             bool allow_tc = true)
{
    const int64_t B = s->B;
    int32_t Ps[kMaxAxes];
    const int n = pfa_prime_powers(B, Ps, kMaxAxes);
    if (n < 0) return false;
    for (int i = 0; i < n; ++i)
        if (!pfa_is_pow2(Ps[i]) && Ps[i] > 2049) return false;  // direct DFT: <= 1024 pairs
    const int64_t cap = (int64_t)max_smem - 1024;                // bytes for tile + twiddles
    auto fits = [&](int64_t elems, int64_t tw) {
        return (pfa_even(elems) + tw) * (int64_t)esz <= cap && (max_tile <= 0 || elems <= max_tile);
    };
    // a stage in one pass gets tensor-core odd axes (tables outside shared memory); the
    // passes of a two-pass stage keep every axis on the FMA pipes
    const int fp32 = esz == 8 ? 1 : 0;
    auto tc_of = [&](int32_t P) { return allow_tc && !pfa_is_pow2(P) && odd_tc(P, fp32) ? 1 : 0; };
    // a one-pass tile filling more than half of shared memory (one CTA per SM): the matrices
    // of odd axes above P = 9 stay in global memory
    const bool big = 2 * pfa_even(B) * (int64_t)esz > (int64_t)max_smem;
    auto gmem_of = [&](int32_t P) { return big && !pfa_is_pow2(P) && P > 9 ? 1 : 0; };
    int64_t tw_one = 0;
    for (int i = 0; i < n; ++i) tw_one += pfa_tw_smem(Ps[i], tc_of(Ps[i]), gmem_of(Ps[i]));
    int32_t order[kMaxAxes];
    int split = n;
    for (int i = 0; i < n; ++i) order[i] = Ps[i];
    const bool one_pass = fits(B, tw_one);
    if (!one_pass) {
        int64_t best = -1;
        unsigned best_mask = 0;
        for (unsigned mask = 1; mask + 1 < (1u << n); ++mask) {
            int64_t pi = 1, twi = 0, two = 0;
            for (int i = 0; i < n; ++i) {
                if (mask >> i & 1) {
                    pi *= Ps[i];
                    twi += pfa_tw_smem(Ps[i], 0, 0);
                } else {
                    two += pfa_tw_smem(Ps[i], 0, 0);
                }
            }
            const int64_t po = B / pi;
            if (!fits(pi, twi) || !fits(po, two)) continue;
            const int64_t worst = pi > po ? pi : po;
            if (best < 0 || worst < best) {
                best = worst;
                best_mask = mask;
            }
        }
        if (best < 0) return false;
        int k = 0;
        for (int i = 0; i < n; ++i)
            if (best_mask >> i & 1) order[k++] = Ps[i];
        split = k;
        for (int i = 0; i < n; ++i)
            if (!(best_mask >> i & 1)) order[k++] = Ps[i];
    }
    s->n_axes = n;
    s->split = split;
    int32_t S = 1;
    int64_t tw_in = 0, tw_out = 0;
    for (int i = 0; i < n; ++i) {
        AxisDesc& A = s->ax[i];
        A.P = order[i];
        A.pow2 = pfa_is_pow2(A.P) ? 1 : 0;
        A.log2P = 0;
        while ((1 << A.log2P) < A.P) ++A.log2P;
        if (!A.pow2) A.log2P = 0;
        A.S = S;
        S *= A.P;
        const int64_t Bp = B / A.P;
        A.rur = (int32_t)(Bp % B);
        A.crt = (int32_t)((Bp * pfa_inv_mod(Bp % A.P, A.P)) % B);
        A.tc = one_pass ? tc_of(A.P) : 0;
        A.gmem = A.tc || (one_pass && gmem_of(A.P)) ? 1 : 0;
        A.tw_off = *tw_cursor;
        *tw_cursor += (int32_t)pfa_tw_elems(A.P, A.tc);
        (i < split ? tw_in : tw_out) += pfa_tw_smem(A.P, A.tc, A.gmem);
    }
    auto note = [&](PassPlan* l, int64_t tile, int64_t tw) {
        const size_t b = (size_t)(pfa_even(tile) + tw) * esz;
        if (b > l->smem) l->smem = b;
        if (tile > l->tile) l->tile = tile;
    };
    *p2 = PassDesc{0, 0, 1, 1, 0, 0, 0, 1};
    if (split == n) {
        *p1 = PassDesc{0, n, 1, 1, 1, (int32_t)B, 1, 1};
        note(l1, B, tw_in + tw_out);
        return true;
    }
    *two_pass = true;
    int64_t inner = 1, outer = 1;
    for (int i = 0; i < split; ++i) inner *= s->ax[i].P;
    for (int i = split; i < n; ++i) outer *= s->ax[i].P;
    if (max_tile > 0) tile_target = max_tile;  // the caller's B-tile sets the two-pass tiles
    int64_t Tb = tile_target / outer;
    if (Tb < 1) Tb = 1;
    if (Tb > inner) Tb = inner;
    while (Tb > 1 && !fits(Tb * outer, tw_out)) --Tb;
    int64_t Ta = tile_target / inner;
    if (Ta < 1) Ta = 1;
    if (Ta > outer) Ta = outer;
    while (Ta > 1 && !fits(Ta * inner, tw_in)) --Ta;
    *p1 = PassDesc{split, n, (int32_t)Tb, 1, (int32_t)((inner + Tb - 1) / Tb), (int32_t)(Tb * outer), 1, 0};
    *p2 = PassDesc{0, split, 1, (int32_t)Ta, (int32_t)((outer + Ta - 1) / Ta), (int32_t)(inner * Ta), 0, 1};
    note(l1, Tb * outer, tw_out);
    note(l2, inner * Ta, tw_in);
    return true;
}

// threads of a bucketization CTA: whole-stage tiles (one CTA per SM, shared memory bound)
// get 512 threads (the kernel's launch bound); smaller two-pass tiles one thread per 16
// elements, so that two CTAs fit an SM's registers
inline int pfa_threads(int64_t tile, size_t)
{
    if (tile >= 8192) return 512;
    int64_t t = (tile / 16 + 31) / 32 * 32;
    return (int)(t < 128 ? 128 : (t > 512 ? 512 : t));
}

}  // namespace sfft
