// ml_table.h -- host side of the first round's ML candidate search on the tensor cores
// (Sec. 3.2 subproblem 2, the search over the L candidates j + q B of a bin, run as the
// product A [Re Z; Im Z] with A holding the conjugated candidate phasors): the words of a
// stage's table of split A fragments, built once per plan, in the two layouts the search
// reads -- split FP16 for m16n8k16 MMAs (locate_ml_tc16, the default) and split TF32 for
// m16n8k8 MMAs (locate_ml_tc).
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cuda_fp16.h>

#include "sfft_internal.cuh"

namespace sfft {

// Word e of lane l's fragment in part h (0: TF32 high parts, 1: low) of fragment tile
// (mt, kt) of a stage's table, for L candidates and R delays with residues tauL[r] = tau_r
// mod L.  The tile is rows 16 mt .. 16 mt + 15 and columns 8 kt .. 8 kt + 7 of A, where row
// g < 8 of a tile is Re c_q and row g + 8 is Im c_q for q = 8 mt + g, and column k < RP
// multiplies Re Z_k, column RP + k multiplies Im Z_k (RP = ml_tc_rp(R)), so that
// c_q = sum_r Z_r conj(e^{2 pi i (q tauL_r mod L) / L}).  Lane l, register e holds
// row l / 4 + 8 (e & 1), column l % 4 + 4 (e >> 1): the m16n8k8 TF32 A-fragment layout.
// Entries past L or R are zero; the phasors are FP64 rounded to FP32, then split.
inline uint32_t ml_tc_word(int L, int R, const int32_t* tauL, int mt, int kt, int h, int l, int e)
{
    const int RP = ml_tc_rp(R);
    const int row = (l >> 2) + (e & 1) * 8, k = kt * 8 + (l & 3) + (e >> 1) * 4;
    const int q = mt * 8 + (row & 7), im = row >> 3;
    const int part = k / RP, r = k % RP;
    float v = 0.0f;
    if (q < L && r < R) {
        const double two_pi = 6.283185307179586476925286766559;
        const double th = two_pi * (double)(((int64_t)q * tauL[r]) % L) / (double)L;
        const double cv = cos(th), sv = sin(th);
        v = (float)(im == 0 ? (part == 0 ? cv : sv) : (part == 0 ? -sv : cv));
    }
    union {
        float f;
        uint32_t u;
    } b;
    b.f = v;
    uint32_t hi, lo;
    tf32_split_bits(b.u, &hi, &lo);
    return h == 0 ? hi : lo;
}

// The FP16 table's entries are the phasor parts times 2^kMlTc16Scale: the low parts of
// entries down to |cos| ~ 1e-2 stay in FP16's normal range.  A power of two applied to
// every candidate of a bin alike leaves its argmax unchanged, so the search never undoes it.
constexpr int kMlTc16Scale = 8;
// k-tiles of 16 of the FP16 layout: delays 8 kk .. 8 kk + 7 per k-tile
inline int ml_tc16_ktiles(int R) { return (R + 7) >> 3; }

// Word e of lane l's fragment in part h (0: FP16 high parts, 1: low) of fragment tile
// (mt, kk) of a stage's FP16 table.  The tile is rows 16 mt .. 16 mt + 15 of A (row g < 8:
// Re c_q, row g + 8: Im c_q, q = 8 mt + g, as in the TF32 layout) and the 16 columns of
// k-tile kk: column k' < 8 multiplies Re Z_{8 kk + k'}, column 8 + k' multiplies
// Im Z_{8 kk + k'}.  Lane l = 4 g + t, register e holds row g + 8 (e & 1), columns
// 2 t + 8 (e >> 1) and the next one, the lower column in the low half: the m16n8k16 FP16
// A-fragment layout.  Each entry is the FP64 phasor part rounded to FP32 and scaled by
// 2^kMlTc16Scale, then split: high = the value rounded to FP16, low = the remainder rounded
// to FP16.  Entries past L or R are zero.
inline uint32_t ml_tc16_word(int L, int R, const int32_t* tauL, int mt, int kk, int h, int l, int e)
{
    const int g = l >> 2, t = l & 3, im = e & 1, q = mt * 8 + g;
    uint16_t half[2];
    for (int j = 0; j < 2; ++j) {
        const int kc = 2 * t + 8 * (e >> 1) + j;  // column within the k-tile
        const int part = kc >> 3, r = 8 * kk + (kc & 7);
        float v = 0.0f;
        if (q < L && r < R) {
            const double two_pi = 6.283185307179586476925286766559;
            const double th = two_pi * (double)(((int64_t)q * tauL[r]) % L) / (double)L;
            const double cv = cos(th), sv = sin(th);
            v = ldexpf((float)(im == 0 ? (part == 0 ? cv : sv) : (part == 0 ? -sv : cv)), kMlTc16Scale);
        }
        const __half hv = __float2half_rn(v);
        const __half lv = __float2half_rn(v - __half2float(hv));
        memcpy(&half[j], h == 0 ? &hv : &lv, 2);
    }
    return (uint32_t)half[0] | ((uint32_t)half[1] << 16);
}

}  // namespace sfft
