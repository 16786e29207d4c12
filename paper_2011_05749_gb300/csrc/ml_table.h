// ml_table.h -- host side of the first round's ML candidate search on the tensor cores
// (Sec. 3.2 subproblem 2, the search over the L candidates j + q B of a bin, run as the
// product A [Re Z; Im Z] with A holding the conjugated candidate phasors): the words of a
// stage's table of split TF32 A fragments, built once per plan in the layout locate_ml_tc
// reads.
#pragma once
#include <math.h>
#include <stdint.h>

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

}  // namespace sfft
