// sfft_internal.cuh -- descriptors and device helpers shared by the libsfft kernels.
//
// Data layout in HBM (per plan workspace, per signal slot s):
//   bins      [s][stage d][delay r][PFA position p]   complex (float2 / double2)
//             stage d starts at y_off_d = R * sum_{d'<d} B_d'; position p is the
//             prime-factor (Good-Thomas) storage order of the B_d outputs, see AxisDesc.
//   scratch   same shape as bins, used between the two passes of a two-pass DFT.
//   decode    per-bin state and lists, see DecodeWs.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sfft {

constexpr int kMaxStages = 4;
constexpr int kMaxDelays = 16;
constexpr int kMaxAxes = 6;

// One axis of the prime-factor decomposition B = prod_a P_a (pairwise co-prime prime
// powers).  Storage position p = sum_a c_a S_a.  Before an axis is transformed its
// coordinate c_a holds input index n_a (bit-reversed for power-of-two axes, which are
// transformed by in-place radix-2 decimation in time); afterwards it holds output k_a in
// natural order.  Input sample index (Ruritanian map): n = sum_a n_a (B / P_a) mod B.
// Output bin (CRT map): j = sum_a k_a crt_a mod B, crt_a = (B/P_a) ((B/P_a)^-1 mod P_a).
struct AxisDesc {
    int32_t P;
    int32_t pow2;    // 1: power of two
    int32_t log2P;
    int32_t S;       // stride in the stage array
    int32_t rur;     // (B / P) mod B
    int32_t crt;     // CRT coefficient
    int32_t tw_off;  // offset of this axis' twiddles in the plan twiddle table
    int32_t tc;      // 1: odd axis done on the tensor cores (fragment table, see odd_tc)
    int32_t gmem;    // 1: the axis' table is read from global memory (not copied to shared)
};

// One DFT pass over a contiguous range of axes [a0, a1) of a stage.  A tile is Tb
// consecutive positions of the dims below a0 times the axes [a0, a1) times Ta consecutive
// positions of the dims from a1 up.
struct PassDesc {
    int32_t a0, a1;
    int32_t Tb, Ta;
    int32_t n_tiles;      // tiles per (signal, delay); 0 = stage not in this launch
    int32_t tile_elems;   // Tb * prod P * Ta
    int32_t src_gather;   // 1: load from x, 0: load from scratch
    int32_t dst_bins;     // 1: store to bins, 0: store to scratch
};

struct StageDesc {
    int32_t B, L;
    int32_t n_axes, split;   // axes [0, split) inner group, [split, n_axes) outer group
    AxisDesc ax[kMaxAxes];
    int32_t tau[kMaxDelays];
    int32_t tauL[kMaxDelays];  // tau mod L: candidate q of a bin shifts delay r's phase by
                               // e^{2 pi i q tauL_r / L}
    int32_t step32[kMaxDelays];  // (32 tauL_r) mod L: the same for q -> q + 32
    int32_t bin_base;        // sum of B of earlier stages
    int32_t y_off;           // R * bin_base
    int32_t r0, r1;          // delay slots holding tau = 0 and tau = 1 (-1 if absent)
    int32_t root_off;        // offset of the L roots of unity (cos, sin)(2 pi t / L)
    float invL;              // 1 / L
    int32_t wtab_off;        // offset of the [R][L] table W[r][q] = (cos, sin)(2 pi (q tauL_r mod L) / L)
    int32_t mltc_off;        // first fragment tile of the stage in the ML tensor-core table (-1 none)
    double T0, T1;           // thresholds on sum_r |Y_r|^2 and on the single-tone residual
    float T0f, T1f;          // the same in FP32 (the FP32 path compares in FP32)
    double T0a, T1a, Tb;     // T0 = T0a sigma^2 + Tb, T1 = T1a sigma^2 + Tb (estimated sigma^2)
};

struct PlanDesc {
    int32_t N;
    int32_t D, R;
    int32_t sumB;            // bins per delay over all stages
    int64_t y_per_sig;       // R * sumB
    int32_t locate;          // 0 ARG, 1 ML, 2 KAY
    int32_t max_rounds;
    int32_t K;
    int32_t root_total;      // sum_d L_d: root-table entries (at st[0].root_off onwards)
    double invN;             // 1 / N
    int32_t mode;            // 0 peeling (Sec. 3.2), 1 one-shot (Sec. 3.1, one stage)
    int32_t ph_shift;        // two-level phasor tables: e^{2 pi i m / N} =
    int32_t ph_lo_off;       //   tw[ph_hi_off + (m >> ph_shift)] * tw[ph_lo_off + (m & mask)]
    int32_t ph_hi_off;
    uint64_t mu;             // floor((2^64 - 1) / N): Barrett reduction modulo N
    int32_t am;              // one-shot: a_m (delay slots 0 .. 3 a_m - 1 hold -a_m .. 2 a_m - 1)
    int32_t kay_m;           // KAY locate: delays per iteration (slot c m + t holds r_c + t 2^c)
    double sv_floor;         // one-shot: singular values at or below this are not counted
    double sp_tol2;          // one-shot: residual tolerance of the subspace pursuit
    double gmed;             // median of Gamma(R, 1), for the sigma^2 estimate
    int32_t noise_auto;      // 1: thresholds from each signal's estimated sigma^2
    int32_t peel_atomic;     // 1: peeling subtracts with unordered atomics on the bins;
                             // 0: per-bin subtraction lists applied in frequency order with
                             //    compensated sums (deterministic)
    int32_t arg_mode;        // ARG locate: bit 0 = angle in FP32 (else FP64), bit 1 = no
                             // residue snap (f = the integer nearest the estimate)
    int32_t pad3;
    StageDesc st[kMaxStages];
};

// Twiddles of one axis in the plan table, as residues t of e^{2 pi i t / P}:
//   power of two: W^t for t < P/2 (radix-2 butterflies);
//   odd P: the (P-1)/2 x KP matrix of t = (n k) mod P, n, k = 1..(P-1)/2, rows padded to
//   KP = a multiple of the output pairs one thread computes (padding entries t = 0).
__host__ __device__ __forceinline__ int odd_group_pairs(int P)
{
    const int pairs = (P - 1) >> 1;
    return pairs <= 1 ? 1 : pairs <= 2 ? 2 : pairs <= 4 ? 4 : 8;
}
__host__ __device__ __forceinline__ int odd_row_len(int P)
{
    const int pairs = (P - 1) >> 1, gp = odd_group_pairs(P);
    return (pairs + gp - 1) / gp * gp;
}
// Odd axes with 17 <= P <= 127 of FP32 stages done in one pass (the whole stage in one
// tile) run their DFTs on the tensor cores instead (two real matrix products with the
// cosine and sine matrices, m16n8k16 FP16 MMAs with operands split into FP16 high and low
// parts); the layout marks them AxisDesc::tc.  Their table holds the MMAs' A fragments,
// already split: for row tile mt (16 outputs k), k-tile kk (16 inputs n) and quarter q
// (cos hi, cos lo, sin hi, sin lo), lane l's four fragment words sit at word
// ((mt KK + kk) 4 + q) 128 + 4 l, as in tc_twiddle_word.  odd_tc: whether P qualifies.
__host__ __device__ __forceinline__ bool odd_tc(int P, int fp32)
{
    return fp32 && (P & 1) && P >= 17 && P <= 127;
}
__host__ __device__ __forceinline__ int tc_mtiles(int P) { return ((P + 1) / 2 + 15) >> 4; }
// groups of 8 input rows (padded to blocks of 32); a k-tile of the MMAs holds two of them
__host__ __device__ __forceinline__ int tc_ktiles(int P) { return (((P + 1) / 2 + 31) >> 5) << 2; }
// input row n of slot i (0..7) of 8-row group kt: blocks of 32 rows, every fourth row.
// k-tile kk's slot 2 t + j is row tc_row(2 kk + j, t), its slot 2 t + 8 + j is row
// tc_row(2 kk + j, t + 4) (t = 0..3, j = 0, 1): the rows a lane holds, 4 apart within a
// block, put the 16 lanes of a half-warp in distinct shared-memory banks.
__host__ __device__ __forceinline__ int tc_row(int kt, int i)
{
    return (kt & 3) + ((kt >> 2) << 5) + (i << 2);
}
// entries of an axis' table; tc = AxisDesc::tc
__host__ __device__ __forceinline__ int axis_tw_count(int P, int pow2, int tc)
{
    if (P <= 1) return 0;
    if (tc) return tc_mtiles(P) * (tc_ktiles(P) >> 1) * 256;  // 8-byte entries
    return pow2 ? (P >> 1) : ((P - 1) >> 1) * odd_row_len(P);
}
// Entries of the axis' table that the bucketization copies into shared memory.  Tables with
// gmem set stay in global memory and are read through the read-only cache: the fragment
// tables of tensor-core axes, and the conjugate-pair matrices of odd axes above P = 9 in
// stages whose one-pass tile fills more than half of shared memory -- there every KB of
// shared memory beyond the tile takes L1 away from the gather's loads in flight (measured:
// 16 KB more made the gather of a 16k-sample tile 16 % slower, 36 KB 56 %), while smaller
// tiles (two-pass stages, two or more CTAs per SM) read the matrices faster from shared
// memory.
__host__ __device__ __forceinline__ int axis_tw_smem(int P, int pow2, int tc, int gmem)
{
    return (tc || gmem) ? 0 : axis_tw_count(P, pow2, 0);
}
// v = hi + lo + e with hi = v cut to TF32 (sign, exponent, 10 mantissa bits) and lo the
// exact remainder cut to TF32 as well, so |e| < 2^-20 |v|
__host__ __device__ __forceinline__ void tf32_split_bits(uint32_t v, uint32_t* hi, uint32_t* lo)
{
    union {
        uint32_t u;
        float f;
    } a, b, r;
    a.u = v;
    b.u = v & 0xffffe000u;
    r.f = a.f - b.f;
    *hi = b.u;
    *lo = r.u & 0xffffe000u;
}
#ifdef __CUDACC__
// d += a b for one 16 x 8 x 8 TF32 tile: a row-major (4 registers), b column-major (2),
// FP32 d
__device__ __forceinline__ void mma_tf32(float* d, uint4 a, uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// d += a b for one 16 x 8 x 16 FP16 tile: a row-major (4 registers of two halves), b
// column-major (2), FP32 d
__device__ __forceinline__ void mma_f16(float* d, uint4 a, uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// (hi, lo) of v0 and v1 as packed half pairs (v0 in the low half): hi = v rounded to FP16,
// lo = the remainder rounded to FP16, so |v - hi - lo| <= 2^-22 |v| while the values stay in
// FP16's normal range
__device__ __forceinline__ void f16_split2(float v0, float v1, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(v0, v1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Word w of the fragment table of a tensor-core odd axis: two halves (columns 2 c' and
// 2 c' + 1 of the m16n8k16 A fragment register c) of the cosine or sine of
// 2 pi (n k mod P) / P (FP64, rounded to FP32), for output row k and the input rows n of
// those slots, zero outside k, n <= (P - 1) / 2; their FP16 high or low parts.
__device__ __forceinline__ uint32_t tc_twiddle_word(int P, int w)
{
    const int KK = tc_ktiles(P) >> 1, pairs = (P - 1) >> 1;
    const int blk = w >> 7, lane = (w >> 2) & 31, c = w & 3;
    const int q = blk & 3, tile = blk >> 2;
    const int mt = tile / KK, kk = tile - mt * KK;
    const int k = mt * 16 + (lane >> 2) + (c & 1) * 8;
    float v[2];
    for (int j = 0; j < 2; ++j) {
        const int n = tc_row(2 * kk + j, (lane & 3) + (c >> 1) * 4);
        v[j] = 0.0f;
        if (k <= pairs && n <= pairs) {
            double sv, cv;
            sincospi(2.0 * (double)((n * k) % P) / (double)P, &sv, &cv);
            v[j] = (float)(q < 2 ? cv : sv);
        }
    }
    uint32_t hi, lo;
    f16_split2(v[0], v[1], hi, lo);
    return (q & 1) ? lo : hi;
}
#endif
__host__ __device__ __forceinline__ int32_t axis_tw_residue(int P, int pow2, int i)
{
    if (pow2) return i;
    const int kp = odd_row_len(P), pairs = (P - 1) >> 1;
    const int n = i / kp + 1, k = i % kp + 1;
    return k > pairs ? 0 : (int32_t)(((int64_t)n * k) % P);
}

// The first round's ML candidate search on the tensor cores (FP32 plans, R <= 16).  For a
// stage's L candidates q and R delays the scores are |c_q|^2 with
//   c_q = sum_r Z_r conj(W[r][q]),  Re c_q = sum_r (Re Z_r cos + Im Z_r sin),
//                                   Im c_q = sum_r (Im Z_r cos - Re Z_r sin),
// (cos, sin) of 2 pi (q tauL_r mod L) / L: one real product A Z of the 16-row m-tile mt of A
// (row i < 8: Re c of candidate 8 mt + i; row 8 + i: its Im c) with the K = 2 RP rows of Z
// (k < RP: Re Z_k, else Im Z_{k - RP}; RP = R rounded up to a multiple of 4, so each of the
// KT = RP / 4 k-tiles of 8 rows holds Z_{t + 4 i} in lane slot t).  A's m16n8k8 TF32
// fragments come pre-split: fragment tile (mt, kt) of a stage is 64 uint4, the high parts
// (lane l at + l) then the low parts (+ 32 + l), each uint4 the lane's (a0, a1, a2, a3) =
// A[g][k], A[g + 8][k], A[g][k + 4], A[g + 8][k + 4] with g = l / 4, k = 8 kt + l % 4.
__host__ __device__ __forceinline__ int ml_tc_rp(int R) { return (R + 3) & ~3; }
__host__ __device__ __forceinline__ int ml_tc_tiles(int L, int R) { return ((L + 7) >> 3) * (ml_tc_rp(R) >> 2); }

// Decode workspace of one signal slot (all arrays sumB entries unless stated).
struct DecodeWs {
    uint8_t* state;      // 0 open, 1 zero-ton, 2 single-ton
    uint32_t* dirty;     // queued for the next round
    int64_t* cand;       // (round << 40) | f of the bin's single-ton, -1 none
    int32_t* list0;      // bins examined in even rounds
    int32_t* list1;      // bins examined in odd rounds
    int32_t* nzl;        // non-zero bins of the current round
    int32_t* cbin;       // single-ton candidates: bin
    int64_t* cf;         //                        frequency
    void* cv;            //                        value (complex of the arithmetic type)
    int64_t* rec_f;      // recovered frequencies
    void* rec_v;         // recovered values
    int32_t* ctr;        // counters, see Ctr
    double* sv;          // one-shot: sumB * a_m singular values, then the vote threshold
    double* sig2;        // noise_auto: the signal's estimated sigma^2 (one per slot)
    int32_t* sub_head;   // peeling: head of the bin's list of pending subtractions, -1 none
    int2* sub_ent;       // peeling: list entries {candidate index, next entry} (D sumB per slot)
};

// the two thresholds of a stage for one signal (Sec. 3.2 subproblem 1), in both types
struct Thr {
    double T0, T1;
    float T0f, T1f;
};

// counter words of a signal slot
enum Ctr : int {
    kCtrRec = 0,        // recovered count
    kCtrResolved = 1,   // bins resolved (zero- or single-ton)
    kCtrIdents = 2,     // bins classified
    kCtrRounds = 3,     // rounds run
    kCtrErr = 4,        // device error (timeout)
    kCtrBarCount = 5,   // group barrier arrivals
    kCtrBarGen = 6,     // group barrier generation
    kCtrDtList = 7,     // one-shot decoder: buckets listed for the FP64 work (in nzl)
    kCtrSub = 8,        // peeling: subtraction-list entries used (all rounds)
    kCtrRoundBase = 9,  // per round r (1-based): [3 r + 0] next-list size, [+1] non-zero
                        // bins, [+2] single-ton candidates
};
constexpr int ctr_words(int max_rounds) { return kCtrRoundBase + 3 * (max_rounds + 2); }

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

__host__ __device__ __forceinline__ int32_t bitrev(int32_t v, int32_t bits)
{
#ifdef __CUDA_ARCH__
    return bits == 0 ? 0 : (int32_t)(__brev((unsigned)v) >> (32 - bits));
#else
    int32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
#endif
}

// bin index j of storage position p in stage s (CRT map)
__host__ __device__ __forceinline__ int32_t pos_to_bin(const StageDesc& s, int32_t p)
{
    int64_t j = 0;
    for (int a = 0; a < s.n_axes; ++a) {
        int32_t k = (p / s.ax[a].S) % s.ax[a].P;
        j += (int64_t)k * s.ax[a].crt;
    }
    return (int32_t)(j % s.B);
}

// storage position of bin j in stage s
__host__ __device__ __forceinline__ int32_t bin_to_pos(const StageDesc& s, int32_t j)
{
    int32_t p = 0;
    for (int a = 0; a < s.n_axes; ++a) p += (j % s.ax[a].P) * s.ax[a].S;
    return p;
}

}  // namespace sfft
