// launch.h -- host-side launchers of the libsfft kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "sfft_internal.cuh"

namespace sfft {

constexpr int kClassifyTile = 2048;  // bins per classify CTA

// Arguments of one bucketization launch (gather + prime-factor DFT passes).
struct BucketArgs {
    PlanDesc pd;
    PassDesc pass[kMaxStages];
    int32_t tile_prefix[kMaxStages + 1];  // cumulative R * n_tiles over stages
    int32_t tiles_per_sig;
    int32_t n_sig;
    const int32_t* nidx;     // per stage (at bin_base): input sample index n of position p
    const void* tw;          // plan twiddles (float2 or double2): (cos, sin)(2 pi t / P)
    const void* const* xs;  // device array of n_sig signal pointers, or nullptr
    const void* x0;          // the signal when xs == nullptr
    void* scratch;           // complex, n_sig * y_per_sig
    void* bins;              // complex, n_sig * y_per_sig
    int32_t x_sys;           // 1: the signal is page-locked host memory read in place
};

struct DecodeArgs {
    PlanDesc pd;
    DecodeWs ws;          // slot 0 pointers; slot s at + s * sumB (ctr: + s * ctr_stride)
    int32_t ctr_stride;
    int32_t G;            // CTAs per signal
    int32_t n_sig;
    int32_t fault;        // 1: one CTA per group leaves before its first barrier (testing)
    long long spin_limit; // polls before a device-side wait gives up
    int32_t wtab_elems;   // largest window of ML phasor tables a classify tile stages
    int32_t wtab_smem;    // 1: classify stages them in shared memory
    int32_t dt_method;    // one-shot Step 2: 1 polynomial roots, 2 enumeration, 3 matrix pencil
    int32_t lanes;        // classify: lanes per bin of the ML search (0 = chosen per tile)
    int32_t ml_tf32;      // classify's tensor-core ML search: 1 = split TF32 (m16n8k8), 0 = split FP16 (m16n8k16)
    const int32_t* pbin;  // position -> bin j, per stage at bin_base
    const int32_t* bpos;  // bin j -> position
    const void* roots;    // the plan's twiddle table: ML phasor tables at st[d].wtab_off
    const uint4* mltc;    // ML tensor-core fragment tables (st[d].mltc_off), or nullptr
    void* bins;           // complex, n_sig * y_per_sig, modified in place
};

struct CompactArgs {
    PlanDesc pd;
    DecodeWs ws;
    int32_t ctr_stride;
    int32_t n_sig;
    int32_t sort_cap;           // pow2 capacity of sortbuf per slot
    int32_t smem_cap;           // pow2 capacity (keys) of the shared-memory sort area
    uint64_t* sortbuf;          // 2 * sort_cap per slot
    int64_t* const* out_idx;    // device array of n_sig pointers, or nullptr
    void* const* out_val;
    int64_t* idx0;              // the outputs when out_idx == nullptr (one signal)
    void* val0;
    int32_t* infos;             // int32[4 * n_sig], when info_rows == nullptr
    int32_t* const* info_rows;  // device array of n_sig pointers to int32[4] rows, or nullptr
};

// precision: 0 = double arithmetic, 1 = float; xdouble: input/output complex128
cudaError_t launch_bucketize(const BucketArgs& a, int precision, int xdouble, int threads,
                             size_t smem, cudaStream_t st);
// persistent one-pass variant with the next tile's gather overlapped (FP32, device x):
// grid CTAs with smem bytes each, tile regions of `region` elements at both ends
cudaError_t launch_bucketize_stream(const BucketArgs& a, int grid, int threads, size_t smem,
                                    int region, cudaStream_t st);
// round 1 of the decoder (classification of every bin) over all signals
cudaError_t launch_classify(const DecodeArgs& a, int precision, cudaStream_t st);
// sigma^2 per signal from the median bin energy (noise_auto plans), before classify
cudaError_t launch_noise_estimate(const DecodeArgs& a, int precision, cudaStream_t st);
// one-shot decoder (three kernels: singular values, vote, solve)
cudaError_t launch_oneshot(const DecodeArgs& a, int precision, cudaStream_t st);
// peeling rounds, G CTAs per signal (cooperative when G > 1)
cudaError_t launch_decode(const DecodeArgs& a, int precision, int threads, bool cooperative,
                          cudaStream_t st);
cudaError_t launch_compact(const CompactArgs& a, int precision, int xdouble, int threads,
                           size_t smem, cudaStream_t st);
// natural-order copy of bins (for sfft_bucketize) and back (for sfft_decode_bins)
cudaError_t launch_bins_to_natural(const PlanDesc& pd, const int32_t* pbin, const void* src,
                                   void* dst, int precision, int to_natural, cudaStream_t st);
cudaError_t launch_twiddles(void* tw, const int32_t* P_of, const int32_t* t_of, int64_t n,
                            int precision, cudaStream_t st);
cudaError_t set_kernel_smem_limits(int max_smem);
int decode_occupancy(int precision, int threads);

}  // namespace sfft
