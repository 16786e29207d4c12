// sfft_plan.h -- the plan object behind sfft_plan_t (internal).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "sfft_internal.cuh"

struct sfft_plan_s {
    sfft::PlanDesc pd;                       // host copy of the device-side description
    sfft::PassDesc pass1[sfft::kMaxStages];  // first bucketization launch, per stage
    sfft::PassDesc pass2[sfft::kMaxStages];  // second launch (two-pass stages only)
    bool need_pass2 = false;
    sfft_opts opts;
    int prec = 1;        // 1 FP32 arithmetic, 0 FP64
    int xdouble = 0;     // 1 complex128 input/output
    size_t esz = 8;      // bytes of one complex of the arithmetic type
    size_t xesz = 8;     // bytes of one complex of the I/O type
    int max_batch = 1;
    int num_sms = 0;
    int max_smem = 0;     // the device's opt-in shared memory per block
    bool stream_ok = false;  // one-pass FP32 plan whose tiles fill more than half of it: the
                             // persistent overlapped bucketization applies
    int decode_occ = 1;
    int threads1 = 256, threads2 = 256;
    size_t smem1 = 0, smem2 = 0;
    // plan tables
    int32_t* d_nidx = nullptr;  // position -> input sample index, per stage
    int32_t* d_pbin = nullptr;  // position -> bin j
    int32_t* d_bpos = nullptr;  // bin j -> position
    void* d_tw = nullptr;       // twiddles of every axis
    void* d_mltc = nullptr;     // the ML search's tensor-core fragment tables (or none)
    // workspace for max_batch signals
    void* d_bins = nullptr;
    void* d_scratch = nullptr;
    void* d_dec = nullptr;
    size_t dec_bytes = 0;
    sfft::DecodeWs ws;
    int32_t ctr_stride = 0;
    size_t ctr_bytes_per_sig = 0;
    uint64_t* d_sortbuf = nullptr;
    int32_t sort_cap = 1, smem_cap = 1;
    // batch pointer tables (signals, outputs, info rows: 4 x max_batch pointers): device
    // copy + two pinned host slots
    void** d_ptrs = nullptr;
    void** h_ptrs[2] = {nullptr, nullptr};
    cudaEvent_t ptr_ev[2] = {nullptr, nullptr};
    int ptr_slot = 0;
    // staging for host-memory inputs/outputs and for sfft_decode_bins
    void* d_x_stage = nullptr;
    void* d_out_stage = nullptr;
    void* d_bins_in = nullptr;
    cudaStream_t aux[2] = {nullptr, nullptr};  // host-buffer batches: copy/compute overlap
    cudaEvent_t aux_ev = nullptr;
    cudaEvent_t aux_join[2] = {nullptr, nullptr};
    void* d_xb_stage = nullptr;   // host-buffer batches: max_batch inputs
    void* d_ob_stage = nullptr;   //                      max_batch outputs + infos
    int32_t wtab_elems = 0;  // largest window of ML phasor tables one classify tile needs
    size_t footprint = 0;  // device bytes owned by the plan
    // phase timing (sfft_plan_set_profiling): CUDA events recorded on the launch stream
    bool prof = false;
    struct PhaseEv {
        cudaEvent_t a, b;
        int phase;
        int launches;
    };
    std::vector<PhaseEv> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[3] = {0, 0, 0};
    int64_t prof_launches[3] = {0, 0, 0};
    int64_t prof_calls[3] = {0, 0, 0};
    // DSFFT plans: one single-stage plan per layer of the binary tree, from the start layer
    // down (layer d of start_layer + i is layers[i]); the parent owns no workspace
    std::vector<sfft_plan_s*> layers;
    int start_layer = 0;
};
