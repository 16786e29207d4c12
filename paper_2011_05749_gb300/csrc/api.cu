// api.cu -- libsfft host library: plans (validation, prime-factor index maps, twiddles,
// thresholds, workspace), execution entry points and error reporting.  The C ABI is
// declared in include/sfft.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "launch.h"
#include "sfft.h"
#include "sfft_internal.cuh"
#include "ml_table.h"
#include "pfa_layout.h"
#include "sfft_plan.h"

using namespace sfft;

namespace sfft {
cudaError_t set_bucketize_smem_limit(int max_smem);
cudaError_t set_compact_smem_limit(int max_smem);
cudaError_t set_classify_smem_limit(int max_smem);

static thread_local char g_last_cuda[256] = "no error";

int cuda_fail(cudaError_t e)
{
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return SFFT_ECUDA;
}

static int cuda_fail_at(cudaError_t e, const char* what, int line)
{
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s (api.cu:%d %s)", cudaGetErrorName(e),
             cudaGetErrorString(e), line, what);
    return SFFT_ECUDA;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail_at(e_, #call, __LINE__); \
    } while (0)

static int64_t gcd64(int64_t a, int64_t b)
{
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct DevInfo {
    int sms = 0, max_smem = 0;
    bool ok = false;
};

static int device_info(DevInfo* out)
{
    static std::mutex mu;
    static DevInfo cache[64];
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return SFFT_EINVAL;
    if (!cache[dev].ok) {
        DevInfo di;
        CK(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&di.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        CK(set_bucketize_smem_limit(di.max_smem));
        CK(set_compact_smem_limit(di.max_smem));
        CK(set_classify_smem_limit(di.max_smem - 16 * 1024));
        di.ok = true;
        cache[dev] = di;
    }
    *out = cache[dev];
    return SFFT_OK;
}

}  // namespace sfft

// ---------------------------------------------------------------------------------------

extern "C" void sfft_opts_default(sfft_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->dtype = SFFT_C64;
    o->precision = SFFT_PREC_FP32;
    o->locate = SFFT_LOCATE_ML;
    o->max_rounds = 64;
    o->max_batch = 1;
    o->noise_var = 0.0;
    o->a_min = 1.0;
    o->eta = 0.0;
    o->c0 = 4.0;
    o->c1 = 2.0;
    o->decoder = SFFT_DECODER_PEEL;
    o->oneshot_am = 3;
    o->kay_m = 2;
}

static void free_plan_memory(sfft_plan_s* p)
{
    void* dev[] = {p->d_nidx, p->d_pbin, p->d_bpos, p->d_tw, p->d_mltc, p->d_bins, p->d_scratch,
                   p->d_dec, p->d_ptrs, p->d_sortbuf, p->d_x_stage, p->d_out_stage,
                   p->d_bins_in, p->d_xb_stage, p->d_ob_stage};
    for (void* q : dev)
        if (q) cudaFree(q);
    for (int i = 0; i < 2; ++i) {
        if (p->h_ptrs[i]) cudaFreeHost(p->h_ptrs[i]);
        if (p->ptr_ev[i]) cudaEventDestroy(p->ptr_ev[i]);
    }
    for (auto& e : p->prof_pending) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : p->prof_pool) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
        if (p->aux[i]) cudaStreamDestroy(p->aux[i]);
        if (p->aux_join[i]) cudaEventDestroy(p->aux_join[i]);
    }
    if (p->aux_ev) cudaEventDestroy(p->aux_ev);
}

extern "C" int sfft_plan_create(sfft_plan_t* out, int64_t N, int32_t K, int32_t n_stages,
                                const int64_t* f, int32_t n_delays, const int64_t* delays,
                                const sfft_opts* opts_in)
{
    if (!out || !f || !delays) return SFFT_EINVAL;
    *out = nullptr;
    sfft_opts o;
    sfft_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (N < 1 || N >= (1ll << 30) || K < 1 || n_stages < 1 || n_stages > kMaxStages ||
        n_delays < 1 || n_delays > kMaxDelays)
        return SFFT_EINVAL;
    if ((o.dtype != SFFT_C64 && o.dtype != SFFT_C128) ||
        (o.precision != SFFT_PREC_FP32 && o.precision != SFFT_PREC_FP64) ||
        (o.locate != SFFT_LOCATE_ARG && o.locate != SFFT_LOCATE_ML && o.locate != SFFT_LOCATE_KAY) ||
        o.max_rounds < 1 ||
        o.max_rounds > 4096 || o.max_batch < 1 || o.max_tile < 0 || o.noise_var < 0 || o.a_min < 0 ||
        o.eta < 0 || o.c0 < 0 || o.c1 < 0)
        return SFFT_EINVAL;
    for (int d = 0; d < n_stages; ++d) {
        if (f[d] < 1 || N % f[d] != 0) return SFFT_EINVAL;
        for (int e = 0; e < d; ++e)
            if (gcd64(f[d], f[e]) != 1) return SFFT_EINVAL;
        for (int r = 0; r < n_delays; ++r) {
            const int64_t t = delays[(int64_t)d * n_delays + r];
            if (t < 0 || t >= N) return SFFT_EINVAL;
            for (int q = 0; q < r; ++q)
                if (delays[(int64_t)d * n_delays + q] == t) return SFFT_EINVAL;
        }
    }
    if (o.decoder == SFFT_DECODER_DSFFT) {
        // binary tree search (Sec. 3.3): N = 2^n, start factor f[0] = N / 2^p, delays {0, 1};
        // one single-stage ARG plan per layer d = p .. n
        if (n_stages != 1 || (N & (N - 1)) != 0 || (f[0] & (f[0] - 1)) != 0 || n_delays != 2 ||
            delays[0] != 0 || delays[1] != 1 || o.noise_auto != 0)
            return SFFT_EINVAL;
        sfft_plan_s* p = new (std::nothrow) sfft_plan_s();
        if (!p) return SFFT_ENOMEM;
        p->opts = o;
        p->max_batch = o.max_batch;
        int n = 0;
        while ((1ll << n) < N) ++n;
        int lp = 0;
        while ((1ll << lp) < f[0]) ++lp;
        p->start_layer = n - lp;
        sfft_opts ol = o;
        ol.decoder = SFFT_DECODER_PEEL;
        ol.locate = SFFT_LOCATE_ARG;
        // layers down to the deepest one the bucketization supports (a power-of-two B is one
        // axis, so B is bounded by what one CTA's shared memory holds)
        for (int64_t L = f[0]; L >= 1; L >>= 1) {
            sfft_plan_t lay = nullptr;
            const int rc = sfft_plan_create(&lay, N, K, 1, &L, 2, delays, &ol);
            if (rc == SFFT_EINVAL && !p->layers.empty()) break;
            if (rc) {
                for (sfft_plan_s* q : p->layers) sfft_plan_destroy(q);
                delete p;
                return rc;
            }
            p->layers.push_back(lay);
            p->footprint += lay->footprint;
        }
        p->pd = p->layers.back()->pd;  // the last layer's description (sizes, K)
        p->prec = p->layers.back()->prec;
        p->xdouble = p->layers.back()->xdouble;
        p->esz = p->layers.back()->esz;
        p->xesz = p->layers.back()->xesz;
        *out = p;
        return SFFT_OK;
    }
    if (o.decoder != SFFT_DECODER_PEEL && o.decoder != SFFT_DECODER_ONESHOT) return SFFT_EINVAL;
    if (o.noise_auto != 0 && (o.noise_auto != 1 || o.decoder != SFFT_DECODER_PEEL)) return SFFT_EINVAL;
    if (o.locate == SFFT_LOCATE_KAY && o.decoder == SFFT_DECODER_PEEL) {
        // structured delays: slot c m + t = r_c + t 2^c (mod N); 2^C >= L_d tells the L_d
        // candidates apart
        const int m = o.kay_m;
        if (m < 2 || n_delays % m != 0 || n_delays / m > 30) return SFFT_EINVAL;
        const int C = n_delays / m;
        for (int d = 0; d < n_stages; ++d) {
            if ((1ll << C) < f[d]) return SFFT_EINVAL;
            for (int c = 0; c < C; ++c)
                for (int t = 1; t < m; ++t) {
                    const int64_t base = delays[(int64_t)d * n_delays + c * m];
                    if (delays[(int64_t)d * n_delays + c * m + t] != (base + ((int64_t)t << c)) % N)
                        return SFFT_EINVAL;
                }
        }
    }
    if (o.decoder == SFFT_DECODER_ONESHOT) {
        // one stage; slots 0 .. 3 a_m - 1 hold -a_m .. 2 a_m - 1 (mod N), then at least 2 a_m
        // random delays (Sec. 4.1, Stage 1); the output holds at most one value per bucket
        const int am = o.oneshot_am;
        if (n_stages != 1 || am < 1 || am > 3 || n_delays < 5 * am || K > N / f[0]) return SFFT_EINVAL;
        if (o.oneshot_method < 0 || o.oneshot_method > 3) return SFFT_EINVAL;
        for (int r = 0; r < 3 * am; ++r)
            if (delays[r] != ((int64_t)r - am + N) % N) return SFFT_EINVAL;
    }
    if (o.fault_inject == 2) return SFFT_ENOMEM;  // injected allocation failure (testing)
    if (o.wait_limit_log2 < 0 || o.fault_inject < 0 || o.fault_inject > 2 || o.decode_ctas < 0)
        return SFFT_EINVAL;
    if (o.classify_lanes < 0 || o.classify_lanes > 32 || (o.classify_lanes & (o.classify_lanes - 1)))
        return SFFT_EINVAL;
    if (o.arg_mode < 0 || o.arg_mode > 3) return SFFT_EINVAL;
    if (o.ml_tc_tf32 != 0 && o.ml_tc_tf32 != 1) return SFFT_EINVAL;
    DevInfo di;
    int rc = device_info(&di);
    if (rc) return rc;

    sfft_plan_s* p = new (std::nothrow) sfft_plan_s();
    if (!p) return SFFT_ENOMEM;
    p->opts = o;
    p->prec = o.precision == SFFT_PREC_FP32 ? 1 : 0;
    p->xdouble = o.dtype == SFFT_C128 ? 1 : 0;
    p->esz = p->prec ? 8 : 16;
    p->xesz = p->xdouble ? 16 : 8;
    p->max_batch = o.max_batch;
    p->num_sms = di.sms;
    p->max_smem = di.max_smem;
    const double eta = o.eta > 0 ? o.eta : (p->prec ? 3e-3 : 1e-6);

    PlanDesc& pd = p->pd;
    memset(&pd, 0, sizeof(pd));
    pd.N = (int32_t)N;
    pd.D = n_stages;
    pd.R = n_delays;
    pd.locate = o.locate;
    pd.max_rounds = o.max_rounds;
    pd.K = K;
    pd.invN = 1.0 / (double)N;
    pd.mu = ~0ull / (uint64_t)N;
    pd.mode = o.decoder == SFFT_DECODER_ONESHOT ? 1 : 0;
    pd.kay_m = o.locate == SFFT_LOCATE_KAY ? o.kay_m : 0;
    pd.noise_auto = o.noise_auto;
    pd.peel_atomic = o.peel_atomic ? 1 : 0;
    pd.arg_mode = o.arg_mode;
    {
        // median of Gamma(R, 1): CDF(x) = 1 - e^{-x} sum_{k<R} x^k / k! = 1/2, by Newton's
        // method from x = R - 1/3 (the density x^{R-1} e^{-x} / (R-1)! is the derivative)
        double x = n_delays - 1.0 / 3.0;
        for (int it = 0; it < 50; ++it) {
            double term = 1.0, sum = 1.0;
            for (int k = 1; k < n_delays; ++k) {
                term *= x / k;
                sum += term;
            }
            const double cdf = 1.0 - exp(-x) * sum;
            const double pdf = exp(-x) * term;  // x^{R-1} e^{-x} / (R-1)!
            const double step = (cdf - 0.5) / pdf;
            x -= step;
            if (fabs(step) < 1e-15 * x) break;
        }
        pd.gmed = x;
    }
    if (pd.mode == 1) {
        // the vote's floor: a_m times the per-delay zero-ton level of a bucket in moment
        // units, sqrt(c0 B sigma^2 + (eta B a_min)^2) / B; the pursuit's residual tolerance
        // P (c1 sigma^2 / B + (eta a_min)^2)
        const double B = (double)(N / f[0]);
        const int am = o.oneshot_am, P = n_delays - 3 * am;
        pd.am = am;
        pd.sv_floor = am * sqrt(o.c0 * B * o.noise_var + (eta * B * o.a_min) * (eta * B * o.a_min)) / B;
        pd.sp_tol2 = P * (o.c1 * o.noise_var / B + (eta * o.a_min) * (eta * o.a_min));
    }

    std::vector<int32_t> h_nidx, h_pbin, h_bpos, tw_P, tw_t;
    int64_t bin_base = 0;
    PassPlan l1, l2;
    p->need_pass2 = false;
    const int64_t tile_target = p->prec ? 4096 : 2048;
    int32_t tw_cursor = 0;
    for (int d = 0; d < n_stages; ++d) {
        StageDesc& s = pd.st[d];
        const int64_t L = f[d], B = N / L;
        s.B = (int32_t)B;
        s.L = (int32_t)L;
        if (!pfa_layout_stage(&s, p->esz, di.max_smem, tile_target, &p->pass1[d], &p->pass2[d],
                              &l1, &l2, &tw_cursor, &p->need_pass2, o.max_tile,
                              o.dft_fma_only == 0)) {
            free_plan_memory(p);
            delete p;
            return SFFT_EINVAL;
        }
        for (int r = 0; r < n_delays; ++r) {
            s.tau[r] = (int32_t)delays[(int64_t)d * n_delays + r];
            s.tauL[r] = (int32_t)(delays[(int64_t)d * n_delays + r] % L);
            s.step32[r] = (int32_t)((32 * (int64_t)s.tauL[r]) % L);
        }
        s.invL = 1.0f / (float)L;
        s.r0 = s.r1 = -1;
        for (int r = 0; r < n_delays; ++r) {
            if (s.tau[r] == 0 && s.r0 < 0) s.r0 = r;
            if (s.tau[r] == 1 && s.r1 < 0) s.r1 = r;
        }
        if (o.locate == SFFT_LOCATE_ARG && (s.r0 < 0 || s.r1 < 0)) {
            free_plan_memory(p);
            delete p;
            return SFFT_EINVAL;
        }
        s.bin_base = (int32_t)bin_base;
        s.y_off = (int32_t)(bin_base * n_delays);
        // thresholds: T0 = R (c0 B sigma^2 + (eta B a_min)^2), T1 with c1
        const double sig_y = (double)B * o.noise_var;
        const double fl = eta * (double)B * o.a_min;
        s.T0 = (double)n_delays * (o.c0 * sig_y + fl * fl);
        s.T1 = (double)n_delays * (o.c1 * sig_y + fl * fl);
        s.T0f = (float)s.T0;
        s.T1f = (float)s.T1;
        s.T0a = (double)n_delays * o.c0 * (double)B;
        s.T1a = (double)n_delays * o.c1 * (double)B;
        s.Tb = (double)n_delays * fl * fl;

        // index maps
        const size_t base = h_nidx.size();
        h_nidx.resize(base + B);
        h_pbin.resize(base + B);
        h_bpos.resize(base + B);
        for (int64_t pos = 0; pos < B; ++pos) {
            int64_t n = 0, j = 0;
            for (int a = 0; a < s.n_axes; ++a) {
                const AxisDesc& A = s.ax[a];
                const int32_t c = (int32_t)((pos / A.S) % A.P);
                const int32_t na = A.pow2 ? bitrev(c, A.log2P) : c;
                n += (int64_t)na * A.rur;
                j += (int64_t)c * A.crt;
            }
            h_nidx[base + pos] = (int32_t)(n % B);
            h_pbin[base + pos] = (int32_t)(j % B);
        }
        for (int64_t pos = 0; pos < B; ++pos) h_bpos[base + h_pbin[base + pos]] = (int32_t)pos;
        for (int64_t jj = 0; jj < B; ++jj) {
            int64_t pp = 0;
            for (int a = 0; a < s.n_axes; ++a) pp += (jj % s.ax[a].P) * s.ax[a].S;
            if (pp != h_bpos[base + jj]) {  // CRT maps must be inverse permutations
                free_plan_memory(p);
                delete p;
                return SFFT_EINVAL;
            }
        }
        bin_base += B;
    }
    // twiddle table: every axis (layout of axis_tw_residue, or the fragment table of a
    // tensor-core axis), then the L roots of each stage
    tw_P.assign((size_t)tw_cursor, 1);
    tw_t.assign((size_t)tw_cursor, 0);
    for (int d = 0; d < n_stages; ++d)
        for (int a = 0; a < pd.st[d].n_axes; ++a) {
            const AxisDesc& A = pd.st[d].ax[a];
            const bool tc = A.tc != 0;
            const int cnt = axis_tw_count(A.P, A.pow2, A.tc);
            for (int i = 0; i < cnt; ++i) {
                // tensor-core axes: -P and the entry's index (fragment table)
                tw_P[(size_t)A.tw_off + i] = tc ? -A.P : A.P;
                tw_t[(size_t)A.tw_off + i] = tc ? i : axis_tw_residue(A.P, A.pow2, i);
            }
        }
    pd.root_total = 0;
    for (int d = 0; d < n_stages; ++d) {
        pd.st[d].root_off = (int32_t)tw_P.size();
        for (int t = 0; t < pd.st[d].L; ++t) {
            tw_P.push_back(pd.st[d].L);
            tw_t.push_back(t);
        }
        pd.root_total += pd.st[d].L;
    }
    // two-level table of the N-th roots of unity for the delay phasors a_r(f):
    // lo[l] = e^{2 pi i l / N} (l < 2^S), hi[h] = e^{2 pi i h 2^S / N}
    pd.ph_shift = 11;
    pd.ph_lo_off = (int32_t)tw_P.size();
    for (int64_t l = 0; l < (1 << pd.ph_shift); ++l) {
        tw_P.push_back((int32_t)N);
        tw_t.push_back((int32_t)(l % N));
    }
    pd.ph_hi_off = (int32_t)tw_P.size();
    for (int64_t h = 0; h <= (N - 1) >> pd.ph_shift; ++h) {
        tw_P.push_back((int32_t)N);
        tw_t.push_back((int32_t)((h << pd.ph_shift) % N));
    }
    // the first round's ML search on the tensor cores (FP32 peeling plans, R <= 16): per
    // stage the split fragments of A, from the same phasors in FP64 rounded to FP32, in the
    // split-FP16 layout (ml_tc16_word) or, with ml_tc_tf32, the split-TF32 one (ml_tc_word);
    // fragment tiles of 256 words either way
    std::vector<uint32_t> h_mltc;
    const bool ml_tc = p->prec == 1 && o.locate == SFFT_LOCATE_ML && pd.mode == 0 && n_delays <= 16;
    for (int d = 0; d < n_stages; ++d) {
        StageDesc& s = pd.st[d];
        s.mltc_off = -1;
        if (!ml_tc) continue;
        s.mltc_off = (int32_t)(h_mltc.size() / 256);
        const int L = s.L, MT = (L + 7) / 8;
        const int KT = o.ml_tc_tf32 ? ml_tc_rp(n_delays) / 4 : ml_tc16_ktiles(n_delays);
        for (int mt = 0; mt < MT; ++mt)
            for (int kt = 0; kt < KT; ++kt)
                for (int h = 0; h < 2; ++h)
                    for (int l = 0; l < 32; ++l)
                        for (int e = 0; e < 4; ++e)
                            h_mltc.push_back(o.ml_tc_tf32 ? ml_tc_word(L, n_delays, s.tauL, mt, kt, h, l, e)
                                                          : ml_tc16_word(L, n_delays, s.tauL, mt, kt, h, l, e));
    }
    // ML candidate phasors per stage: W[r][q] = e^{2 pi i (q tauL_r mod L) / L}, a row of L
    // candidates per delay
    for (int d = 0; d < n_stages; ++d) {
        pd.st[d].wtab_off = (int32_t)tw_P.size();
        const int64_t L = pd.st[d].L;
        for (int r = 0; r < n_delays; ++r)
            for (int64_t q = 0; q < L; ++q) {
                tw_P.push_back((int32_t)L);
                tw_t.push_back((int32_t)((q * pd.st[d].tauL[r]) % L));
            }
    }
    pd.sumB = (int32_t)bin_base;
    // largest window of phasor tables one classify tile needs: its stages' tables
    p->wtab_elems = 0;
    for (int64_t b0 = 0; b0 < pd.sumB; b0 += kClassifyTile) {
        const int64_t b1 = std::min<int64_t>(pd.sumB, b0 + kClassifyTile) - 1;
        int d0 = 0, d1 = 0;
        while (d0 + 1 < n_stages && b0 >= pd.st[d0 + 1].bin_base) ++d0;
        while (d1 + 1 < n_stages && b1 >= pd.st[d1 + 1].bin_base) ++d1;
        const int32_t n = pd.st[d1].wtab_off + n_delays * pd.st[d1].L - pd.st[d0].wtab_off;
        p->wtab_elems = std::max(p->wtab_elems, n);
    }
    pd.y_per_sig = (int64_t)bin_base * n_delays;
    p->smem1 = l1.smem;
    p->smem2 = l2.smem;
    p->threads1 = pfa_threads(l1.tile, p->esz);
    p->threads2 = pfa_threads(l2.tile, p->esz);
    p->stream_ok = o.overlap_gather != 0 && !p->need_pass2 && p->prec == 1 && !p->xdouble &&
                   2 * p->smem1 > (size_t)di.max_smem;

    // device memory
    const size_t nb = (size_t)pd.sumB, mb = (size_t)p->max_batch;
    const size_t ybytes = (size_t)pd.y_per_sig * p->esz * mb;
    p->ctr_stride = (int32_t)align_up((size_t)ctr_words(pd.max_rounds), 64);
    p->sort_cap = 1;
    while ((size_t)p->sort_cap < nb) p->sort_cap <<= 1;
    {
        // shared-memory keys of the compaction sort: a power of two within the device limit,
        // and no more than both key arrays of 2 K recovered coefficients need, so that two
        // 1024-thread CTAs share an SM (larger counts sort in the slot's global buffer)
        int cap = 1;
        while ((size_t)cap * 2 * sizeof(uint64_t) <= (size_t)di.max_smem - 1024) cap <<= 1;
        int want = 1;
        while (want < 2 * K) want <<= 1;
        p->smem_cap = std::min(std::min(2 * p->sort_cap, cap), std::max(1024, 2 * want));
    }
    // decode workspace, one block carved into arrays
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o2 = off;
        off = align_up(off + bytes, 256);
        return o2;
    };
    const size_t o_state = carve(nb * mb);
    const size_t o_dirty = carve(4 * nb * mb);
    const size_t o_cand = carve(8 * nb * mb);
    const size_t o_l0 = carve(4 * nb * mb);
    const size_t o_l1 = carve(4 * nb * mb);
    const size_t o_nzl = carve(4 * nb * mb);
    const size_t o_cbin = carve(4 * nb * mb);
    const size_t o_cf = carve(8 * nb * mb);
    const size_t o_cv = carve(p->esz * nb * mb);
    const size_t o_rf = carve(8 * nb * mb);
    const size_t o_rv = carve(p->esz * nb * mb);
    const size_t o_ctr = carve(4 * (size_t)p->ctr_stride * mb);
    const size_t o_sv = pd.mode == 1 ? carve(8 * (nb * pd.am + 1) * mb) : 0;
    const size_t o_s2 = pd.noise_auto ? carve(8 * mb) : 0;
    // peeling's per-bin subtraction lists: heads, and D entries per bin (each bin becomes a
    // candidate at most once, and an accepted candidate queues at most one entry per stage)
    const bool lists = pd.mode == 0;
    const size_t o_sh = lists ? carve(4 * nb * mb) : 0;
    const size_t o_se = lists ? carve(8 * (size_t)n_stages * nb * mb) : 0;
    p->dec_bytes = off;
    p->ctr_bytes_per_sig = 4 * (size_t)p->ctr_stride;

    cudaError_t e = cudaSuccess;
    auto dmalloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMalloc(ptr, bytes);
    };
    dmalloc((void**)&p->d_nidx, 4 * h_nidx.size());
    dmalloc((void**)&p->d_pbin, 4 * h_pbin.size());
    dmalloc((void**)&p->d_bpos, 4 * h_bpos.size());
    dmalloc(&p->d_tw, p->esz * tw_P.size());
    dmalloc((void**)&p->d_mltc, 4 * h_mltc.size());
    dmalloc(&p->d_bins, ybytes);
    if (p->need_pass2) dmalloc(&p->d_scratch, ybytes);
    dmalloc(&p->d_dec, p->dec_bytes);
    dmalloc((void**)&p->d_ptrs, 4 * sizeof(void*) * mb);
    dmalloc((void**)&p->d_sortbuf, 2 * sizeof(uint64_t) * (size_t)p->sort_cap * mb);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaHostAlloc((void**)&p->h_ptrs[i], 4 * sizeof(void*) * mb, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ptr_ev[i], cudaEventDisableTiming);
    }
    int32_t* d_twP = nullptr;
    int32_t* d_twt = nullptr;
    dmalloc((void**)&d_twP, 4 * tw_P.size());
    dmalloc((void**)&d_twt, 4 * tw_t.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_nidx, h_nidx.data(), 4 * h_nidx.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_pbin, h_pbin.data(), 4 * h_pbin.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_bpos, h_bpos.data(), 4 * h_bpos.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h_mltc.empty())
        e = cudaMemcpy(p->d_mltc, h_mltc.data(), 4 * h_mltc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_twP, tw_P.data(), 4 * tw_P.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_twt, tw_t.data(), 4 * tw_t.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_twiddles(p->d_tw, d_twP, d_twt, (int64_t)tw_P.size(), p->prec, 0);
    if (e == cudaSuccess) e = cudaMemset(p->d_dec, 0, p->dec_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (d_twP) cudaFree(d_twP);
    if (d_twt) cudaFree(d_twt);
    if (e != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? SFFT_ENOMEM : cuda_fail(e);
        free_plan_memory(p);
        delete p;
        return code;
    }
    unsigned char* base = (unsigned char*)p->d_dec;
    DecodeWs& w = p->ws;
    w.state = (uint8_t*)(base + o_state);
    w.dirty = (uint32_t*)(base + o_dirty);
    w.cand = (int64_t*)(base + o_cand);
    w.list0 = (int32_t*)(base + o_l0);
    w.list1 = (int32_t*)(base + o_l1);
    w.nzl = (int32_t*)(base + o_nzl);
    w.cbin = (int32_t*)(base + o_cbin);
    w.cf = (int64_t*)(base + o_cf);
    w.cv = base + o_cv;
    w.rec_f = (int64_t*)(base + o_rf);
    w.rec_v = base + o_rv;
    w.ctr = (int32_t*)(base + o_ctr);
    w.sv = pd.mode == 1 ? (double*)(base + o_sv) : nullptr;
    w.sig2 = pd.noise_auto ? (double*)(base + o_s2) : nullptr;
    w.sub_head = lists ? (int32_t*)(base + o_sh) : nullptr;
    w.sub_ent = lists ? (int2*)(base + o_se) : nullptr;
    p->footprint = 4 * 3 * h_nidx.size() + p->esz * tw_P.size() + 4 * h_mltc.size() +
                   ybytes * (p->need_pass2 ? 2 : 1) +
                   p->dec_bytes + 2 * sizeof(uint64_t) * (size_t)p->sort_cap * mb;
    p->decode_occ = decode_occupancy(p->prec, 512);
    *out = p;
    return SFFT_OK;
}

extern "C" void sfft_plan_destroy(sfft_plan_t p)
{
    if (!p) return;
    for (sfft_plan_s* q : p->layers) sfft_plan_destroy(q);
    p->layers.clear();
    cudaDeviceSynchronize();
    free_plan_memory(p);
    delete p;
}

extern "C" int64_t sfft_plan_num_bins(sfft_plan_t p) { return p ? p->pd.sumB : -1; }

extern "C" int sfft_plan_noise_var(sfft_plan_t p, int32_t slot, double* out)
{
    if (!p || !out || !p->pd.noise_auto || slot < 0 || slot >= p->max_batch || !p->ws.sig2)
        return SFFT_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, p->ws.sig2 + slot, sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SFFT_OK : sfft::cuda_fail(e);
}

namespace sfft {

static cudaEvent_t prof_event(sfft_plan_s* p)
{
    if (!p->prof_pool.empty()) {
        cudaEvent_t e = p->prof_pool.back();
        p->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// bracket one phase (0 bucketize, 1 decode, 2 compact) with events on the launch stream
struct PhaseScope {
    sfft_plan_s* p;
    cudaStream_t st;
    int phase, launches;
    cudaEvent_t a = nullptr;
    PhaseScope(sfft_plan_s* p_, cudaStream_t st_, int phase_, int launches_)
        : p(p_), st(st_), phase(phase_), launches(launches_)
    {
        if (p->prof) {
            a = prof_event(p);
            cudaEventRecord(a, st);
        }
    }
    ~PhaseScope()
    {
        if (p->prof && a) {
            cudaEvent_t b = prof_event(p);
            cudaEventRecord(b, st);
            p->prof_pending.push_back({a, b, phase, launches});
        }
    }
};

// Workspace of slots [slot0, slot0 + n): decode arrays, counters
static DecodeWs ws_at(const sfft_plan_s* p, int slot0)
{
    DecodeWs w = p->ws;
    const size_t so = (size_t)slot0 * p->pd.sumB;
    w.state += so;
    w.dirty += so;
    w.cand += so;
    w.list0 += so;
    w.list1 += so;
    w.nzl += so;
    w.cbin += so;
    w.cf += so;
    w.cv = (unsigned char*)w.cv + so * p->esz;
    w.rec_f += so;
    w.rec_v = (unsigned char*)w.rec_v + so * p->esz;
    w.ctr += (size_t)slot0 * p->ctr_stride;
    if (w.sv) w.sv += (size_t)slot0 * ((size_t)p->pd.sumB * p->pd.am + 1);
    if (w.sig2) w.sig2 += slot0;
    if (w.sub_head) {
        w.sub_head += so;
        w.sub_ent += so * p->pd.D;
    }
    return w;
}

// One bucketization pass of plan p (pass 0 or 1) with the arguments a: the persistent
// overlapped kernel where it applies (device signals), else one CTA per tile.
static cudaError_t bucketize_pass(const sfft_plan_s* p, const BucketArgs& a, int pass,
                                  cudaStream_t st)
{
    if (pass == 0 && p->stream_ok && !a.x_sys)
        return launch_bucketize_stream(a, p->num_sms, 512, ((size_t)p->max_smem - 1024) & ~(size_t)15,
                                       (int)(p->smem1 / 8), st);
    return launch_bucketize(a, p->prec, p->xdouble, pass == 0 ? p->threads1 : p->threads2,
                            pass == 0 ? p->smem1 : p->smem2, st);
}

// Enqueue the whole path for n signals of one plan in workspace slots [slot0, slot0 + n)
// (slot0 + n <= max_batch).  For n > 1 the signal and output pointers come from device
// tables d_xs / d_idx / d_val; for n == 1 from x0 / idx0 / val0.  Info rows: signal i's at
// d_rows[i] when d_rows is given, else at infos + 4 i.  The decode counters of the slots
// are zero on entry (plan creation zeroes them, every compaction re-zeroes them after
// reading).
int run_chunk(sfft_plan_s* p, int n, const void* x0, const void* const* d_xs,
              int64_t* idx0, void* val0, int64_t* const* d_idx, void* const* d_val,
              int32_t* infos, const void* bins_in, cudaStream_t st, int slot0 = 0,
              bool x_sys = false, int32_t* const* d_rows = nullptr)
{
    PlanDesc& pd = p->pd;
    void* bins = (unsigned char*)p->d_bins + (size_t)slot0 * pd.y_per_sig * p->esz;
    void* scratch = p->d_scratch ? (unsigned char*)p->d_scratch + (size_t)slot0 * pd.y_per_sig * p->esz
                                 : nullptr;
    const DecodeWs ws = ws_at(p, slot0);
    if (bins_in) {
        // caller-supplied natural-order bins (sfft_decode_bins): permute to storage order
        CK(launch_bins_to_natural(pd, p->d_pbin, bins_in, bins, p->prec, 0, st));
    } else {
        PhaseScope ps(p, st, 0, p->need_pass2 ? 2 : 1);
        BucketArgs a;
        memset(&a, 0, sizeof(a));
        a.pd = pd;
        a.n_sig = n;
        a.nidx = p->d_nidx;
        a.tw = p->d_tw;
        a.xs = d_xs;
        a.x0 = x0;
        a.scratch = scratch;
        a.bins = bins;
        a.x_sys = x_sys ? 1 : 0;
        for (int pass = 0; pass < (p->need_pass2 ? 2 : 1); ++pass) {
            const PassDesc* src = pass == 0 ? p->pass1 : p->pass2;
            a.tile_prefix[0] = 0;
            for (int d = 0; d < kMaxStages; ++d) {
                a.pass[d] = d < pd.D ? src[d] : PassDesc{};
                a.tile_prefix[d + 1] = a.tile_prefix[d] + (d < pd.D ? src[d].n_tiles * pd.R : 0);
            }
            a.tiles_per_sig = a.tile_prefix[kMaxStages];
            CK(bucketize_pass(p, a, pass, st));
        }
    }
    DecodeArgs da;
    memset(&da, 0, sizeof(da));
    da.pd = pd;
    da.ws = ws;
    da.ctr_stride = p->ctr_stride;
    da.n_sig = n;
    da.pbin = p->d_pbin;
    da.bpos = p->d_bpos;
    da.bins = bins;
    da.roots = p->d_tw;
    da.mltc = reinterpret_cast<const uint4*>(p->d_mltc);
    da.wtab_elems = p->wtab_elems;
    // a tile's phasor tables go to shared memory up to 160 KB (up to 96 KB two classify
    // CTAs still fit an SM)
    da.wtab_smem = (size_t)p->wtab_elems * p->esz <= 160 * 1024 ? 1 : 0;
    da.dt_method = p->opts.oneshot_method == 0 ? 2 : p->opts.oneshot_method;
    da.lanes = p->opts.classify_lanes;
    da.ml_tf32 = p->opts.ml_tc_tf32;
    const int threads = 512;
    const int total = p->num_sms * p->decode_occ;
    // later rounds touch O(K) bins: about one CTA per 256 expected single-tons
    int G = 1;
    if (n < total) {
        G = (int)std::min<int64_t>(total / n, ((int64_t)pd.K + 255) / 256);
        if (p->opts.decode_ctas > 0) G = (int)std::min<int64_t>(total / n, p->opts.decode_ctas);
        G = std::max(G, 1);
    }
    da.G = G;
    da.fault = p->opts.fault_inject == 1 ? 1 : 0;
    da.spin_limit = 1ll << (p->opts.wait_limit_log2 > 0 ? std::min(p->opts.wait_limit_log2, 40) : 22);
    if (pd.mode == 1) {
        PhaseScope ps(p, st, 1, 3);
        CK(launch_oneshot(da, p->prec, st));
    } else {
        PhaseScope ps(p, st, 1, pd.noise_auto ? 4 : 2);
        if (pd.noise_auto) CK(launch_noise_estimate(da, p->prec, st));
        CK(launch_classify(da, p->prec, st));
        CK(launch_decode(da, p->prec, threads, G > 1, st));
    }

    CompactArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.pd = pd;
    ca.ws = ws;
    ca.ctr_stride = p->ctr_stride;
    ca.n_sig = n;
    ca.sort_cap = p->sort_cap;
    ca.smem_cap = p->smem_cap;
    ca.sortbuf = p->d_sortbuf + (size_t)slot0 * 2 * p->sort_cap;
    ca.out_idx = d_idx;
    ca.out_val = d_val;
    ca.infos = infos;
    ca.info_rows = d_rows;
    ca.idx0 = idx0;
    ca.val0 = val0;
    {
        PhaseScope ps(p, st, 2, 1);
        CK(launch_compact(ca, p->prec, p->xdouble, 1024, sizeof(uint64_t) * (size_t)p->smem_cap, st));
    }
    return SFFT_OK;
}

static bool is_host_ptr(const void* ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace sfft

namespace sfft {
// DSFFT (Sec. 3.3): execute the layer plans from the start layer down until a layer's bins
// are all resolved (every efficient node single-frequency) or the last layer; the outputs
// are that layer's.  Reads each layer's status back to the host.
static int dsfft_execute(sfft_plan_s* p, const void* x, int64_t* out_idx, void* out_val,
                         int32_t* out_info, cudaStream_t st)
{
    const bool hf = is_host_ptr(out_info);
    int32_t info[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < p->layers.size(); ++i) {
        const int rc = sfft_execute(p->layers[i], x, out_idx, out_val, out_info, st);
        if (rc) return rc;
        if (hf) {
            memcpy(info, out_info, sizeof(info));
        } else {
            CK(cudaMemcpyAsync(info, out_info, sizeof(info), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        if (info[1] == SFFT_OK || info[1] == SFFT_ETIMEDOUT || i + 1 == p->layers.size()) {
            const int32_t d = p->start_layer + (int32_t)i;
            if (hf) {
                out_info[2] = d;
            } else {
                CK(cudaMemcpyAsync(out_info + 2, &d, sizeof(d), cudaMemcpyHostToDevice, st));
                CK(cudaStreamSynchronize(st));
            }
            return SFFT_OK;
        }
    }
    return SFFT_OK;
}
}  // namespace sfft

extern "C" int sfft_execute(sfft_plan_t p, const void* x, int64_t* out_idx, void* out_val,
                            int32_t* out_info, void* stream)
{
    if (!p || !x || !out_idx || !out_val || !out_info) return SFFT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (!p->layers.empty()) return dsfft_execute(p, x, out_idx, out_val, out_info, st);
    const bool hx = is_host_ptr(x), hi = is_host_ptr(out_idx), hv = is_host_ptr(out_val),
               hf = is_host_ptr(out_info);
    if (!(hx || hi || hv || hf)) return run_chunk(p, 1, x, nullptr, out_idx, out_val, nullptr, nullptr, out_info, nullptr, st);
    // host buffers: stage through device memory owned by the plan
    const size_t xb = (size_t)p->pd.N * p->xesz;
    const size_t ob = align_up((size_t)p->pd.K * 8, 256) + align_up((size_t)p->pd.K * p->xesz, 256) + 256;
    if (!p->d_out_stage) CK(cudaMalloc(&p->d_out_stage, ob));
    unsigned char* ostage = (unsigned char*)p->d_out_stage;
    int64_t* di = (int64_t*)ostage;
    void* dv = ostage + align_up((size_t)p->pd.K * 8, 256);
    int32_t* dinfo = (int32_t*)(ostage + ob - 256);
    const void* dx = x;
    bool x_sys = false;
    if (hx && p->opts.host_gather) {
        // page-locked host signal: the bucketization reads it in place through its
        // device-side address; pageable memory falls through to the copy
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, x) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer) {
            dx = at.devicePointer;
            x_sys = true;
        } else {
            cudaGetLastError();
        }
    }
    if (hx && !x_sys) {
        if (!p->d_x_stage) CK(cudaMalloc(&p->d_x_stage, xb));
        CK(cudaMemcpyAsync(p->d_x_stage, x, xb, cudaMemcpyHostToDevice, st));
        dx = p->d_x_stage;
    }
    int rc = run_chunk(p, 1, dx, nullptr, hi ? di : out_idx, hv ? dv : out_val, nullptr, nullptr,
                       hf ? dinfo : out_info, nullptr, st, 0, x_sys);
    if (rc) return rc;
    if (hi) CK(cudaMemcpyAsync(out_idx, di, (size_t)p->pd.K * 8, cudaMemcpyDeviceToHost, st));
    if (hv) CK(cudaMemcpyAsync(out_val, dv, (size_t)p->pd.K * p->xesz, cudaMemcpyDeviceToHost, st));
    if (hf) CK(cudaMemcpyAsync(out_info, dinfo, 16, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SFFT_OK;
}

namespace sfft {

static int fill_ptr_table(sfft_plan_s* p, int m, const void* const* xs, int64_t* const* idx,
                          void* const* val, int32_t* const* rows, cudaStream_t st)
{
    const int slot = p->ptr_slot;
    p->ptr_slot ^= 1;
    CK(cudaEventSynchronize(p->ptr_ev[slot]));
    void** h = p->h_ptrs[slot];
    const size_t mb = (size_t)p->max_batch;
    for (int i = 0; i < m; ++i) {
        h[i] = (void*)xs[i];
        h[mb + i] = (void*)idx[i];
        h[2 * mb + i] = val[i];
        h[3 * mb + i] = rows ? (void*)rows[i] : nullptr;
    }
    CK(cudaMemcpyAsync(p->d_ptrs, h, 4 * sizeof(void*) * mb, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(p->ptr_ev[slot], st));
    return SFFT_OK;
}

static int ensure_aux(sfft_plan_s* p)
{
    for (int i = 0; i < 2; ++i) {
        if (!p->aux[i]) CK(cudaStreamCreateWithFlags(&p->aux[i], cudaStreamNonBlocking));
        if (!p->aux_join[i]) CK(cudaEventCreateWithFlags(&p->aux_join[i], cudaEventDisableTiming));
    }
    if (!p->aux_ev) CK(cudaEventCreateWithFlags(&p->aux_ev, cudaEventDisableTiming));
    return SFFT_OK;
}

// n signals of one plan with device buffers, max_batch per launch group.  (Splitting a
// group into sub-batches on two streams, so that one sub-batch's decode overlaps the
// next one's bucketization, measured slower: the kernels contend and the smaller launches
// leave longer wave tails.)
static int execute_group_device(sfft_plan_s* p, int n, const void* const* xs, int64_t* const* idx,
                                void* const* val, int32_t* const* rows, cudaStream_t st)
{
    const size_t mb = (size_t)p->max_batch;
    for (int c0 = 0; c0 < n; c0 += p->max_batch) {
        const int m = std::min(p->max_batch, n - c0);
        int rc;
        if (m == 1) {
            rc = run_chunk(p, 1, xs[c0], nullptr, idx[c0], val[c0], nullptr, nullptr, rows[c0],
                           nullptr, st);
        } else {
            if ((rc = fill_ptr_table(p, m, xs + c0, idx + c0, val + c0, rows + c0, st))) return rc;
            rc = run_chunk(p, m, nullptr, (const void* const*)p->d_ptrs, nullptr, nullptr,
                           (int64_t* const*)(p->d_ptrs + mb), (void* const*)(p->d_ptrs + 2 * mb),
                           nullptr, nullptr, st, 0, false, (int32_t* const*)(p->d_ptrs + 3 * mb));
        }
        if (rc) return rc;
    }
    return SFFT_OK;
}

// n signals of one plan with host buffers: each launch group is split into sub-batches
// that alternate between two streams, so the copies of one sub-batch overlap the kernels
// of the other; the call returns when every output is in host memory.
static int execute_group_host(sfft_plan_s* p, int n, const void* const* xs, int64_t* const* idx,
                              void* const* val, int32_t* const* rows, cudaStream_t st)
{
    const size_t mb = (size_t)p->max_batch;
    const size_t xb = (size_t)p->pd.N * p->xesz;
    const size_t ib = align_up((size_t)p->pd.K * 8, 256), vb = align_up((size_t)p->pd.K * p->xesz, 256);
    if (!p->d_xb_stage) CK(cudaMalloc(&p->d_xb_stage, xb * mb));
    if (!p->d_ob_stage) CK(cudaMalloc(&p->d_ob_stage, (ib + vb) * mb + 16 * mb));
    int rc0 = ensure_aux(p);
    if (rc0) return rc0;
    unsigned char* ob = (unsigned char*)p->d_ob_stage;
    int32_t* dinf = (int32_t*)(ob + (ib + vb) * mb);
    std::vector<const void*> sx(mb);
    std::vector<int64_t*> si(mb);
    std::vector<void*> sv(mb);
    for (size_t i = 0; i < mb; ++i) {
        sx[i] = (unsigned char*)p->d_xb_stage + xb * i;
        si[i] = (int64_t*)(ob + ib * i);
        sv[i] = ob + ib * mb + vb * i;
    }
    // the staging pointer table is the same for every group
    CK(cudaEventRecord(p->aux_ev, st));
    CK(cudaStreamWaitEvent(p->aux[0], p->aux_ev, 0));
    CK(cudaStreamWaitEvent(p->aux[1], p->aux_ev, 0));
    int rc = fill_ptr_table(p, (int)mb, sx.data(), si.data(), sv.data(), nullptr, p->aux[0]);
    if (rc) return rc;
    CK(cudaEventRecord(p->aux_ev, p->aux[0]));
    CK(cudaStreamWaitEvent(p->aux[1], p->aux_ev, 0));
    for (int c0 = 0; c0 < n; c0 += p->max_batch) {
        const int m = std::min(p->max_batch, n - c0);
        const int nsub = std::min(m, 4);
        for (int h = 0; h < nsub; ++h) {
            const int s0 = m * h / nsub, s1 = m * (h + 1) / nsub, ms = s1 - s0;
            if (ms <= 0) continue;
            cudaStream_t ss = p->aux[h & 1];
            for (int i = s0; i < s1; ++i)
                CK(cudaMemcpyAsync((void*)sx[i], xs[c0 + i], xb, cudaMemcpyHostToDevice, ss));
            if (ms == 1)
                rc = run_chunk(p, 1, sx[s0], nullptr, si[s0], sv[s0], nullptr, nullptr, dinf + 4 * s0,
                               nullptr, ss, s0);
            else
                rc = run_chunk(p, ms, nullptr, (const void* const*)p->d_ptrs + s0, nullptr, nullptr,
                               (int64_t* const*)(p->d_ptrs + mb + s0), (void* const*)(p->d_ptrs + 2 * mb + s0),
                               dinf + 4 * s0, nullptr, ss, s0);
            if (rc) return rc;
            for (int i = s0; i < s1; ++i) {
                CK(cudaMemcpyAsync(idx[c0 + i], si[i], (size_t)p->pd.K * 8, cudaMemcpyDeviceToHost, ss));
                CK(cudaMemcpyAsync(val[c0 + i], sv[i], (size_t)p->pd.K * p->xesz, cudaMemcpyDeviceToHost, ss));
            }
            // info rows: one copy when the caller's rows are consecutive, else one per row
            bool consecutive = true;
            for (int i = s0 + 1; i < s1; ++i) consecutive &= rows[c0 + i] == rows[c0 + s0] + 4 * (i - s0);
            if (consecutive) {
                CK(cudaMemcpyAsync(rows[c0 + s0], dinf + 4 * s0, 16 * (size_t)ms, cudaMemcpyDeviceToHost, ss));
            } else {
                for (int i = s0; i < s1; ++i)
                    CK(cudaMemcpyAsync(rows[c0 + i], dinf + 4 * i, 16, cudaMemcpyDeviceToHost, ss));
            }
        }
        // the staging buffers are reused by the next launch group
        CK(cudaStreamSynchronize(p->aux[0]));
        CK(cudaStreamSynchronize(p->aux[1]));
    }
    return SFFT_OK;
}

// n signals of one plan; rows[i] is signal i's info row (int32[4])
int execute_group(sfft_plan_s* p, int n, const void* const* xs, int64_t* const* idx,
                  void* const* val, int32_t* const* rows, cudaStream_t st, bool host = false)
{
    if (!p->layers.empty()) {  // DSFFT: each signal searches its own layers
        for (int i = 0; i < n; ++i) {
            const int rc = sfft_execute(p, xs[i], idx[i], val[i], rows[i], st);
            if (rc) return rc;
        }
        return SFFT_OK;
    }
    return host ? execute_group_host(p, n, xs, idx, val, rows, st)
                : execute_group_device(p, n, xs, idx, val, rows, st);
}
}  // namespace sfft

extern "C" int sfft_execute_batch(int32_t n, const sfft_plan_t* plans, const void* const* xs,
                                  int64_t* const* idx, void* const* val, int32_t* infos,
                                  void* stream)
{
    if (n < 0 || (n > 0 && (!plans || !xs || !idx || !val || !infos))) return SFFT_EINVAL;
    if (n == 0) return SFFT_OK;
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !xs[i] || !idx[i] || !val[i]) return SFFT_EINVAL;
    // all buffers on the device, or all in host memory (staged through the plans)
    const bool host = is_host_ptr(xs[0]);
    for (int i = 0; i < n; ++i)
        if (is_host_ptr(xs[i]) != host || is_host_ptr(idx[i]) != host || is_host_ptr(val[i]) != host)
            return SFFT_EINVAL;
    if (is_host_ptr(infos) != host) return SFFT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // group signals by plan (first-seen order of plans); a group need not be consecutive in
    // the batch: each signal's info row is passed by pointer
    struct Group {
        sfft_plan_s* p;
        std::vector<const void*> x;
        std::vector<int64_t*> i;
        std::vector<void*> v;
        std::vector<int32_t*> r;
    };
    std::vector<Group> groups;
    std::vector<char> done(n, 0);
    for (int i = 0; i < n; ++i) {
        if (done[i]) continue;
        Group g;
        g.p = plans[i];
        for (int k = i; k < n; ++k)
            if (!done[k] && plans[k] == g.p) {
                done[k] = 1;
                g.x.push_back(xs[k]);
                g.i.push_back(idx[k]);
                g.v.push_back(val[k]);
                g.r.push_back(infos + 4 * (size_t)k);
            }
        groups.push_back(std::move(g));
    }
    // With device buffers and several plans, every group after the first runs on a stream of
    // its own plan, forked from and joined back into the caller's stream, so the groups
    // overlap on the device (the smaller signals' launches fill the larger ones' tails).
    // Each plan's workspace serves only its own group, so the streams share nothing.
    const bool fork = !host && groups.size() > 1;
    std::vector<sfft_plan_s*> forked;
    for (size_t g = 0; g < groups.size(); ++g) {
        Group& G = groups[g];
        cudaStream_t gs = st;
        if (fork && g > 0 && G.p->layers.empty()) {
            const int rca = ensure_aux(G.p);
            if (rca) return rca;
            CK(cudaEventRecord(G.p->aux_ev, st));
            CK(cudaStreamWaitEvent(G.p->aux[0], G.p->aux_ev, 0));
            gs = G.p->aux[0];
            forked.push_back(G.p);
        }
        const int rc = execute_group(G.p, (int)G.x.size(), G.x.data(), G.i.data(), G.v.data(),
                                     G.r.data(), gs, host);
        if (rc) return rc;
    }
    for (sfft_plan_s* q : forked) {
        CK(cudaEventRecord(q->aux_join[0], q->aux[0]));
        CK(cudaStreamWaitEvent(st, q->aux_join[0], 0));
    }
    return SFFT_OK;
}

namespace sfft {

// ---- autotuning cache: one JSON object, key -> {"max_tile": .., ...}, in a file ----------
static std::mutex g_tune_mu;
static std::string g_tune_path;

struct TuneEntry {
    int max_tile, overlap_gather, classify_lanes, decode_ctas;
    double rate;
};

// the schedule fields of the cache, in file order
static const char* const kTuneFields[] = {"max_tile", "overlap_gather", "classify_lanes",
                                           "decode_ctas", "rate"};

static std::string tune_key(int64_t N, int32_t K, int32_t D, const int64_t* f, int32_t R,
                            const sfft_opts& o, int32_t n)
{
    std::string k = "N=" + std::to_string(N) + ";f=";
    for (int d = 0; d < D; ++d) k += (d ? "," : "") + std::to_string(f[d]);
    k += ";R=" + std::to_string(R) + ";K=" + std::to_string(K) + ";batch=" + std::to_string(n) +
         ";dtype=" + std::to_string(o.dtype) + ";prec=" + std::to_string(o.precision) +
         ";locate=" + std::to_string(o.locate) + ";noise_auto=" + std::to_string(o.noise_auto) +
         ";decoder=" + std::to_string(o.decoder) + ";fma_only=" + std::to_string(o.dft_fma_only);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
        k += ";gpu=" + std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "sm";
    for (char& c : k)
        if (c == '"' || c == '\\') c = '_';
    return k;
}

// every entry of the cache file: key -> the text of its object
static std::vector<std::pair<std::string, std::string>> tune_read(const std::string& path)
{
    std::vector<std::pair<std::string, std::string>> out;
    FILE* fp = fopen(path.c_str(), "rb");
    if (!fp) return out;
    std::string txt;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), fp)) > 0) txt.append(buf, got);
    fclose(fp);
    size_t i = 0;
    while (true) {
        const size_t q0 = txt.find('"', i);
        if (q0 == std::string::npos) break;
        const size_t q1 = txt.find('"', q0 + 1);
        const size_t b0 = q1 == std::string::npos ? q1 : txt.find('{', q1);
        const size_t b1 = b0 == std::string::npos ? b0 : txt.find('}', b0);
        if (b1 == std::string::npos) break;
        out.emplace_back(txt.substr(q0 + 1, q1 - q0 - 1), txt.substr(b0, b1 - b0 + 1));
        i = b1 + 1;
    }
    return out;
}

static bool tune_field(const std::string& obj, const char* name, double* v)
{
    const std::string pat = std::string("\"") + name + "\"";
    const size_t at = obj.find(pat);
    if (at == std::string::npos) return false;
    const size_t colon = obj.find(':', at + pat.size());
    if (colon == std::string::npos) return false;
    char* end = nullptr;
    *v = strtod(obj.c_str() + colon + 1, &end);
    return end != obj.c_str() + colon + 1;
}

static bool tune_lookup(const std::string& key, TuneEntry* e)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_path.empty()) return false;
    for (auto& kv : tune_read(g_tune_path)) {
        if (kv.first != key) continue;
        double v[5];
        for (int i = 0; i < 5; ++i)
            if (!tune_field(kv.second, kTuneFields[i], &v[i])) return false;
        *e = TuneEntry{(int)v[0], (int)v[1], (int)v[2], (int)v[3], v[4]};
        return true;
    }
    return false;
}

static void tune_store(const std::string& key, const TuneEntry& e)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_path.empty()) return;
    auto all = tune_read(g_tune_path);
    char obj[256];
    snprintf(obj, sizeof(obj),
             "{\"max_tile\": %d, \"overlap_gather\": %d, \"classify_lanes\": %d, "
             "\"decode_ctas\": %d, \"rate\": %.6g}",
             e.max_tile, e.overlap_gather, e.classify_lanes, e.decode_ctas, e.rate);
    bool found = false;
    for (auto& kv : all)
        if (kv.first == key) {
            kv.second = obj;
            found = true;
        }
    if (!found) all.emplace_back(key, obj);
    const std::string tmp = g_tune_path + ".tmp";
    FILE* fp = fopen(tmp.c_str(), "wb");
    if (!fp) return;
    fputs("{\n", fp);
    for (size_t i = 0; i < all.size(); ++i)
        fprintf(fp, "  \"%s\": %s%s\n", all[i].first.c_str(), all[i].second.c_str(),
                i + 1 < all.size() ? "," : "");
    fputs("}\n", fp);
    fclose(fp);
    rename(tmp.c_str(), g_tune_path.c_str());
}

}  // namespace sfft

extern "C" int sfft_autotune_cache(const char* path)
{
    std::lock_guard<std::mutex> lk(sfft::g_tune_mu);
    sfft::g_tune_path = path ? path : "";
    return SFFT_OK;
}

extern "C" int sfft_autotune(int64_t N, int32_t K, int32_t n_stages, const int64_t* f,
                             int32_t n_delays, const int64_t* delays, const sfft_opts* base,
                             int32_t n, const void* const* xs, void* stream, sfft_opts* best,
                             double* best_rate)
{
    if (!base || !best || !xs || !f || !delays || n < 1 || n_stages < 1) return SFFT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const std::string key = tune_key(N, K, n_stages, f, n_delays, *base, n);
    sfft_opts bo = *base;
    bo.max_batch = n;
    TuneEntry cached;
    if (tune_lookup(key, &cached)) {
        bo.max_tile = cached.max_tile;
        bo.overlap_gather = cached.overlap_gather;
        bo.classify_lanes = cached.classify_lanes;
        bo.decode_ctas = cached.decode_ctas;
        *best = bo;
        if (best_rate) *best_rate = cached.rate;
        return SFFT_OK;
    }
    std::vector<int64_t*> idx(n);
    std::vector<void*> val(n);
    int32_t* infos = nullptr;
    void* outbuf = nullptr;
    const size_t xesz = base->dtype == SFFT_C128 ? 16 : 8;
    const size_t per = align_up((size_t)K * 8, 256) + align_up((size_t)K * xesz, 256);
    CK(cudaMalloc(&outbuf, per * n));
    if (cudaMalloc((void**)&infos, 16 * (size_t)n) != cudaSuccess) {
        cudaFree(outbuf);
        return SFFT_ENOMEM;
    }
    for (int i = 0; i < n; ++i) {
        idx[i] = (int64_t*)((unsigned char*)outbuf + per * i);
        val[i] = (unsigned char*)outbuf + per * i + align_up((size_t)K * 8, 256);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SFFT_OK;
    // signals/s of one schedule: 2 warm-up and 3 timed batches; -1 if it cannot run
    auto trial = [&](const sfft_opts& o) -> double {
        sfft_plan_t p = nullptr;
        if (sfft_plan_create(&p, N, K, n_stages, f, n_delays, delays, &o) != SFFT_OK) return -1.0;
        std::vector<sfft_plan_t> ps(n, p);
        int r = SFFT_OK;
        for (int w = 0; w < 2 && r == SFFT_OK; ++w)
            r = sfft_execute_batch(n, ps.data(), xs, idx.data(), val.data(), infos, st);
        const int reps = 3;
        cudaEventRecord(e0, st);
        for (int w = 0; w < reps && r == SFFT_OK; ++w)
            r = sfft_execute_batch(n, ps.data(), xs, idx.data(), val.data(), infos, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        sfft_plan_destroy(p);
        if (r != SFFT_OK) {
            rc = r;
            return -1.0;
        }
        return (double)n * reps / (ms / 1e3);
    };
    // coordinate descent over the schedule axes, from the defaults: the B-tile (largest DFT
    // tile a CTA holds: whole stage, or two passes of smaller tiles), the gather schedule
    // (persistent overlapped or one CTA per tile), the lanes per bin of the ML search, the
    // CTAs per signal of the peeling rounds
    sfft_opts cur = bo;
    cur.max_tile = 0;
    cur.overlap_gather = 0;
    cur.classify_lanes = 0;
    cur.decode_ctas = 0;
    double best_v = trial(cur);
    auto sweep = [&](int sfft_opts::*field, std::initializer_list<int> values) {
        for (int v : values) {
            if (cur.*field == v) continue;
            sfft_opts o = cur;
            o.*field = v;
            const double r = trial(o);
            if (r > best_v * 1.01) {
                best_v = r;
                cur = o;
            }
        }
    };
    sweep(&sfft_opts::max_tile, {16384, 8192, 4096});
    sweep(&sfft_opts::overlap_gather, {1});
    if (base->locate == SFFT_LOCATE_ML) sweep(&sfft_opts::classify_lanes, {1, 2, 4, 8, 16, 32});
    sweep(&sfft_opts::decode_ctas, {1, 2, 4, 8});
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(outbuf);
    cudaFree(infos);
    if (best_v < 0) return rc ? rc : SFFT_EINVAL;
    tune_store(key, TuneEntry{cur.max_tile, cur.overlap_gather, cur.classify_lanes, cur.decode_ctas,
                              best_v});
    *best = cur;
    if (best_rate) *best_rate = best_v;
    return SFFT_OK;
}

extern "C" int sfft_plan_set_profiling(sfft_plan_t p, int enable)
{
    if (!p) return SFFT_EINVAL;
    p->prof = enable != 0;
    return SFFT_OK;
}

extern "C" int sfft_plan_profile(sfft_plan_t p, double* ms, int64_t* launches, int64_t* calls,
                                 int reset)
{
    if (!p) return SFFT_EINVAL;
    for (auto& e : p->prof_pending) {
        CK(cudaEventSynchronize(e.b));
        float t = 0;
        CK(cudaEventElapsedTime(&t, e.a, e.b));
        p->prof_ms[e.phase] += t;
        p->prof_launches[e.phase] += e.launches;
        p->prof_calls[e.phase] += 1;
        p->prof_pool.push_back(e.a);
        p->prof_pool.push_back(e.b);
    }
    p->prof_pending.clear();
    for (int i = 0; i < 3; ++i) {
        if (ms) ms[i] = p->prof_ms[i];
        if (launches) launches[i] = p->prof_launches[i];
        if (calls) calls[i] = p->prof_calls[i];
        if (reset) {
            p->prof_ms[i] = 0;
            p->prof_launches[i] = 0;
            p->prof_calls[i] = 0;
        }
    }
    return SFFT_OK;
}

extern "C" int sfft_bucketize(sfft_plan_t p, const void* x, void* bins, void* stream)
{
    if (!p || !x || !bins || !p->layers.empty()) return SFFT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    BucketArgs a;
    memset(&a, 0, sizeof(a));
    a.pd = p->pd;
    a.n_sig = 1;
    a.nidx = p->d_nidx;
    a.tw = p->d_tw;
    a.x0 = x;
    a.scratch = p->d_scratch;
    a.bins = p->d_bins;
    for (int pass = 0; pass < (p->need_pass2 ? 2 : 1); ++pass) {
        const PassDesc* src = pass == 0 ? p->pass1 : p->pass2;
        a.tile_prefix[0] = 0;
        for (int d = 0; d < kMaxStages; ++d) {
            a.pass[d] = d < p->pd.D ? src[d] : PassDesc{};
            a.tile_prefix[d + 1] = a.tile_prefix[d] + (d < p->pd.D ? src[d].n_tiles * p->pd.R : 0);
        }
        a.tiles_per_sig = a.tile_prefix[kMaxStages];
        CK(bucketize_pass(p, a, pass, st));
    }
    CK(launch_bins_to_natural(p->pd, p->d_pbin, p->d_bins, bins, p->prec, 1, st));
    return SFFT_OK;
}

extern "C" int sfft_decode_bins(sfft_plan_t p, const void* bins, int64_t* out_idx, void* out_val,
                                int32_t* out_info, void* stream)
{
    if (!p || !bins || !out_idx || !out_val || !out_info || !p->layers.empty()) return SFFT_EINVAL;
    return run_chunk(p, 1, nullptr, nullptr, out_idx, out_val, nullptr, nullptr, out_info, bins,
                     (cudaStream_t)stream);
}

extern "C" const char* sfft_error_string(int code)
{
    switch (code) {
        case SFFT_OK: return "ok";
        case SFFT_PENDING: return "pending";
        case SFFT_INCOMPLETE: return "incomplete: peeling ended with unresolved bins";
        case SFFT_EINVAL: return "invalid argument";
        case SFFT_ENOMEM: return "out of memory";
        case SFFT_ECUDA: return "CUDA error";
        case SFFT_ETIMEDOUT: return "device wait timed out";
        case SFFT_EADMIT: return "request exceeds the server memory budget";
        case SFFT_ENOTFOUND: return "unknown ticket";
        case SFFT_EBUSY: return "server queue full";
        case SFFT_ETOOBIG: return "problem larger than the static scratch of sfft_bucketize_static";
        default: return "unknown code";
    }
}

extern "C" const char* sfft_last_cuda_error(void) { return sfft::g_last_cuda; }
