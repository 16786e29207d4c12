// noalloc.cu -- sfft_bucketize_static: the bucketization (gather + prime-factor DFTs)
// without any device allocation.
//
// Who needs it: code that cannot call cudaMalloc -- a host application or framework whose
// own allocator has already reserved the GPU's memory (a further cudaMalloc fails or is
// not allowed), or a latency-critical loop where cudaMalloc/cudaFree would synchronise the
// device and stall other streams.  Such callers cannot create a plan (plans own device
// tables and workspace), so this entry point takes the problem description directly.
//
// Memory: the index maps, twiddles, the inter-pass scratch of two-pass stages and the
// storage-order bins all live in one file-scope __device__ array of kStaticBytes (16 MiB),
// which every GPU that loads the library holds until the process exits.  Problems needing
// more are rejected with SFFT_ETOOBIG.  Every call rewrites the parts it uses (nothing has
// to start at zero); calls share the one array, so calls that overlap on the GPU (other
// streams, other host threads) race and must be ordered by the caller.
//
// Device address: in host code the array's name is only a host-side stand-in, so every
// call resolves the device address with cudaGetSymbolAddress, with the caller's device
// current (cheap next to the launches, and it stays right if the device's context is torn
// down and made again).  The first call on each device also loads the library's device
// code there, so it should come before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "launch.h"
#include "pfa_layout.h"
#include "sfft.h"
#include "sfft_internal.cuh"

namespace sfft {
cudaError_t set_bucketize_smem_limit(int max_smem);
int cuda_fail(cudaError_t e);
}  // namespace sfft

using namespace sfft;

namespace {

constexpr size_t kStaticBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;

// Tables of one call, computed on the device from the description: input sample index and
// bin of every storage position, and the twiddles of every axis.
template <typename T>
__global__ void static_tables_kernel(const __grid_constant__ PlanDesc pd, int32_t* nidx,
                                     int32_t* pbin, typename C2<T>::t* tw, int32_t n_tw)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < pd.sumB) {
        int d = 0;
        while (d + 1 < pd.D && i >= pd.st[d + 1].bin_base) ++d;
        const StageDesc& s = pd.st[d];
        const int32_t pos = (int32_t)(i - s.bin_base);
        int64_t n = 0, j = 0;
        for (int a = 0; a < s.n_axes; ++a) {
            const AxisDesc& A = s.ax[a];
            const int32_t c = (pos / A.S) % A.P;
            n += (int64_t)(A.pow2 ? bitrev(c, A.log2P) : c) * A.rur;
            j += (int64_t)c * A.crt;
        }
        nidx[i] = (int32_t)(n % s.B);
        pbin[i] = (int32_t)(j % s.B);
    }
    if (i < n_tw) {
        // the axis owning twiddle slot i (layout of axis_tw_residue, or the fragment table
        // of a tensor-core axis)
        for (int d = 0; d < pd.D; ++d)
            for (int a = 0; a < pd.st[d].n_axes; ++a) {
                const AxisDesc& A = pd.st[d].ax[a];
                const int cnt = axis_tw_count(A.P, A.pow2, A.tc);
                if (i >= A.tw_off && i < A.tw_off + cnt) {
                    if constexpr (sizeof(T) == 4) {
                        if (A.tc) {
                            const int e = (int)(i - A.tw_off);
                            tw[i] = typename C2<T>::t{__uint_as_float(tc_twiddle_word(A.P, 2 * e)),
                                                      __uint_as_float(tc_twiddle_word(A.P, 2 * e + 1))};
                            continue;
                        }
                    }
                    double sv, cv;
                    const int32_t t = axis_tw_residue(A.P, A.pow2, (int)(i - A.tw_off));
                    sincospi(2.0 * (double)t / (double)A.P, &sv, &cv);
                    tw[i] = typename C2<T>::t{(T)cv, (T)sv};
                }
            }
    }
}

// the array's device address on the current device, and the device's shared-memory limit
// (applied to the bucketization kernels)
int device_scratch(void** ptr, int* max_smem)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return SFFT_EINVAL;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    int sm = 0;
    e = cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    e = set_bucketize_smem_limit(sm);
    if (e != cudaSuccess) return cuda_fail(e);
    *ptr = p;
    *max_smem = sm;
    return SFFT_OK;
}

// The prime-factor maps of a stage's layout must be inverse permutations: position p holds
// bin j = sum_a k_a crt_a mod B (k_a the p's coordinate on axis a), and bin j sits at
// sum_a (j mod P_a) S_a.  Checked on the host without allocating; a layout that fails it
// would store bins in the wrong places.
bool crt_maps_consistent(const StageDesc& s)
{
    for (int32_t pos = 0; pos < s.B; ++pos) {
        int64_t j = 0;
        for (int a = 0; a < s.n_axes; ++a) j += (int64_t)((pos / s.ax[a].S) % s.ax[a].P) * s.ax[a].crt;
        if (bin_to_pos(s, (int32_t)(j % s.B)) != pos) return false;
    }
    return true;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" int sfft_bucketize_static(int64_t N, int32_t n_stages, const int64_t* f,
                                     int32_t n_delays, const int64_t* delays, int32_t precision,
                                     int32_t dtype, const void* x, void* bins, void* stream)
{
    if (!f || !delays || !x || !bins) return SFFT_EINVAL;
    if (N < 1 || N >= (1ll << 30) || n_stages < 1 || n_stages > kMaxStages || n_delays < 1 ||
        n_delays > kMaxDelays)
        return SFFT_EINVAL;
    if ((precision != SFFT_PREC_FP32 && precision != SFFT_PREC_FP64) ||
        (dtype != SFFT_C64 && dtype != SFFT_C128))
        return SFFT_EINVAL;
    for (int d = 0; d < n_stages; ++d) {
        if (f[d] < 1 || N % f[d] != 0) return SFFT_EINVAL;
        for (int e = 0; e < d; ++e)
            if (pfa_gcd(f[d], f[e]) != 1) return SFFT_EINVAL;
        for (int r = 0; r < n_delays; ++r) {
            const int64_t t = delays[(int64_t)d * n_delays + r];
            if (t < 0 || t >= N) return SFFT_EINVAL;
            for (int q = 0; q < r; ++q)
                if (delays[(int64_t)d * n_delays + q] == t) return SFFT_EINVAL;
        }
    }
    const int prec = precision == SFFT_PREC_FP32 ? 1 : 0;
    const size_t esz = prec ? 8 : 16;
    int64_t sumB = 0;
    for (int d = 0; d < n_stages; ++d) sumB += N / f[d];
    // size check before any device work (index tables and the two bin arrays; the exact
    // check, twiddles included, follows the layout below)
    const size_t need = up256(4 * (size_t)sumB) * 2 + 2 * up256(esz * (size_t)sumB * n_delays);
    if (need > kStaticBytes) return SFFT_ETOOBIG;

    void* base = nullptr;
    int max_smem = 0;
    int rc = device_scratch(&base, &max_smem);
    if (rc) return rc;

    BucketArgs a;
    memset(&a, 0, sizeof(a));
    PassDesc pass2[kMaxStages];
    memset(pass2, 0, sizeof(pass2));
    PlanDesc& pd = a.pd;
    pd.N = (int32_t)N;
    pd.D = n_stages;
    pd.R = n_delays;
    pd.K = 1;
    const int64_t tile_target = prec ? 4096 : 2048;
    int32_t n_tw = 0, bin_base = 0;
    PassPlan l1, l2;
    bool two = false;
    for (int d = 0; d < n_stages; ++d) {
        StageDesc& s = pd.st[d];
        const int64_t L = f[d], B = N / L;
        s.B = (int32_t)B;
        s.L = (int32_t)L;
        if (!pfa_layout_stage(&s, esz, max_smem, tile_target, &a.pass[d], &pass2[d], &l1, &l2,
                              &n_tw, &two))
            return SFFT_EINVAL;
        if (!crt_maps_consistent(s)) return SFFT_EINVAL;
        for (int r = 0; r < n_delays; ++r) s.tau[r] = (int32_t)delays[(int64_t)d * n_delays + r];
        s.r0 = s.r1 = -1;
        s.bin_base = bin_base;
        s.y_off = bin_base * n_delays;
        bin_base += (int32_t)B;
    }
    pd.sumB = bin_base;
    pd.y_per_sig = (int64_t)bin_base * n_delays;

    // carve the static array: nidx | pbin | twiddles | scratch | storage-order bins
    unsigned char* p = (unsigned char*)base;
    int32_t* nidx = (int32_t*)p;
    p += up256(4 * (size_t)sumB);
    int32_t* pbin = (int32_t*)p;
    p += up256(4 * (size_t)sumB);
    void* tw = p;
    p += up256(esz * (size_t)n_tw);
    void* scratch = p;
    p += up256(esz * (size_t)pd.y_per_sig);
    void* sbins = p;
    p += up256(esz * (size_t)pd.y_per_sig);
    if ((size_t)(p - (unsigned char*)base) > kStaticBytes) return SFFT_ETOOBIG;

    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nt = sumB > n_tw ? sumB : n_tw;
    const unsigned grid = (unsigned)((nt + 255) / 256);
    if (prec)
        static_tables_kernel<float><<<grid, 256, 0, st>>>(pd, nidx, pbin, (float2*)tw, n_tw);
    else
        static_tables_kernel<double><<<grid, 256, 0, st>>>(pd, nidx, pbin, (double2*)tw, n_tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);

    a.n_sig = 1;
    a.nidx = nidx;
    a.tw = tw;
    a.x0 = x;
    a.scratch = scratch;
    a.bins = sbins;
    for (int pass = 0; pass < (two ? 2 : 1); ++pass) {
        if (pass == 1)
            for (int d = 0; d < kMaxStages; ++d) a.pass[d] = d < n_stages ? pass2[d] : PassDesc{};
        a.tile_prefix[0] = 0;
        for (int d = 0; d < kMaxStages; ++d)
            a.tile_prefix[d + 1] = a.tile_prefix[d] + (d < n_stages ? a.pass[d].n_tiles * n_delays : 0);
        a.tiles_per_sig = a.tile_prefix[kMaxStages];
        e = launch_bucketize(a, prec, dtype == SFFT_C128 ? 1 : 0,
                             pfa_threads(pass == 0 ? l1.tile : l2.tile, esz), pass == 0 ? l1.smem : l2.smem, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    e = launch_bins_to_natural(pd, pbin, sbins, bins, prec, 1, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return SFFT_OK;
}
