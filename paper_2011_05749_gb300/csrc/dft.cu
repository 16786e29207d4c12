// dft.cu -- bucketization kernels: strided delayed gather (Eq. 5, with the shift of
// Eq. 3-4) fused with the B-point DFTs of Eq. 6 / Eq. 19.
//
// Each B_d-point DFT is split by the prime-factor (Good-Thomas) map into co-prime
// prime-power axes, so no twiddles are needed between axes: odd axes are done as direct
// DFTs with the conjugate-pair symmetry (a 2P-real-FMA inner product per output pair),
// power-of-two axes as in-place radix-2 decimation-in-time FFTs.  A tile of the stage
// array lives in shared memory for a whole pass.  When B_d fits in shared memory the stage
// is one pass straight from x to the bins; otherwise the outer axes run first (from x into
// scratch) and the inner axes second (scratch to bins).  No tensor cores: this is not a
// dense contraction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "sfft_internal.cuh"

namespace sfft {

// In-place P-point DFTs (P odd) along one axis of a shared-memory tile.
//   sub-DFT m starts at (m % LS) + (m / LS) * LS * P, element n at + n * LS.
// X_k = x_0 + sum_{n=1}^{(P-1)/2} [ (x_n + x_{P-n}) cos(2 pi n k / P)
//                                   - i (x_n - x_{P-n}) sin(2 pi n k / P) ],
// X_{P-k} the same with the sine term negated.  Thread (g, m) computes GP output pairs.
template <typename T, int GP>
__device__ void axis_dft_odd(typename C2<T>::t* s, const typename C2<T>::t* tw, int P, int LS,
                             int TS)
{
    using V = typename C2<T>::t;
    const int M = TS / P;
    const int pairs = (P - 1) >> 1;
    const int NG = (pairs + GP - 1) / GP;
    const int Mc = max(1, (int)blockDim.x / NG);
    const int g = threadIdx.x / Mc;
    const int ml = threadIdx.x - g * Mc;
    for (int m0 = 0; m0 < M; m0 += Mc) {
        const int m = m0 + ml;
        const bool act = g < NG && m < M;
        V acc[GP], sac[GP];
        int idx[GP], kk[GP];
        V x0 = {0, 0}, dc = {0, 0};
        int base = 0;
        if (act) {
            base = (m % LS) + (m / LS) * LS * P;
            x0 = s[base];
            dc = x0;
#pragma unroll
            for (int i = 0; i < GP; ++i) {
                const int k = g * GP + 1 + i;
                kk[i] = k <= pairs ? k : 0;
                idx[i] = 0;
                acc[i] = {0, 0};
                sac[i] = {0, 0};
            }
            for (int n = 1; n <= pairs; ++n) {
                const V xa = s[base + n * LS];
                const V xb = s[base + (P - n) * LS];
                const V av = {xa.x + xb.x, xa.y + xb.y};
                const V bv = {xa.x - xb.x, xa.y - xb.y};
                dc.x += av.x;
                dc.y += av.y;
#pragma unroll
                for (int i = 0; i < GP; ++i) {
                    idx[i] += kk[i];
                    if (idx[i] >= P) idx[i] -= P;
                    const V w = tw[idx[i]];
                    acc[i].x = fma(av.x, w.x, acc[i].x);
                    acc[i].y = fma(av.y, w.x, acc[i].y);
                    sac[i].x = fma(bv.x, w.y, sac[i].x);
                    sac[i].y = fma(bv.y, w.y, sac[i].y);
                }
            }
        }
        __syncthreads();
        if (act) {
            if (g == 0) s[base] = dc;
#pragma unroll
            for (int i = 0; i < GP; ++i) {
                if (kk[i] == 0) continue;
                const int k = kk[i];
                const V c = {x0.x + acc[i].x, x0.y + acc[i].y};
                s[base + k * LS] = V{c.x + sac[i].y, c.y - sac[i].x};
                s[base + (P - k) * LS] = V{c.x - sac[i].y, c.y + sac[i].x};
            }
        }
        __syncthreads();
    }
}

// In-place radix-2 decimation-in-time FFTs of length P = 2^log2P along one axis; the
// input is stored bit-reversed along the axis, the output comes out in natural order.
// tw[t] = (cos, sin)(2 pi t / P), t < P / 2.
template <typename T>
__device__ void axis_fft_pow2(typename C2<T>::t* s, const typename C2<T>::t* tw, int P,
                              int log2P, int LS, int TS)
{
    using V = typename C2<T>::t;
    const int M = TS / P;
    const int half = P >> 1;
    const int nb = M * half;
    for (int lh = 0; lh < log2P; ++lh) {
        const int h = 1 << lh;
        for (int w = threadIdx.x; w < nb; w += blockDim.x) {
            int i, m;
            if (LS == 1) {
                i = w & (half - 1);
                m = w >> (log2P - 1);
            } else {
                m = w % M;
                i = w / M;
            }
            const int grp = i >> lh, ii = i & (h - 1);
            const int base = (m % LS) + (m / LS) * LS * P;
            const int p0 = base + ((grp << (lh + 1)) + ii) * LS;
            const int p1 = p0 + h * LS;
            const V wv = tw[ii << (log2P - 1 - lh)];
            const V u = s[p0], v = s[p1];
            const V vt = {v.x * wv.x + v.y * wv.y, v.y * wv.x - v.x * wv.y};
            s[p0] = V{u.x + vt.x, u.y + vt.y};
            s[p1] = V{u.x - vt.x, u.y - vt.y};
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void axis_dft_odd_dispatch(typename C2<T>::t* s,
                                                      const typename C2<T>::t* tw, int P,
                                                      int LS, int TS)
{
    const int pairs = (P - 1) >> 1;
    if (pairs <= 1)
        axis_dft_odd<T, 1>(s, tw, P, LS, TS);
    else if (pairs <= 2)
        axis_dft_odd<T, 2>(s, tw, P, LS, TS);
    else if (pairs <= 4)
        axis_dft_odd<T, 4>(s, tw, P, LS, TS);
    else
        axis_dft_odd<T, 8>(s, tw, P, LS, TS);
}

template <typename XS, typename V>
__device__ __forceinline__ V load_sample(const void* x, int32_t i)
{
    using XV = typename C2<XS>::t;
    const XV v = __ldg(reinterpret_cast<const XV*>(x) + i);
    return V{(decltype(V{}.x))v.x, (decltype(V{}.x))v.y};
}

// One block = one tile of one (signal, stage, delay).  Block order within a signal:
// (stage, tile, delay), so the delays of a tile run back to back and share x's sectors.
template <typename T, typename XS>
__global__ void __launch_bounds__(512) bucketize_kernel(const __grid_constant__ BucketArgs a)
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
    V* tws = s + TS;

    // twiddles of this pass' axes
    {
        const V* twg = reinterpret_cast<const V*>(a.tw);
        int off = 0;
        for (int ax = a0; ax < a1; ++ax) {
            const int n = st.ax[ax].pow2 ? (st.ax[ax].P >> 1) : st.ax[ax].P;
            for (int t = threadIdx.x; t < n; t += blockDim.x) tws[off + t] = twg[st.ax[ax].tw_off + t];
            off += n;
        }
    }

    const int64_t slot = (int64_t)sig * a.pd.y_per_sig + st.y_off + (int64_t)r * st.B;
    const void* x = a.xs ? a.xs[sig] : a.x0;
    const int tau = st.tau[r], L = st.L, N = a.pd.N;
    const int32_t* nidx = a.nidx + st.bin_base;
    const V* scr = reinterpret_cast<const V*>(a.scratch);

    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
        const int tb = e % Tb;
        const int rest = e / Tb;
        const int g = rest % G;
        const int ta = rest / G;
        const int pb = tb0 + tb, pa = ta0 + ta;
        V v = {0, 0};
        if (pb < Sb && pa < above) {
            const int p = pb + Sb * g + Sab * pa;
            if (ps.src_gather) {
                int xi = __ldg(nidx + p) * L + tau;
                if (xi >= N) xi -= N;
                v = load_sample<XS, V>(x, xi);
            } else {
                v = __ldcg(scr + slot + p);
            }
        }
        s[e] = v;
    }
    __syncthreads();

    int off = 0;
    for (int ax = a0; ax < a1; ++ax) {
        const AxisDesc& A = st.ax[ax];
        const int LS = Tb * (A.S / Sb);
        if (A.pow2)
            axis_fft_pow2<T>(s, tws + off, A.P, A.log2P, LS, TS);
        else if (A.P > 1)
            axis_dft_odd_dispatch<T>(s, tws + off, A.P, LS, TS);
        off += A.pow2 ? (A.P >> 1) : A.P;
    }

    V* dst = reinterpret_cast<V*>(ps.dst_bins ? a.bins : a.scratch);
    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
        const int tb = e % Tb;
        const int rest = e / Tb;
        const int g = rest % G;
        const int ta = rest / G;
        const int pb = tb0 + tb, pa = ta0 + ta;
        if (pb < Sb && pa < above) {
            const int p = pb + Sb * g + Sab * pa;
            __stcg(dst + slot + p, s[e]);
        }
    }
}

template <typename T>
__global__ void twiddle_kernel(typename C2<T>::t* tw, const int32_t* P_of, const int32_t* t_of,
                               int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
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

cudaError_t launch_bucketize(const BucketArgs& a, int precision, int xdouble, int threads,
                             size_t smem, cudaStream_t st)
{
    const unsigned grid = (unsigned)a.n_sig * (unsigned)a.tiles_per_sig;
    if (grid == 0) return cudaSuccess;
    if (precision == 1) {
        if (xdouble)
            bucketize_kernel<float, double><<<grid, threads, smem, st>>>(a);
        else
            bucketize_kernel<float, float><<<grid, threads, smem, st>>>(a);
    } else {
        if (xdouble)
            bucketize_kernel<double, double><<<grid, threads, smem, st>>>(a);
        else
            bucketize_kernel<double, float><<<grid, threads, smem, st>>>(a);
    }
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
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(bucketize_kernel<float, float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(bucketize_kernel<float, double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(bucketize_kernel<double, float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    return cudaFuncSetAttribute(bucketize_kernel<double, double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

}  // namespace sfft
