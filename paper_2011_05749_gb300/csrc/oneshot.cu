// oneshot.cu -- the sFFT-DT one-shot decoder (Sec. 3.1, Eq. 7-18; Sec. 4.1, Stage 2) on the
// bins of a single stage of B buckets (L = N / B candidates per bucket).
//
// Delay slots: r = 0 .. 3 a_m - 1 hold tau = r - a_m (mod N), so bucket i's moments are
// m_k = Y[k + a_m][i] / B = sum_{f = i mod B} xhat_f z_f^k, z_f = e^{2 pi i f / N}
// (Eq. 7-8); the remaining P slots hold the random delays of Step 3.
//
//   DT1  Step 1: singular values of each bucket's Hankel matrix M_{a_m} = [m_{r+c}]
//        (Eq. 10-11), as square roots of the eigenvalues of M^H M (cyclic complex Jacobi).
//   DT2  the vote: per signal, the K-th largest singular value above the floor, by an
//        8-bit radix select on the FP64 bit patterns (one CTA per signal).
//   DT3  Steps 2-3, one warp per bucket with a > 0 votes.  Step 2 by one of the paper's
//        three methods: C = M_a^{-1} M_s (Eq. 14), then |P(z)| (Eq. 12) at every candidate
//        (the lanes split them) and the a smallest (method 2, the default), or the roots of
//        P(z) (method 1); or the matrix pencil on the right singular vectors of Eq. 15's
//        Toeplitz Y (method 3, as Sec. 4.1 runs it), whose eigenvalues are the z_j.  Roots
//        are snapped to the bucket's candidates by angle.  Then subspace
//        pursuit over the atoms {f, f + B, f - B} with the P random-delay measurements
//        (Eq. 18), lane r holding measurement r.
// The per-bucket arithmetic is FP64 whatever the bins' type (position and value
// estimation).  Results go to the slot's recovered list; compaction follows as for the
// peeling decoder.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "launch.h"
#include "sfft_internal.cuh"

namespace sfft {

namespace {

constexpr int kSolveThreads = 256;           // 8 warps, one bucket each
// per-warp shared scratch of the matrix pencil (pencil_points): moments W[0 .. 6], H at
// W[8 .. 23], its eigenvectors at W[24 .. 39], G (3 x 3) at W[40 .. 48]; rounded up to a
// multiple of 4 entries so that every warp's slice starts on a 64-byte boundary
constexpr int kPencilWords = 52;
static_assert(40 + 3 * 3 <= kPencilWords, "pencil scratch must hold G for a_m = 3");
constexpr int kMaxAtoms = 9;                 // 3 a_m
constexpr int kMaxFit = 6;                   // 2 a_m atoms in a union fit

struct Cd {
    double x, y;
};
__device__ __forceinline__ Cd cd(double x, double y) { return Cd{x, y}; }
__device__ __forceinline__ Cd operator+(Cd a, Cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ Cd operator-(Cd a, Cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ Cd operator*(Cd a, Cd b)
{
    return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ Cd conjd(Cd a) { return {a.x, -a.y}; }
__device__ __forceinline__ double abs2(Cd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ Cd divd(Cd a, Cd b)
{
    const double d = 1.0 / abs2(b);
    return {(a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d};
}

// e^{2 pi i t / N} for 0 <= t < N from the plan's two-level root table (entries of the
// plan's arithmetic type): e^{2 pi i (t >> s) 2^s / N} e^{2 pi i (t & (2^s - 1)) / N}
template <typename T>
__device__ __forceinline__ Cd root_n(const PlanDesc& pd, const void* roots, int64_t t)
{
    using V = typename C2<T>::t;
    const V* tw = reinterpret_cast<const V*>(roots);
    const V hi = __ldg(tw + pd.ph_hi_off + (int)(t >> pd.ph_shift));
    const V lo = __ldg(tw + pd.ph_lo_off + (int)(t & ((1 << pd.ph_shift) - 1)));
    return Cd{(double)hi.x, (double)hi.y} * Cd{(double)lo.x, (double)lo.y};
}

__device__ __forceinline__ int ldv(const int32_t* p) { return *(const volatile int32_t*)p; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ Cd warp_sum(Cd v) { return {warp_sum(v.x), warp_sum(v.y)}; }

// Solve A x = b (n <= kMaxFit, complex, row-major n x n in shared memory) by Gaussian
// elimination with partial pivoting, as LAPACK's gesv does; false on an exactly zero pivot.
// One lane works; A and b are overwritten, x replaces b.
__device__ bool solve_lane(Cd* A, Cd* b, int n)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = abs2(A[k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            const double v = abs2(A[i * n + k]);
            if (v > best) {
                best = v;
                piv = i;
            }
        }
        if (best == 0.0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                const Cd t = A[k * n + j];
                A[k * n + j] = A[piv * n + j];
                A[piv * n + j] = t;
            }
            const Cd t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            const Cd l = divd(A[i * n + k], A[k * n + k]);
            for (int j = k + 1; j < n; ++j) A[i * n + j] = A[i * n + j] - l * A[k * n + j];
            b[i] = b[i] - l * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        Cd s = b[k];
        for (int j = k + 1; j < n; ++j) s = s - A[k * n + j] * b[j];
        b[k] = divd(s, A[k * n + k]);
    }
    return true;
}

// Eigenvalues of a Hermitian n x n matrix (n = NN <= 3, unrolled so G stays in registers)
// by cyclic Jacobi rotations: for the pivot g = G[p][q] = |g| e^{i phi}, the phase e^{-i phi}
// on coordinate q makes the 2 x 2 block real symmetric, and the rotation with
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (G_qq - G_pp) / (2 |g|), annihilates it.
template <int NN>
__device__ __forceinline__ void jacobi_rotate(Cd (&G)[3][3], int p, int q)
{
    const double ag = sqrt(abs2(G[p][q]));
    const double a = G[p][p].x, b = G[q][q].x;
    if (ag <= 1e-300 || ag <= 1e-18 * (fabs(a) + fabs(b))) {
        G[p][q] = G[q][p] = cd(0, 0);
        return;
    }
    const Cd e = {G[p][q].x / ag, G[p][q].y / ag};  // e^{i phi}
    const double zeta = (b - a) / (2.0 * ag);
    const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                        : (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
#pragma unroll
    for (int r = 0; r < NN; ++r) {
        if (r == p || r == q) continue;
        const Cd grp = G[r][p], grq = G[r][q];
        const Cd eg = conjd(e) * grq;
        const Cd nrp = {c * grp.x - s * eg.x, c * grp.y - s * eg.y};
        const Cd nrq = {s * grp.x + c * eg.x, s * grp.y + c * eg.y};
        G[r][p] = nrp;
        G[p][r] = conjd(nrp);
        G[r][q] = nrq;
        G[q][r] = conjd(nrq);
    }
    G[p][p] = cd(a - t * ag, 0);
    G[q][q] = cd(b + t * ag, 0);
    G[p][q] = G[q][p] = cd(0, 0);
}

template <int NN>
__device__ __forceinline__ void hermitian_eigenvalues(Cd (&G)[3][3], double* ev)
{
    for (int sweep = 0; sweep < 8; ++sweep) {
        double off = 0.0, diag = 0.0;
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            diag += fabs(G[p][p].x);
#pragma unroll
            for (int q = p + 1; q < NN; ++q) off += abs2(G[p][q]);
        }
        if (off <= 1e-30 * diag * diag) break;  // off-diagonal below 1e-15 of the diagonal
#pragma unroll
        for (int p = 0; p < NN; ++p)
#pragma unroll
            for (int q = p + 1; q < NN; ++q) jacobi_rotate<NN>(G, p, q);
    }
#pragma unroll
    for (int p = 0; p < NN; ++p) ev[p] = G[p][p].x;
}

// principal square root of w = a + b i: with r = |w|, t = sqrt((r + |a|) / 2); then
// (t, b / (2 t)) for a >= 0, and (|b| / (2 t), +-t) with the sign of b for a < 0
__device__ __forceinline__ Cd csqrt_d(Cd w)
{
    const double r = sqrt(abs2(w));
    if (r == 0.0) return cd(0, 0);
    const double t = sqrt(0.5 * (r + fabs(w.x)));
    if (w.x >= 0) return cd(t, w.y / (2.0 * t));
    return cd(fabs(w.y) / (2.0 * t), w.y >= 0 ? t : -t);
}

// The n <= 3 roots of z^n + c[n-1] z^{n-1} + ... + c[0].  n = 1, 2 in closed form (Sec. 3.1,
// method 1; the quadratic as q = -(c1 + s sqrt(c1^2 - 4 c0)) / 2 with the sign s that
// avoids cancellation, roots q and c0 / q); n = 3 by the Durand-Kerner (Weierstrass)
// simultaneous iteration z_k <- z_k - p(z_k) / prod_{l != k} (z_k - z_l) from
// (0.4 + 0.9 i)^k, at most 200 sweeps.
__device__ void poly_roots(const Cd* c, int n, Cd* z)
{
    if (n == 1) {
        z[0] = cd(-c[0].x, -c[0].y);
        return;
    }
    if (n == 2) {
        const Cd d = csqrt_d(c[1] * c[1] - cd(4.0 * c[0].x, 4.0 * c[0].y));
        const Cd t1 = c[1] + d, t2 = c[1] - d;
        const Cd t = abs2(t1) >= abs2(t2) ? t1 : t2;
        const Cd q = cd(-0.5 * t.x, -0.5 * t.y);
        z[0] = q;
        z[1] = abs2(q) > 0 ? divd(c[0], q) : cd(0, 0);
        return;
    }
    const Cd w = cd(0.4, 0.9);
    z[0] = cd(1, 0);
    z[1] = w;
    z[2] = w * w;
    for (int it = 0; it < 200; ++it) {
        double moved = 0.0;
        for (int k = 0; k < 3; ++k) {
            Cd pz = cd(1, 0);
            for (int t = 2; t >= 0; --t) pz = pz * z[k] + c[t];
            Cd den = cd(1, 0);
            for (int l = 0; l < 3; ++l)
                if (l != k) den = den * (z[k] - z[l]);
            if (abs2(den) == 0.0) continue;
            const Cd dz = divd(pz, den);
            z[k] = z[k] - dz;
            moved = fmax(moved, abs2(dz) / fmax(1.0, abs2(z[k])));
        }
        if (moved < 1e-30) break;
    }
}

// Positions of n points z (methods 1 and 3): u = ((arg z) N / (2 pi) - j) / B mod L is the
// fractional candidate index; the points take candidates in order of increasing
// |u - round(u)| (lower index on ties), each the nearest q not yet taken: round(u), then
// alternately one step further on u's side and on the other side.  q ascending out.
__device__ void snap_positions(const Cd* z, int n, int j, int B, int L, int32_t N, int* q_out)
{
    double u[3], q0[3], err[3];
    int ord[3];
    for (int t = 0; t < n; ++t) {
        const double f = atan2(z[t].y, z[t].x) * (double)N / (2.0 * 3.14159265358979323846);
        double v = fmod((f - (double)j) / (double)B, (double)L);
        if (v < 0) v += (double)L;
        u[t] = v;
        q0[t] = floor(v + 0.5);
        err[t] = fabs(v - q0[t]);
        ord[t] = t;
    }
    for (int i = 1; i < n; ++i)
        for (int k = i; k > 0 && err[ord[k - 1]] > err[ord[k]]; --k) {
            const int x = ord[k];
            ord[k] = ord[k - 1];
            ord[k - 1] = x;
        }
    int taken[3], nt = 0;
    for (int s = 0; s < n; ++s) {
        const int t = ord[s];
        const int side = u[t] >= q0[t] ? 1 : -1;
        const int base = (int)q0[t];
        int q = ((base % L) + L) % L;
        for (int k = 1; k < 2 * L; ++k) {
            bool used = false;
            for (int e = 0; e < nt; ++e) used |= taken[e] == q;
            if (!used) break;
            const int step = (k + 1) / 2 * ((k & 1) ? side : -side);
            q = (((base + step) % L) + L) % L;
        }
        taken[nt++] = q;
    }
    for (int i = 1; i < nt; ++i)
        for (int k = i; k > 0 && taken[k - 1] > taken[k]; --k) {
            const int x = taken[k];
            taken[k] = taken[k - 1];
            taken[k - 1] = x;
        }
    for (int t = 0; t < nt; ++t) q_out[t] = taken[t];
}

}  // namespace

// DT1a: one thread per (signal, bin position b).  Every singular value of M_{a_m} is at most
// ||M||_F; a bucket whose ||M||_F (in the bins' type) is clearly below the vote's floor
// cannot be voted: its singular values are written as zeros.  The others are listed (in
// the slot's nzl array, count in ctr[kCtrDtList]) for the FP64 work of DT1b and DT3.
template <typename T>
__global__ void dt_screen_kernel(const __grid_constant__ DecodeArgs a)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int B = pd.sumB, am = pd.am;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)a.n_sig * B) return;
    const int sig = (int)(gid / B), b = (int)(gid - (int64_t)sig * B);
    const V* Y = reinterpret_cast<const V*>(a.bins) + (int64_t)sig * pd.y_per_sig;
    T e[5];  // |Y_k|^2 of m_0 .. m_{2 a_m - 2}
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        e[k] = 0;
        if (k < 2 * am - 1) {
            const V y = __ldcg(Y + (int64_t)(k + am) * B + b);
            e[k] = y.x * y.x + y.y * y.y;
        }
    }
    T fro = 0;  // ||M||_F^2 B^2: m_{r+c} appears once per (r, c)
#pragma unroll
    for (int k = 0; k < 5; ++k) fro += (T)min(k + 1, 2 * am - 1 - k) * e[k];
    const double fl = 0.8 * pd.sv_floor * (double)B;
    if ((double)fro < fl * fl) {
        double* out = a.ws.sv + (int64_t)sig * ((int64_t)B * am + 1) + (int64_t)b * am;
        for (int t = 0; t < am; ++t) out[t] = 0.0;
        return;
    }
    int32_t* ctr = a.ws.ctr + (int64_t)sig * a.ctr_stride;
    a.ws.nzl[(int64_t)sig * B + atomicAdd(ctr + kCtrDtList, 1)] = b;
}

// DT1b: the listed buckets' a_m singular values, descending, at sv[b * a_m ..], in FP64.
// Grid (x, signal), threads striding over the signal's list.
template <typename T, int AM>
__global__ void dt_sv_kernel(const __grid_constant__ DecodeArgs a)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const int B = pd.sumB;
    constexpr int am = AM;
    const int sig = blockIdx.y;
    const int n = ldv(a.ws.ctr + (int64_t)sig * a.ctr_stride + kCtrDtList);
    const V* Y = reinterpret_cast<const V*>(a.bins) + (int64_t)sig * pd.y_per_sig;
    const double invB = 1.0 / (double)B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = __ldcg(a.ws.nzl + (int64_t)sig * B + i);
        Cd m[2 * AM - 1];  // m_0 .. m_{2 a_m - 2}
#pragma unroll
        for (int k = 0; k < 2 * AM - 1; ++k) {
            const V y = __ldcg(Y + (int64_t)(k + am) * B + b);
            m[k] = cd((double)y.x * invB, (double)y.y * invB);
        }
        // G = M^H M with M[r][c] = m_{r+c}: G[p][q] = sum_r conj(m_{r+p}) m_{r+q}
        Cd G[3][3];
#pragma unroll
        for (int p = 0; p < AM; ++p)
#pragma unroll
            for (int q = 0; q < AM; ++q) {
                Cd s = cd(0, 0);
#pragma unroll
                for (int r = 0; r < AM; ++r) s = s + conjd(m[r + p]) * m[r + q];
                G[p][q] = s;
            }
        double sv[3];
        hermitian_eigenvalues<AM>(G, sv);
#pragma unroll
        for (int t = 0; t < AM; ++t) sv[t] = sqrt(fmax(sv[t], 0.0));
#pragma unroll
        for (int u = 1; u < AM; ++u)  // descending
#pragma unroll
            for (int k = u; k > 0; --k)
                if (sv[k - 1] < sv[k]) {
                    const double t = sv[k];
                    sv[k] = sv[k - 1];
                    sv[k - 1] = t;
                }
        double* out = a.ws.sv + (int64_t)sig * ((int64_t)B * am + 1) + (int64_t)b * am;
#pragma unroll
        for (int t = 0; t < AM; ++t) out[t] = sv[t];
    }
}

// DT2: one CTA per signal.  theta = the K-th largest singular value among those above the
// floor (the smallest passing one when fewer), stored after the signal's singular values;
// +inf when none passes.  Also sets the signal's counters: every bin resolved (a bucket
// whose Eq. 14 turns out singular takes one back), one round, B identifications.
__global__ void __launch_bounds__(1024) dt_vote_kernel(const __grid_constant__ DecodeArgs a)
{
    const PlanDesc& pd = a.pd;
    const int sig = blockIdx.x;
    const int n = pd.sumB * pd.am;
    double* sv = a.ws.sv + (int64_t)sig * ((int64_t)n + 1);
    const double floor_v = pd.sv_floor;
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_need, s_total;
    if (threadIdx.x == 0) {
        s_total = 0;
        s_prefix = 0;
    }
    __syncthreads();
    // only listed buckets can hold values above the floor (the others were written as zeros)
    const int nl = ldv(a.ws.ctr + (int64_t)sig * a.ctr_stride + kCtrDtList);
    const int32_t* list = a.ws.nzl + (int64_t)sig * pd.sumB;
    const int am = pd.am, nv = nl * am;
    auto value = [&](int i) { return __ldcg(sv + (int64_t)__ldcg(list + i / am) * am + i % am); };
    int cnt = 0;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) cnt += value(i) > floor_v;
    atomicAdd(&s_total, cnt);
    __syncthreads();
    const int total = s_total;
    if (threadIdx.x == 0) s_need = min(pd.K, total);
    unsigned long long mask = 0;
    for (int shift = 56; shift >= 0 && total > 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            const double v = value(i);
            if (!(v > floor_v)) continue;
            const unsigned long long u = (unsigned long long)__double_as_longlong(v);
            if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cum = 0, need = s_need;
            for (int d = 255; d >= 0; --d) {
                if (cum + (int)hist[d] >= need) {
                    s_prefix = prefix | ((unsigned long long)d << shift);
                    s_need = need - cum;
                    break;
                }
                cum += (int)hist[d];
            }
        }
        mask |= 255ull << shift;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sv[n] = total > 0 ? __longlong_as_double((long long)s_prefix) : __longlong_as_double(0x7ff0000000000000ll);
        int32_t* ctr = a.ws.ctr + (int64_t)sig * a.ctr_stride;
        ctr[kCtrResolved] = pd.sumB;
        ctr[kCtrIdents] = pd.sumB;
        ctr[kCtrRounds] = 1;
    }
}

template <typename T>
__device__ __noinline__ void dt_solve_bucket(const DecodeArgs& a, int sig, int b);

// DT3: grid (x, signal); each warp takes listed buckets of its signal in turn; buckets
// without a vote are skipped.
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) dt_solve_kernel(const __grid_constant__ DecodeArgs a)
{
    const int sig = blockIdx.y;
    const int n = ldv(a.ws.ctr + (int64_t)sig * a.ctr_stride + kCtrDtList);
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb)
        dt_solve_bucket<T>(a, sig, __ldcg(a.ws.nzl + (int64_t)sig * a.pd.sumB + i));
}

// Eigen-decomposition of the Hermitian n x n matrix G (n <= 4, row stride 4) by cyclic
// complex Jacobi rotations, as in jacobi_rotate (the phase e^{-i phi} on coordinate q, then
// the real rotation), with the rotations accumulated into V (V <- V J): G ends diagonal with
// the eigenvalues, and column k of V is the eigenvector of G[k][k].  G and V live in the
// warp's shared scratch, which keeps the solve kernel's stack frame small.
__device__ void hermitian_eigen_vectors(Cd* G, Cd* V, int n)
{
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) V[r * 4 + c] = cd(r == c ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += fabs(G[p * 4 + p].x);
            for (int q = p + 1; q < n; ++q) off += abs2(G[p * 4 + q]);
        }
        if (off <= 1e-30 * diag * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double ag = sqrt(abs2(G[p * 4 + q]));
                const double ga = G[p * 4 + p].x, gb = G[q * 4 + q].x;
                if (ag <= 1e-300 || ag <= 1e-18 * (fabs(ga) + fabs(gb))) {
                    G[p * 4 + q] = G[q * 4 + p] = cd(0, 0);
                    continue;
                }
                const Cd e = {G[p * 4 + q].x / ag, G[p * 4 + q].y / ag};
                const double zeta = (gb - ga) / (2.0 * ag);
                const double t = fabs(zeta) > 1e150
                                     ? 0.5 / zeta
                                     : (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int r = 0; r < n; ++r) {
                    if (r == p || r == q) continue;
                    const Cd grp = G[r * 4 + p], eg = conjd(e) * G[r * 4 + q];
                    const Cd nrp = {c * grp.x - s * eg.x, c * grp.y - s * eg.y};
                    const Cd nrq = {s * grp.x + c * eg.x, s * grp.y + c * eg.y};
                    G[r * 4 + p] = nrp;
                    G[p * 4 + r] = conjd(nrp);
                    G[r * 4 + q] = nrq;
                    G[q * 4 + r] = conjd(nrq);
                }
                G[p * 4 + p] = cd(ga - t * ag, 0);
                G[q * 4 + q] = cd(gb + t * ag, 0);
                G[p * 4 + q] = G[q * 4 + p] = cd(0, 0);
                for (int r = 0; r < n; ++r) {
                    const Cd vp = V[r * 4 + p], vq = conjd(e) * V[r * 4 + q];
                    V[r * 4 + p] = cd(c * vp.x - s * vq.x, c * vp.y - s * vq.y);
                    V[r * 4 + q] = cd(s * vp.x + c * vq.x, s * vp.y + c * vq.y);
                }
            }
    }
}

// Step 2, method 3 as sFFT-DT3.0 runs it (Sec. 4.1) for one bucket, by one lane: Y[r][c] =
// m_{r-c} ((a + 1) x (a + 1), Eq. 15); its right singular vectors are the eigenvectors of
// Y^H Y; V_s = those of the a largest eigenvalues; with V_1 = V_s without its last row and
// V_2 = V_s without its first, the eigenvalues of G = V_1^{-1} V_2 (the roots of its
// characteristic polynomial) are the z_j (Y = U diag(p) U^H with U[r][j] = z_j^r, so V_s
// spans U's columns).  A, rhs: scratch (a^2 and a).
template <typename T>
__device__ void pencil_points(const typename C2<T>::t* Y, int b, int B, int am, int na,
                              double invB, Cd* A, Cd* rhs, Cd* W, Cd* z)
{
    // W (shared, kPencilWords entries): m_k at W[k + na] (k = -na .. na), H = Y^H Y at
    // W[8 ..] and its eigenvectors at W[24 ..] (row stride 4), G = V_1^{-1} V_2 at W[40 ..]
    // (row stride 3, up to W[48] for na = 3)
    Cd* m = W;
    Cd* H = W + 8;
    Cd* V = W + 24;
    Cd* G = W + 40;
    for (int k = -na; k <= na; ++k) {
        const typename C2<T>::t y = __ldcg(Y + (int64_t)(k + am) * B + b);
        m[k + na] = cd((double)y.x * invB, (double)y.y * invB);
    }
    const int n = na + 1;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            Cd h = cd(0, 0);
            for (int k = 0; k < n; ++k) h = h + conjd(m[k - r + na]) * m[k - c + na];
            H[r * 4 + c] = h;
        }
    hermitian_eigen_vectors(H, V, n);
    int idx[4] = {0, 1, 2, 3};
    for (int i = 1; i < n; ++i)
        for (int k = i; k > 0 && H[idx[k - 1] * 5].x < H[idx[k] * 5].x; --k) {
            const int x = idx[k];
            idx[k] = idx[k - 1];
            idx[k - 1] = x;
        }
    for (int d = 0; d < na; ++d) {
        for (int u = 0; u < na; ++u) {
            for (int v = 0; v < na; ++v) A[u * na + v] = V[u * 4 + idx[v]];  // V_1
            rhs[u] = V[(u + 1) * 4 + idx[d]];                                // V_2, column d
        }
        const bool ok = solve_lane(A, rhs, na);
        for (int u = 0; u < na; ++u) G[u * 3 + d] = ok ? rhs[u] : cd(0, 0);
    }
    Cd c[3];
    if (na == 1) {
        c[0] = cd(-G[0].x, -G[0].y);
    } else if (na == 2) {
        const Cd tr = G[0] + G[4];
        c[1] = cd(-tr.x, -tr.y);
        c[0] = G[0] * G[4] - G[1] * G[3];
    } else {
        const Cd tr = G[0] + G[4] + G[8];
        c[2] = cd(-tr.x, -tr.y);
        c[1] = (G[0] * G[4] - G[1] * G[3]) + (G[0] * G[8] - G[2] * G[6]) +
               (G[4] * G[8] - G[5] * G[7]);
        const Cd det = G[0] * (G[4] * G[8] - G[5] * G[7]) -
                       G[1] * (G[3] * G[8] - G[5] * G[6]) +
                       G[2] * (G[3] * G[7] - G[4] * G[6]);
        c[0] = cd(-det.x, -det.y);
    }
    poly_roots(c, na, z);
}

// Steps 2-3 of one voted bucket by one warp (every lane calls with the same b).
template <typename T>
__device__ __noinline__ void dt_solve_bucket(const DecodeArgs& a, int sig, int b)
{
    using V = typename C2<T>::t;
    const PlanDesc& pd = a.pd;
    const StageDesc& st = pd.st[0];
    const int B = pd.sumB, am = pd.am, L = st.L;
    const int32_t N = pd.N;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const double* sv = a.ws.sv + (int64_t)sig * ((int64_t)B * am + 1);
    const double theta = __ldcg(sv + (int64_t)B * am);
    int na = 0;
    for (int t = 0; t < am; ++t) {
        const double v = __ldcg(sv + (int64_t)b * am + t);
        na += (v >= theta && v > pd.sv_floor) ? 1 : 0;
    }
    if (na == 0) return;

    __shared__ Cd s_A[kSolveThreads / 32][kMaxFit * kMaxFit];
    __shared__ Cd s_b[kSolveThreads / 32][kMaxFit];
    __shared__ int s_ok[kSolveThreads / 32];
    Cd* A = s_A[wib];
    Cd* rhs = s_b[wib];
    int32_t* ctr = a.ws.ctr + (int64_t)sig * a.ctr_stride;
    const V* Y = reinterpret_cast<const V*>(a.bins) + (int64_t)sig * pd.y_per_sig;
    const double invB = 1.0 / (double)B;
    const int j = __ldg(a.pbin + b);

    // moments m_0 .. m_{2a-1}, lane k loads m_k
    Cd mk = cd(0, 0);
    if (lane < 2 * na) {
        const V y = __ldcg(Y + (int64_t)(lane + am) * B + b);
        mk = cd((double)y.x * invB, (double)y.y * invB);
    }
    const int method = a.dt_method;  // Step 2: 1 polynomial roots, 2 enumeration, 3 pencil
    Cd c[3] = {cd(0, 0), cd(0, 0), cd(0, 0)};
    if (method != 3) {
        // Eq. 14: M_a C = M_s, M_a[r][c] = m_{r+c}, M_s[r] = -m_{a+r}
        for (int idx = 0; idx < na * na; ++idx) {
            const int r = idx / na, cc = idx - r * na;
            const double x = __shfl_sync(0xffffffffu, mk.x, r + cc), y = __shfl_sync(0xffffffffu, mk.y, r + cc);
            if (lane == 0) A[idx] = cd(x, y);
        }
        for (int r = 0; r < na; ++r) {
            const double x = __shfl_sync(0xffffffffu, mk.x, na + r), y = __shfl_sync(0xffffffffu, mk.y, na + r);
            if (lane == 0) rhs[r] = cd(-x, -y);
        }
        __syncwarp();
        if (lane == 0) s_ok[wib] = solve_lane(A, rhs, na) ? 1 : 0;
        __syncwarp();
        if (!s_ok[wib]) {
            if (lane == 0) atomicSub(ctr + kCtrResolved, 1);
            return;
        }
        for (int t = 0; t < 3; ++t) c[t] = t < na ? rhs[t] : cd(0, 0);
        __syncwarp();
    }

    int pos_q[3];
    if (method == 1 || method == 3) {
        // methods 1 and 3: lane 0 finds the points z_j and snaps them to candidates
        __shared__ int s_pos[kSolveThreads / 32][3];
        __shared__ Cd s_w[kSolveThreads / 32][kPencilWords];
        if (lane == 0) {
            Cd z[3];
            if (method == 1)
                poly_roots(c, na, z);
            else
                pencil_points<T>(Y, b, B, am, na, invB, A, rhs, s_w[wib], z);
            snap_positions(z, na, j, B, L, N, s_pos[wib]);
        }
        __syncwarp();
        for (int t = 0; t < na; ++t) pos_q[t] = s_pos[wib][t];
        __syncwarp();
    } else {
        // Step 2 (enumeration): candidates q = lane, lane + 32, ...; z = e^{2 pi i (j + q B) / N}
        // by a rotation e^{2 pi i 32 / L} per step from z_lane
        double bv[3];
        int bq[3];
        for (int t = 0; t < 3; ++t) {
            bv[t] = 1e300;
            bq[t] = 0x7fffffff;
        }
        {
            Cd z = root_n<T>(pd, a.roots, ((int64_t)j + (int64_t)lane * B) % N);
            const Cd w = root_n<T>(pd, a.roots, (32 * (int64_t)B) % N);  // e^{2 pi i 32 / L}
            for (int q = lane; q < L; q += 32) {
                if (((q - lane) & 1023) == 0 && q != lane) z = root_n<T>(pd, a.roots, ((int64_t)j + (int64_t)q * B) % N);
                Cd pz = cd(1, 0);
                for (int t = na - 1; t >= 0; --t) pz = pz * z + c[t];
                const double v = abs2(pz);
                // keep the na smallest (v, q), lower q first on ties; q only grows
                int k = na;
                while (k > 0 && v < bv[k - 1]) --k;
                if (k < na) {
                    for (int t = na - 1; t > k; --t) {
                        bv[t] = bv[t - 1];
                        bq[t] = bq[t - 1];
                    }
                    bv[k] = v;
                    bq[k] = q;
                }
                z = z * w;
            }
        }
        // merge across lanes: na rounds of a warp argmin over (v, q)
        for (int t = 0; t < na; ++t) {
            double v = bv[0];
            int q = bq[0];
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int oq = __shfl_xor_sync(0xffffffffu, q, o);
                if (ov < v || (ov == v && oq < q)) {
                    v = ov;
                    q = oq;
                }
            }
            pos_q[t] = q;
            if (bq[0] == q) {  // the owner pops its head
                for (int u = 0; u + 1 < 3; ++u) {
                    bv[u] = bv[u + 1];
                    bq[u] = bq[u + 1];
                }
                bv[2] = 1e300;
                bq[2] = 0x7fffffff;
            }
        }
        // positions ascending
        for (int i = 1; i < na; ++i)
            for (int k = i; k > 0 && pos_q[k - 1] > pos_q[k]; --k) {
                const int t = pos_q[k];
                pos_q[k] = pos_q[k - 1];
                pos_q[k - 1] = t;
            }
    }

    // Step 3: subspace pursuit.  Dictionary: for each position f, the atoms f, f + B, f - B
    // (mod N) in that order, duplicates dropped.
    int64_t dic[kMaxAtoms];
    int nd = 0;
    for (int t = 0; t < na; ++t) {
        const int64_t f = (int64_t)j + (int64_t)pos_q[t] * B;
        const int64_t cand[3] = {f, (f + B) % N, (f - B + N) % N};
        for (int s = 0; s < 3; ++s) {
            bool dup = false;
            for (int u = 0; u < nd; ++u) dup |= dic[u] == cand[s];
            if (!dup) dic[nd++] = cand[s];
        }
    }
    const int P = pd.R - 3 * am;
    const bool mine = lane < P;
    Cd y = cd(0, 0);
    Cd phi[kMaxAtoms];
    if (mine) {
        const V v = __ldcg(Y + (int64_t)(3 * am + lane) * B + b);
        y = cd((double)v.x * invB, (double)v.y * invB);
    }
    const int64_t tau = mine ? (int64_t)st.tau[3 * am + lane] : 0;
    for (int d = 0; d < kMaxAtoms; ++d) phi[d] = (mine && d < nd) ? root_n<T>(pd, a.roots, (dic[d] * tau) % N) : cd(0, 0);

    // least squares on the atoms sup[0..ns) by the normal equations; returns the residual
    // energy, the coefficients in p[], and this lane's residual in *r
    auto fit = [&](const int* sup, int ns, Cd* p, Cd* r, bool* ok) -> double {
        for (int u = 0; u < ns; ++u) {
            Cd pu = cd(0, 0), hu = cd(0, 0);
            for (int d = 0; d < kMaxAtoms; ++d)
                if (d == sup[u]) pu = phi[d];
            hu = warp_sum(conjd(pu) * y);
            if (lane == 0) rhs[u] = hu;
            for (int v = 0; v < ns; ++v) {
                Cd pv = cd(0, 0);
                for (int d = 0; d < kMaxAtoms; ++d)
                    if (d == sup[v]) pv = phi[d];
                const Cd g = warp_sum(conjd(pu) * pv);
                if (lane == 0) A[u * ns + v] = g;
            }
        }
        __syncwarp();
        if (lane == 0) s_ok[wib] = solve_lane(A, rhs, ns) ? 1 : 0;
        __syncwarp();
        *ok = s_ok[wib] != 0;
        for (int u = 0; u < ns; ++u) p[u] = rhs[u];
        __syncwarp();
        Cd res = y;
        for (int u = 0; u < ns; ++u) {
            Cd pu = cd(0, 0);
            for (int d = 0; d < kMaxAtoms; ++d)
                if (d == sup[u]) pu = phi[d];
            res = res - pu * p[u];
        }
        if (!mine) res = cd(0, 0);
        *r = res;
        return warp_sum(abs2(res));
    };

    int S[3];
    for (int t = 0; t < na; ++t) {
        const int64_t f = (int64_t)j + (int64_t)pos_q[t] * B;
        for (int d = 0; d < nd; ++d)
            if (dic[d] == f) S[t] = d;
    }
    Cd p[kMaxFit], r;
    bool ok = true;
    double res = fit(S, na, p, &r, &ok);
    for (int it = 0; it < 8 && ok; ++it) {
        if (res <= pd.sp_tol2) break;
        // the na atoms outside S most correlated with the residual (lower index on ties)
        double corr[kMaxAtoms];
        for (int d = 0; d < kMaxAtoms; ++d) corr[d] = d < nd ? abs2(warp_sum(conjd(phi[d]) * r)) : -1.0;
        int Tu[kMaxFit], nt = 0;
        for (int t = 0; t < na; ++t) Tu[nt++] = S[t];
        for (int e = 0; e < na; ++e) {
            int bestd = -1;
            for (int d = 0; d < nd; ++d) {
                bool used = false;
                for (int u = 0; u < nt; ++u) used |= Tu[u] == d;
                if (!used && (bestd < 0 || corr[d] > corr[bestd])) bestd = d;
            }
            if (bestd < 0) break;
            Tu[nt++] = bestd;
        }
        Cd pT[kMaxFit], rT;
        bool okT = true;
        fit(Tu, nt, pT, &rT, &okT);
        if (!okT) break;
        // keep the na largest |p| of the union (lower position on ties), in union order
        bool keep[kMaxFit] = {false, false, false, false, false, false};
        for (int e = 0; e < na; ++e) {
            int bi = -1;
            for (int u = 0; u < nt; ++u)
                if (!keep[u] && (bi < 0 || abs2(pT[u]) > abs2(pT[bi]))) bi = u;
            keep[bi] = true;
        }
        int S2[3], n2 = 0;
        for (int u = 0; u < nt; ++u)
            if (keep[u]) S2[n2++] = Tu[u];
        Cd p2[kMaxFit], r2;
        bool ok2 = true;
        const double res2 = fit(S2, na, p2, &r2, &ok2);
        if (!ok2 || res2 >= res) break;
        for (int t = 0; t < na; ++t) {
            S[t] = S2[t];
            p[t] = p2[t];
        }
        res = res2;
        r = r2;
    }
    if (!ok) {
        if (lane == 0) atomicSub(ctr + kCtrResolved, 1);
        return;
    }
    if (lane == 0) {
        const int k0 = atomicAdd(ctr + kCtrRec, na);
        int64_t* rf = a.ws.rec_f + (int64_t)sig * pd.sumB;
        V* rv = reinterpret_cast<V*>(a.ws.rec_v) + (int64_t)sig * pd.sumB;
        for (int t = 0; t < na; ++t) {
            if (k0 + t >= pd.sumB) {  // more votes than buckets: cannot store
                atomicSub(ctr + kCtrResolved, 1);
                break;
            }
            rf[k0 + t] = dic[S[t]];
            rv[k0 + t] = V{(T)p[t].x, (T)p[t].y};
        }
    }
}

cudaError_t launch_oneshot(const DecodeArgs& a, int precision, cudaStream_t st)
{
    if (a.n_sig == 0) return cudaSuccess;
    const int64_t n = (int64_t)a.n_sig * a.pd.sumB;
    const unsigned g1 = (unsigned)((n + 255) / 256);
    // listed buckets are a small share: CTAs of 64 threads, about 4864 of them in all (32 per
    // SM), split over the signals
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)a.pd.sumB + 63) / 64,
                                                                         4864 / a.n_sig + 1));
    const dim3 g2(gx, (unsigned)a.n_sig);
    auto sv = [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        dt_screen_kernel<T><<<g1, 256, 0, st>>>(a);
        if (a.pd.am == 1)
            dt_sv_kernel<T, 1><<<g2, 64, 0, st>>>(a);
        else if (a.pd.am == 2)
            dt_sv_kernel<T, 2><<<g2, 64, 0, st>>>(a);
        else
            dt_sv_kernel<T, 3><<<g2, 64, 0, st>>>(a);
    };
    if (precision == 1)
        sv((float*)nullptr);
    else
        sv((double*)nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dt_vote_kernel<<<(unsigned)a.n_sig, 1024, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // warps of 4864 in all (32 per SM), split over the signals
    const dim3 g3((unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)a.pd.sumB + 7) / 8,
                                                                   4864 / 8 / a.n_sig + 1)),
                  (unsigned)a.n_sig);
    if (precision == 1)
        dt_solve_kernel<float><<<g3, kSolveThreads, 0, st>>>(a);
    else
        dt_solve_kernel<double><<<g3, kSolveThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sfft
