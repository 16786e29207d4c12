/*
 * sfft_oracle.c -- plain, slow FP64 CPU oracle for the aliasing-filter sparse FFT
 * (FFAST / R-FFAST peeling), written from Li, Jiang, Chen, "On Performance of Sparse
 * Fast Fourier Transform Algorithms Using the Aliasing Filter" (arXiv 2011.05749).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is checked
 * against.  It shares no code, header, table or constant with the CUDA path.  Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline leg may build,
 * load or call it; the library never does.
 *
 * Conventions (one convention for the whole project):
 *   - time signal x_n = sum_k xhat_k exp(+2 pi i k n / N), i.e. xhat is the paper's
 *     normalised spectrum of Eq. 2 (xhat = (1/N) sum_n x_n omega_N^{kn}, omega_N = e^{-2 pi i/N}).
 *   - stage d has subsampling factor L_d = f[d] and B_d = N / L_d buckets (Eq. 5).
 *   - delay tau is an advance: the sample is x[(m L_d + tau) mod N], 0 <= tau < N (Eq. 3-4
 *     with the opposite sign; the paper's delay is -tau).
 *   - bins are UNNORMALISED B-point DFTs of the delayed subsample (Eq. 6 and Eq. 19):
 *       Y_{d,r}[j] = sum_{m<B} x[(m L + tau_r) mod N] e^{-2 pi i j m / B}
 *                  = B * sum_{k = j mod B} xhat_k e^{+2 pi i k tau_r / N}.
 *
 * Every function below states the passage of the paper it follows.  Where the paper is
 * silent the readings are:
 *   - thresholds (Sec. 3.2, subproblem 1, T0/T1 unspecified):
 *       T0_d = R (c0 B_d sigma^2 + (eta B_d a_min)^2),  T1_d = R (c1 B_d sigma^2 + (eta B_d a_min)^2)
 *     with sigma^2 the noise variance per time sample;
 *   - locate: ARG reads the phase of Y(tau=1) conj(Y(tau=0)) (Sec. 3.2, subproblem 2, exactly
 *     sparse case) and snaps it to the candidate set {j, j+B, ..., j+(L-1)B}; ML picks the
 *     candidate of that set whose delay phasors best correlate with the bin vector; KAY
 *     (general sparse case, Eq. 21-22) reads one bit of f / N per iteration of structured
 *     delays r_c + t 2^c and takes the candidate nearest the interval the bits leave;
 *   - value: least squares over all R delays (the LSM of the general sparse case);
 *   - a frequency that is a singleton in several stages in one round is taken from the
 *     lowest stage; a frequency already recovered in an earlier round is not taken again;
 *   - peeling stops when a round leaves no bin to re-examine, or after max_rounds rounds.
 *
 * Parity status: every function here is pinned by the CPU tests (closed forms, the paper's
 * N = 20 worked example, brute force, numpy's FFT) except the noisy-input decoding path,
 * whose decisions have no printed values to pin against ("parity unpinned" beyond
 * self-consistency and recovery of the generator's truth).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

#define OR_ZERO 1
#define OR_SINGLE 2
#define OR_MULTI 3

static const double OR_TWO_PI = 6.283185307179586476925286766559;

/* e^{+2 pi i t / n} for an integer residue 0 <= t < n. */
static cplx unit_phasor(int64_t t, int64_t n)
{
    double a = OR_TWO_PI * (double)t / (double)n;
    return CMPLX(cos(a), sin(a));
}

static int64_t pos_mod(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------------------- */
/* Eq. 1-2: dense DFT, xhat_k = (1/N) sum_n x_n e^{-2 pi i k n / N}.  O(N^2); tiny N only. */
int oracle_dense_dft(int64_t N, const cplx* x, cplx* xhat)
{
    if (N <= 0 || !x || !xhat) return OR_EINVAL;
    for (int64_t k = 0; k < N; ++k) {
        cplx acc = 0;
        for (int64_t n = 0; n < N; ++n) {
            int64_t t = (int64_t)(((__int128)k * n) % N);
            acc += x[n] * conj(unit_phasor(t, N));
        }
        xhat[k] = acc / (double)N;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Bucketization, Eq. 3-6 and Eq. 19: for every stage d and delay r, subsample the
 * advanced signal at stride L_d (Eq. 5) and take a naive B_d-point DFT of it (no FFT).     */

typedef struct {
    const cplx* y;  /* the delayed subsample y[m] = x[(m L + tau) mod N], m < B (Eq. 5) */
    int64_t B;
    const cplx* w;  /* w[t] = e^{-2 pi i t / B} */
    cplx* Y;        /* B outputs */
    int64_t j0, j1; /* output range of this worker */
} bucket_job;

/* Y[j] = sum_m y[m] e^{-2 pi i j m / B}, the twiddle indexed by (j m) mod B */
static void* bucket_worker(void* arg)
{
    bucket_job* jb = (bucket_job*)arg;
    for (int64_t j = jb->j0; j < jb->j1; ++j) {
        cplx acc = 0;
        int64_t t = 0; /* (j * m) mod B */
        for (int64_t m = 0; m < jb->B; ++m) {
            acc += jb->y[m] * jb->w[t];
            t += j;
            if (t >= jb->B) t -= jb->B;
        }
        jb->Y[j] = acc;
    }
    return NULL;
}

/* Y layout: stage-major, then delay, then bin j in natural order:
 *   Y[off_d + r * B_d + j],  off_d = R * sum_{d' < d} B_{d'}.
 * delays[d * R + r] = tau_{d,r}.  n_threads <= 0 means 1.                                 */
int oracle_bucketize(int64_t N, int32_t n_stages, const int64_t* f, int32_t R,
                     const int64_t* delays, const cplx* x, cplx* Y, int32_t n_threads)
{
    if (N <= 0 || n_stages <= 0 || R <= 0 || !f || !delays || !x || !Y) return OR_EINVAL;
    if (n_threads <= 0) n_threads = 1;
    int64_t off = 0;
    for (int32_t d = 0; d < n_stages; ++d) {
        int64_t L = f[d];
        if (L <= 0 || N % L != 0) return OR_EINVAL;
        int64_t B = N / L;
        cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)B);
        cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)B);
        if (!w || !y) { free(w); free(y); return OR_ENOMEM; }
        for (int64_t t = 0; t < B; ++t) w[t] = conj(unit_phasor(t, B));
        for (int32_t r = 0; r < R; ++r) {
            int64_t tau = delays[(int64_t)d * R + r];
            if (tau < 0 || tau >= N) { free(w); free(y); return OR_EINVAL; }
            for (int64_t m = 0; m < B; ++m) y[m] = x[(int64_t)(((__int128)m * L + tau) % N)];
            cplx* Yd = Y + off + (int64_t)r * B;
            int nt = n_threads;
            if ((int64_t)nt > B) nt = (int)B;
            pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
            bucket_job* jobs = (bucket_job*)malloc(sizeof(bucket_job) * (size_t)nt);
            if (!th || !jobs) { free(th); free(jobs); free(w); free(y); return OR_ENOMEM; }
            for (int i = 0; i < nt; ++i) {
                jobs[i].y = y; jobs[i].B = B;
                jobs[i].w = w; jobs[i].Y = Yd;
                jobs[i].j0 = B * i / nt; jobs[i].j1 = B * (i + 1) / nt;
            }
            char* spawned = (char*)calloc((size_t)nt, 1);
            for (int i = 1; i < nt; ++i) {
                if (spawned && pthread_create(&th[i], NULL, bucket_worker, &jobs[i]) == 0)
                    spawned[i] = 1;
                else
                    bucket_worker(&jobs[i]); /* no thread: run this share inline */
            }
            bucket_worker(&jobs[0]);
            for (int i = 1; i < nt; ++i)
                if (spawned && spawned[i]) pthread_join(th[i], NULL);
            free(spawned); free(th); free(jobs);
        }
        off += (int64_t)R * B;
        free(w);
        free(y);
    }
    return OR_OK;
}

/* One bin Y_{d,r}[j] computed directly as a dot product (the same definition, one output):
 * used to check sampled outputs at sizes where the full bucketization is too slow.         */
int oracle_bin(int64_t N, int64_t L, int64_t tau, int64_t j, const cplx* x, cplx* out)
{
    if (N <= 0 || L <= 0 || N % L != 0 || !x || !out) return OR_EINVAL;
    int64_t B = N / L;
    cplx acc = 0;
    for (int64_t m = 0; m < B; ++m) {
        int64_t n = (int64_t)(((__int128)m * L + tau) % N);
        int64_t t = (int64_t)(((__int128)j * m) % B);
        acc += x[n] * conj(unit_phasor(t, B));
    }
    *out = acc;
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Peeling decoder: Sec. 3.2 (Eq. 19-20, subproblems 1-3, genie-assisted peeling in
 * parallel rounds) and Sec. 4.2 (FFAST delays {0,1,2}; R-FFAST random delays).           */

typedef struct {
    double noise_var; /* sigma^2 per time sample; 0 = exactly sparse */
    double a_min;     /* smallest significant |xhat| */
    double eta;       /* relative numerical floor of the thresholds */
    double c0, c1;    /* zero-ton / single-ton threshold multipliers */
    int32_t locate;   /* 0 = ARG (needs delays 0 and 1 in every stage), 1 = ML, 2 = KAY */
    int32_t max_rounds;
    int32_t kay_m;    /* KAY: delays per iteration m (slots c m + t hold r_c + t 2^c) */
    int32_t noise_auto; /* 1: estimate sigma^2 from the median bin energy (noise_var unused) */
} oracle_opts;

typedef struct {
    int32_t status;          /* 0 all bins resolved, 1 bins left unresolved */
    int32_t rounds;          /* classification rounds run */
    int32_t n_recovered;     /* frequencies recovered before truncation to K */
    int32_t n_out;           /* entries written to out_idx/out_val */
    int64_t idents;          /* bins classified, summed over rounds */
    int64_t unresolved;      /* bins never resolved */
    double noise_var;        /* sigma^2 the thresholds used (estimated with noise_auto) */
} oracle_stats;

/* per round counters, filled when the caller passes arrays of max_rounds entries */
typedef struct {
    int64_t* idents;
    int64_t* n_zero;
    int64_t* n_single;
    int64_t* n_multi;
    int64_t* n_accepted;
} oracle_round_log;

/* e^{+2 pi i (f tau mod N) / N}: the phasor a delay imprints on frequency f (Eq. 4, 19),
 * from an exact integer product.                                                          */
static cplx delay_phasor(int64_t f, int64_t tau, int64_t N)
{
    int64_t t = (int64_t)(((__int128)f * tau) % N);
    return unit_phasor(t, N);
}

/* Least-squares single-tone fit of the bin vector y (R entries) at frequency f:
 * v = (1/(R B)) sum_r y_r conj(a_r(f)), residual rho = sum_r |y_r - B v a_r(f)|^2.        */
static void fit_tone(const cplx* y, int32_t R, const int64_t* tau, int64_t f, int64_t N,
                     int64_t B, cplx* v_out, double* rho_out)
{
    cplx c = 0;
    for (int32_t r = 0; r < R; ++r) c += y[r] * conj(delay_phasor(f, tau[r], N));
    cplx v = c / ((double)R * (double)B);
    double rho = 0;
    for (int32_t r = 0; r < R; ++r) {
        cplx e = y[r] - (double)B * v * delay_phasor(f, tau[r], N);
        rho += creal(e) * creal(e) + cimag(e) * cimag(e);
    }
    *v_out = v;
    *rho_out = rho;
}

/* Median of the Gamma(R, 1) distribution (the sum of R unit exponentials): the x with
 * P(R, x) = 1 - e^{-x} sum_{k<R} x^k / k! = 1/2, by bisection.                            */
double oracle_gamma_median(int32_t R)
{
    double lo = 0.0, hi = 4.0 * R + 10.0;
    for (int it = 0; it < 200; ++it) {
        double x = 0.5 * (lo + hi), term = 1.0, sum = 1.0;
        for (int32_t k = 1; k < R; ++k) {
            term *= x / k;
            sum += term;
        }
        double cdf = 1.0 - exp(-x) * sum;
        if (cdf < 0.5) lo = x; else hi = x;
    }
    return 0.5 * (lo + hi);
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Noise variance per time sample from the bins (no counterpart in the paper: the
 * thresholds of Sec. 3.2 assume sigma^2 known): a bin holding only noise has R delays of
 * CN(0, B sigma^2) values, so E / B = sum_r |Y_r|^2 / B is sigma^2 times a Gamma(R, 1)
 * variable; with K much below sum B almost every bin is such, and sigma^2 is the lower
 * median of E / B over all bins divided by the Gamma(R, 1) median.                       */
double oracle_noise_estimate(int64_t N, int32_t n_stages, const int64_t* f, int32_t R,
                             const cplx* Y)
{
    int64_t nb = 0;
    for (int32_t d = 0; d < n_stages; ++d) nb += N / f[d];
    double* e = (double*)malloc(sizeof(double) * (size_t)nb);
    if (!e) return -1.0;
    int64_t i = 0, off = 0;
    for (int32_t d = 0; d < n_stages; ++d) {
        int64_t B = N / f[d];
        for (int64_t j = 0; j < B; ++j) {
            double E = 0;
            for (int32_t r = 0; r < R; ++r) {
                cplx y = Y[off + (int64_t)r * B + j];
                E += creal(y) * creal(y) + cimag(y) * cimag(y);
            }
            e[i++] = E / (double)B;
        }
        off += (int64_t)R * B;
    }
    qsort(e, (size_t)nb, sizeof(double), cmp_double);
    double med = e[(nb - 1) / 2];
    free(e);
    return med / oracle_gamma_median(R);
}

/* Kay's weights of Eq. 22 for m delays per iteration: w_t, t = 0 .. m-2 */
static double kay_weight(int32_t m, int32_t t)
{
    double u = (2.0 * t - m + 2.0) / (2.0 * m);
    return 3.0 * m / (2.0 * ((double)m * m - 1.0)) * (1.0 - 4.0 * u * u);
}

/* R-FFAST single-ton locate of the general sparse case (Sec. 3.2, subproblem 2): the delay
 * slots form C = R / m iterations, slot c m + t holding r_c + t 2^c.  Iteration c gives
 * the phase differences Delta_t = arg(y_{c,t+1} conj(y_{c,t})), t < m - 1, each about
 * 2 pi 2^c f / N (mod 2 pi); Eq. 21 averages them with the weights of Eq. 22 into an
 * estimate of the angle of omega^{2^c f}, omega = e^{2 pi i / N}.  The binary search reads
 * one bit per iteration: the angle in [0, pi) keeps the lower half of the current range of
 * f / N, otherwise the upper half, so after C iterations f / N lies in
 * [k / 2^C, (k + 1) / 2^C).  The candidate j + q B of the bin nearest the centre of that
 * interval (around the circle of N frequencies) is the location.
 * Reading where the paper is silent: when L divides 2^c, every candidate of the bin gives
 * the same 2^c f / N mod 1 = 2^c j / N mod 1, so the phase of that iteration carries no
 * information and can sit exactly on the decision boundary (j = 0); its bit is then taken
 * from j by integer arithmetic, floor(2^{c+1} j / N) mod 2.                               */
static int64_t locate_kay(const cplx* yv, int32_t R, int32_t m, int64_t j, int64_t B, int64_t L,
                          int64_t N)
{
    int32_t C = R / m;
    int64_t k = 0;
    for (int32_t c = 0; c < C; ++c) {
        if ((((int64_t)1 << c) % L) == 0) {
            k = 2 * k + (((j << (c + 1)) / N) & 1);
            continue;
        }
        double th = 0.0;
        for (int32_t t = 0; t + 1 < m; ++t)
            th += kay_weight(m, t) * carg(yv[c * m + t + 1] * conj(yv[c * m + t]));
        double ph = fmod(th, OR_TWO_PI);
        if (ph < 0) ph += OR_TWO_PI;
        k = 2 * k + (ph >= OR_TWO_PI / 2 ? 1 : 0);
    }
    double target = ((double)k + 0.5) * (double)N / ldexp(1.0, C);
    double qd = floor((target - (double)j) / (double)B + 0.5);
    return j + pos_mod((int64_t)qd, L) * B;
}

typedef struct { int64_t f; cplx v; } rec_entry;

static int cmp_rec_by_f(const void* a, const void* b)
{
    int64_t fa = ((const rec_entry*)a)->f, fb = ((const rec_entry*)b)->f;
    return (fa > fb) - (fa < fb);
}

/* larger |v| first; equal magnitudes: lower f first (the K largest, Sec. 2.1) */
static int cmp_rec_by_mag(const void* a, const void* b)
{
    const rec_entry* x = (const rec_entry*)a;
    const rec_entry* y = (const rec_entry*)b;
    double mx = cabs(x->v), my = cabs(y->v);
    if (mx > my) return -1;
    if (mx < my) return 1;
    return (x->f > y->f) - (x->f < y->f);
}

/* Decode bins Y (layout of oracle_bucketize, modified in place) into at most K
 * (frequency, value) pairs sorted by frequency.  rec_f / rec_v (capacity sum_d B_d, may be
 * NULL) receive every recovered pair in acceptance order.                                 */
int oracle_decode(int64_t N, int32_t n_stages, const int64_t* f, int32_t R, const int64_t* delays,
                  cplx* Y, int32_t K, const oracle_opts* opt, int64_t* out_idx, cplx* out_val,
                  int64_t* rec_f, cplx* rec_v, oracle_stats* st, const oracle_round_log* log)
{
    if (N <= 0 || n_stages <= 0 || R <= 0 || K < 0 || !f || !delays || !Y || !opt || !st)
        return OR_EINVAL;
    int32_t D = n_stages;
    int64_t* B = (int64_t*)calloc((size_t)D, sizeof(int64_t));
    int64_t* binbase = (int64_t*)calloc((size_t)D + 1, sizeof(int64_t));
    int64_t* yoff = (int64_t*)calloc((size_t)D, sizeof(int64_t));
    double* T0 = (double*)calloc((size_t)D, sizeof(double));
    double* T1 = (double*)calloc((size_t)D, sizeof(double));
    if (!B || !binbase || !yoff || !T0 || !T1) return OR_ENOMEM;
    for (int32_t d = 0; d < D; ++d)
        if (f[d] <= 0 || N % f[d] != 0) return OR_EINVAL;
    const double noise_var = opt->noise_auto ? oracle_noise_estimate(N, D, f, R, Y) : opt->noise_var;
    if (noise_var < 0) return OR_ENOMEM;
    st->noise_var = noise_var;
    for (int32_t d = 0; d < D; ++d) {
        B[d] = N / f[d];
        binbase[d + 1] = binbase[d] + B[d];
        yoff[d] = (int64_t)R * binbase[d];
        /* Sec. 3.2 subproblem 1: ||y||^2 <= T0 zero-ton, ||y - poly||^2 <= T1 single-ton */
        double sig_y = (double)B[d] * noise_var;
        double floor_ = opt->eta * (double)B[d] * opt->a_min;
        T0[d] = (double)R * (opt->c0 * sig_y + floor_ * floor_);
        T1[d] = (double)R * (opt->c1 * sig_y + floor_ * floor_);
    }
    int64_t nb = binbase[D];

    /* ARG locate needs tau = 0 and tau = 1 in every stage (Sec. 3.2 subproblem 2) */
    int32_t* r0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)D);
    int32_t* r1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)D);
    for (int32_t d = 0; d < D; ++d) {
        r0[d] = r1[d] = -1;
        for (int32_t r = 0; r < R; ++r) {
            if (delays[(int64_t)d * R + r] == 0 && r0[d] < 0) r0[d] = r;
            if (delays[(int64_t)d * R + r] == 1 && r1[d] < 0) r1[d] = r;
        }
        if (opt->locate == 0 && (r0[d] < 0 || r1[d] < 0)) return OR_EINVAL;
    }
    if (opt->locate == 2) {
        /* C = R / m iterations must tell the L candidates of every stage apart: 2^C >= L */
        if (opt->kay_m < 2 || R % opt->kay_m != 0 || R / opt->kay_m > 30) return OR_EINVAL;
        for (int32_t d = 0; d < D; ++d)
            if (((int64_t)1 << (R / opt->kay_m)) < f[d]) return OR_EINVAL;
    }

    unsigned char* state = (unsigned char*)calloc((size_t)nb, 1); /* 0 open, else class */
    int64_t* cand_f = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    int32_t* cand_round = (int32_t*)malloc(sizeof(int32_t) * (size_t)nb);
    unsigned char* queued = (unsigned char*)calloc((size_t)nb, 1);
    int64_t* active = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    int64_t* s_bin = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    int64_t* s_f = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    cplx* s_v = (cplx*)malloc(sizeof(cplx) * (size_t)nb);
    rec_entry* rec = (rec_entry*)malloc(sizeof(rec_entry) * (size_t)nb);
    cplx* yv = (cplx*)malloc(sizeof(cplx) * (size_t)R);
    if (!state || !cand_f || !cand_round || !queued || !active || !next || !s_bin || !s_f || !s_v ||
        !rec || !yv)
        return OR_ENOMEM;
    for (int64_t b = 0; b < nb; ++b) { cand_f[b] = -1; cand_round[b] = -1; }

    /* Step 1 of the first peeling examines every bin */
    int64_t n_active = nb;
    for (int64_t b = 0; b < nb; ++b) active[b] = b;
    int64_t n_rec = 0, idents = 0;
    int32_t round = 0;

    while (n_active > 0 && round < opt->max_rounds) {
        round++;
        int64_t nz = 0, ns = 0, nm = 0, n_s = 0;
        /* Step 1: identify every examined bin from the state at the start of the round */
        for (int64_t a = 0; a < n_active; ++a) {
            int64_t b = active[a];
            queued[b] = 0;
            int32_t d = 0;
            while (b >= binbase[d + 1]) d++;
            int64_t j = b - binbase[d];
            const int64_t* tau = delays + (int64_t)d * R;
            double E = 0;
            for (int32_t r = 0; r < R; ++r) {
                yv[r] = Y[yoff[d] + (int64_t)r * B[d] + j];
                E += creal(yv[r]) * creal(yv[r]) + cimag(yv[r]) * cimag(yv[r]);
            }
            idents++;
            if (E <= T0[d]) { state[b] = OR_ZERO; nz++; continue; }
            int64_t L = f[d], fq;
            if (opt->locate == 2) {
                fq = locate_kay(yv, R, opt->kay_m, j, B[d], L, N);
            } else if (opt->locate == 0) {
                /* FFAST phase encoding: angle of y(1)/y(0) times N / 2 pi, snapped to the bin's
                 * candidate set {j + q B} */
                cplx ratio = yv[r1[d]] * conj(yv[r0[d]]);
                double fe = carg(ratio) * (double)N / OR_TWO_PI;
                double qd = floor((fe - (double)j) / (double)B[d] + 0.5);
                int64_t q = pos_mod((int64_t)qd, L);
                fq = j + q * B[d];
            } else {
                /* enumerate the L candidates and keep the best delay-phasor correlation */
                double best = -1.0;
                fq = j;
                for (int64_t q = 0; q < L; ++q) {
                    int64_t fc = j + q * B[d];
                    cplx c = 0;
                    for (int32_t r = 0; r < R; ++r) c += yv[r] * conj(delay_phasor(fc, tau[r], N));
                    double s = creal(c) * creal(c) + cimag(c) * cimag(c);
                    if (s > best) { best = s; fq = fc; }
                }
            }
            cplx v;
            double rho;
            fit_tone(yv, R, tau, fq, N, B[d], &v, &rho);
            if (rho <= T1[d]) {
                state[b] = OR_SINGLE;
                cand_f[b] = fq;
                cand_round[b] = round;
                s_bin[n_s] = b; s_f[n_s] = fq; s_v[n_s] = v; n_s++;
                ns++;
            } else {
                nm++;
            }
        }
        /* Step 2: take every new singleton once (lowest stage wins), subtract its
         * contribution from the bin it maps to in every stage (Eq. 20)                    */
        int64_t n_next = 0, n_acc = 0;
        for (int64_t s = 0; s < n_s; ++s) {
            int64_t b = s_bin[s], fq = s_f[s];
            int32_t d = 0;
            while (b >= binbase[d + 1]) d++;
            int accept = 1;
            for (int32_t e = 0; e < D && accept; ++e) {
                if (e == d) continue;
                int64_t be = binbase[e] + fq % B[e];
                if (cand_f[be] == fq &&
                    (cand_round[be] < round || (cand_round[be] == round && e < d)))
                    accept = 0;
            }
            if (!accept) continue;
            n_acc++;
            rec[n_rec].f = fq;
            rec[n_rec].v = s_v[s];
            n_rec++;
            for (int32_t e = 0; e < D; ++e) {
                int64_t je = fq % B[e];
                int64_t be = binbase[e] + je;
                const int64_t* tau = delays + (int64_t)e * R;
                for (int32_t r = 0; r < R; ++r)
                    Y[yoff[e] + (int64_t)r * B[e] + je] -=
                        (double)B[e] * s_v[s] * delay_phasor(fq, tau[r], N);
                if (state[be] == 0 && !queued[be]) { queued[be] = 1; next[n_next++] = be; }
            }
        }
        if (log) {
            if (log->idents) log->idents[round - 1] = n_active;
            if (log->n_zero) log->n_zero[round - 1] = nz;
            if (log->n_single) log->n_single[round - 1] = ns;
            if (log->n_multi) log->n_multi[round - 1] = nm;
            if (log->n_accepted) log->n_accepted[round - 1] = n_acc;
        }
        /* Step 3: repeat on the bins whose content changed */
        int64_t* t = active; active = next; next = t;
        n_active = n_next;
    }

    int64_t unresolved = 0;
    for (int64_t b = 0; b < nb; ++b) unresolved += state[b] == 0 || state[b] == OR_MULTI;
    if (rec_f || rec_v)
        for (int64_t i = 0; i < n_rec; ++i) {
            if (rec_f) rec_f[i] = rec[i].f;
            if (rec_v) rec_v[i] = rec[i].v;
        }

    /* output: the K largest recovered coefficients, sorted by frequency (Sec. 2.1) */
    int64_t n_out = n_rec;
    if (n_rec > K) {
        qsort(rec, (size_t)n_rec, sizeof(rec_entry), cmp_rec_by_mag);
        n_out = K;
    }
    qsort(rec, (size_t)n_out, sizeof(rec_entry), cmp_rec_by_f);
    for (int64_t i = 0; i < n_out; ++i) {
        if (out_idx) out_idx[i] = rec[i].f;
        if (out_val) out_val[i] = rec[i].v;
    }
    st->status = unresolved > 0 ? 1 : 0;
    st->rounds = round;
    st->n_recovered = (int32_t)n_rec;
    st->n_out = (int32_t)n_out;
    st->idents = idents;
    st->unresolved = unresolved;

    free(B); free(binbase); free(yoff); free(T0); free(T1); free(r0); free(r1);
    free(state); free(cand_f); free(cand_round); free(queued); free(active); free(next);
    free(s_bin); free(s_f); free(s_v); free(rec); free(yv);
    return OR_OK;
}
