/*
 * FP64 CPU oracle for the polyphase filter bank (PFB) channeliser.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no source,
 * header, table or helper with the CUDA library; it is the plain, slow,
 * obviously-correct definition the CUDA kernels are checked against.
 *
 * What it computes (paper: TINA, arXiv 2408.16551):
 *   - Prototype filter h[n], n < L = P*T: a windowed sinc with cutoff 1/P
 *     (read Nyquist-normalised: zero crossings every P samples), normalised so
 *     that sum(h) = 1.  The paper only says the taps are "divided between the
 *     P branches" (Sec. 5.2); the window/sinc/normalisation is this library's
 *     stated reading.
 *   - Branch decomposition x_p(f) = x[f*P + p] (Sec. 5.2, eq. for y_p(n')).
 *   - Polyphase FIR, the cross-correlation form that the FIR-as-convolution
 *     mapping computes (Sec. 4.3, O(w) = sum_n I(w+n) K(n)):
 *         y[s,p] = sum_{m<T} h[m*P + p] * x[(s+m)*P + p],  s < S = F - T + 1.
 *   - DFT as the product with the Fourier matrix (Sec. 4.1, Z = X F), forward
 *     sign, no normalisation:
 *         X[s,k] = sum_{p<P} y[s,p] * exp(-2*pi*i * ((p*k) mod P) / P).
 *
 * Parity status: every function here is pinned by tests under tests/ against
 * values that do not come from this file (library routines, closed forms,
 * brute force, invariants and the paper's worked unfolding example).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846264338327950288

enum { OR_WIN_HANN = 0, OR_WIN_HAMMING = 1, OR_WIN_BLACKMAN = 2, OR_WIN_USER = 3 };

/* Symmetric window over L points (w[0] = w[L-1]). */
static double window_value(int kind, int64_t n, int64_t L) {
    if (L <= 1) return 1.0;
    double a = 2.0 * ORACLE_PI * (double)n / (double)(L - 1);
    switch (kind) {
    case OR_WIN_HANN: return 0.5 - 0.5 * cos(a);
    case OR_WIN_HAMMING: return 0.54 - 0.46 * cos(a);
    case OR_WIN_BLACKMAN: return 0.42 - 0.5 * cos(a) + 0.08 * cos(2.0 * a);
    default: return 1.0;
    }
}

static double sinc(double u) {
    if (u == 0.0) return 1.0;
    return sin(ORACLE_PI * u) / (ORACLE_PI * u);
}

/* Windowed-sinc prototype of length L = P*T (any L >= 1 is accepted so that
 * tests can call it with odd lengths).  Returns 0 on success, -1 on bad input.
 * USER taps are copied unchanged (no normalisation). */
int oracle_prototype(int64_t P, int64_t L, int kind, const double *user, double *h) {
    if (P < 1 || L < 1 || h == NULL) return -1;
    if (kind == OR_WIN_USER) {
        if (user == NULL) return -1;
        memcpy(h, user, (size_t)L * sizeof(double));
        return 0;
    }
    if (kind < 0 || kind > OR_WIN_BLACKMAN) return -1;
    double c = 0.5 * (double)(L - 1);
    double sum = 0.0;
    for (int64_t n = 0; n < L; ++n) {
        h[n] = window_value(kind, n, L) * sinc(((double)n - c) / (double)P);
        sum += h[n];
    }
    if (sum == 0.0) return -1;
    for (int64_t n = 0; n < L; ++n) h[n] /= sum;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Polyphase FIR                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *xr, *xi, *h;
    int64_t P, T, s0, s1;
    double *yr, *yi; /* rows relative to the first requested spectrum */
    int64_t row0;
} fir_job;

static void *fir_worker(void *arg) {
    fir_job *j = (fir_job *)arg;
    for (int64_t s = j->s0; s < j->s1; ++s) {
        double *orow_r = j->yr + (s - j->row0) * j->P;
        double *orow_i = j->yi + (s - j->row0) * j->P;
        for (int64_t p = 0; p < j->P; ++p) {
            double ar = 0.0, ai = 0.0;
            for (int64_t m = 0; m < j->T; ++m) {
                double hv = j->h[m * j->P + p];
                int64_t idx = (s + m) * j->P + p;
                ar += hv * j->xr[idx];
                ai += hv * j->xi[idx];
            }
            orow_r[p] = ar;
            orow_i[p] = ai;
        }
    }
    return NULL;
}

static int run_jobs(void *(*fn)(void *), void *jobs, size_t job_size, int n) {
    if (n <= 1) {
        fn(jobs);
        return 0;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n);
    if (!th) return -1;
    int started = 0;
    for (int i = 0; i < n; ++i) {
        if (pthread_create(&th[i], NULL, fn, (char *)jobs + (size_t)i * job_size) != 0) {
            fn((char *)jobs + (size_t)i * job_size); /* run inline if a thread cannot start */
            th[i] = 0;
        } else {
            started++;
        }
    }
    for (int i = 0; i < n; ++i)
        if (th[i]) pthread_join(th[i], NULL);
    free(th);
    (void)started;
    return 0;
}

/* Number of spectra for N samples: F = floor(N/P) frames, S = max(0, F-T+1). */
int64_t oracle_num_spectra(int64_t N, int64_t P, int64_t T) {
    if (P < 1 || T < 1 || N < 0) return -1;
    int64_t F = N / P;
    int64_t S = F - T + 1;
    return S > 0 ? S : 0;
}

/* y[s - s0, p] for s in [s0, s0+ns).  x holds N complex samples (re, im split). */
int oracle_fir(const double *xr, const double *xi, int64_t N, int64_t P, int64_t T,
               const double *h, int64_t s0, int64_t ns, double *yr, double *yi,
               int nthreads) {
    int64_t S = oracle_num_spectra(N, P, T);
    if (S < 0 || s0 < 0 || ns < 0 || s0 + ns > S) return -1;
    if (ns == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ns) nthreads = (int)ns;
    fir_job *jobs = (fir_job *)calloc((size_t)nthreads, sizeof(fir_job));
    if (!jobs) return -1;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].xr = xr; jobs[t].xi = xi; jobs[t].h = h;
        jobs[t].P = P; jobs[t].T = T;
        jobs[t].s0 = s0 + ns * t / nthreads;
        jobs[t].s1 = s0 + ns * (t + 1) / nthreads;
        jobs[t].yr = yr; jobs[t].yi = yi; jobs[t].row0 = s0;
    }
    int rc = run_jobs(fir_worker, jobs, sizeof(fir_job), nthreads);
    free(jobs);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Naive DFT over each row (the product with the Fourier matrix)            */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *yr, *yi, *cr, *ci; /* cr/ci: cos/sin table of 2*pi*r/P */
    int64_t P, r0, r1;
    double *Xr, *Xi;
} dft_job;

static void *dft_worker(void *arg) {
    dft_job *j = (dft_job *)arg;
    int64_t P = j->P;
    for (int64_t s = j->r0; s < j->r1; ++s) {
        const double *yr = j->yr + s * P, *yi = j->yi + s * P;
        for (int64_t k = 0; k < P; ++k) {
            double ar = 0.0, ai = 0.0;
            for (int64_t p = 0; p < P; ++p) {
                int64_t r = (p * k) % P;
                /* (yr + i yi) * (cos - i sin) */
                double c = j->cr[r], sn = j->ci[r];
                ar += yr[p] * c + yi[p] * sn;
                ai += yi[p] * c - yr[p] * sn;
            }
            j->Xr[s * P + k] = ar;
            j->Xi[s * P + k] = ai;
        }
    }
    return NULL;
}

int oracle_dft(const double *yr, const double *yi, int64_t nrows, int64_t P,
               double *Xr, double *Xi, int nthreads) {
    if (P < 1 || nrows < 0) return -1;
    if (nrows == 0) return 0;
    double *cr = (double *)malloc(sizeof(double) * (size_t)P);
    double *ci = (double *)malloc(sizeof(double) * (size_t)P);
    if (!cr || !ci) { free(cr); free(ci); return -1; }
    for (int64_t r = 0; r < P; ++r) {
        double a = 2.0 * ORACLE_PI * (double)r / (double)P;
        cr[r] = cos(a);
        ci[r] = sin(a);
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrows) nthreads = (int)nrows;
    dft_job *jobs = (dft_job *)calloc((size_t)nthreads, sizeof(dft_job));
    if (!jobs) { free(cr); free(ci); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].yr = yr; jobs[t].yi = yi; jobs[t].cr = cr; jobs[t].ci = ci;
        jobs[t].P = P;
        jobs[t].r0 = nrows * t / nthreads;
        jobs[t].r1 = nrows * (t + 1) / nthreads;
        jobs[t].Xr = Xr; jobs[t].Xi = Xi;
    }
    int rc = run_jobs(dft_worker, jobs, sizeof(dft_job), nthreads);
    free(jobs); free(cr); free(ci);
    return rc;
}

/* Full channeliser for spectra [s0, s0+ns): FIR, then DFT of each row. */
int oracle_pfb(const double *xr, const double *xi, int64_t N, int64_t P, int64_t T,
               const double *h, int64_t s0, int64_t ns, double *Xr, double *Xi,
               int nthreads) {
    if (ns < 0) return -1;
    if (ns == 0) return 0;
    double *yr = (double *)malloc(sizeof(double) * (size_t)(ns * P));
    double *yi = (double *)malloc(sizeof(double) * (size_t)(ns * P));
    if (!yr || !yi) { free(yr); free(yi); return -1; }
    int rc = oracle_fir(xr, xi, N, P, T, h, s0, ns, yr, yi, nthreads);
    if (rc == 0) rc = oracle_dft(yr, yi, ns, P, Xr, Xi, nthreads);
    free(yr); free(yi);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Oversampled channeliser and the convolution tap order                    */
/* ------------------------------------------------------------------------ */

/* Spectra of a channeliser with hop D: windows of P*T samples starting at
 * s*D; S = floor((N - P*T)/D) + 1 for N >= P*T, else 0. */
int64_t oracle_num_spectra_hop(int64_t N, int64_t P, int64_t T, int64_t D) {
    if (P < 1 || T < 1 || D < 1 || N < 0) return -1;
    if (N < P * T) return 0;
    return (N - P * T) / D + 1;
}

typedef struct {
    const double *xr, *xi, *h;
    int64_t P, T, D, s0, s1, row0;
    int reverse;
    double *yr, *yi;
} fir_hop_job;

static void *fir_hop_worker(void *arg) {
    fir_hop_job *j = (fir_hop_job *)arg;
    for (int64_t s = j->s0; s < j->s1; ++s) {
        double *orow_r = j->yr + (s - j->row0) * j->P;
        double *orow_i = j->yi + (s - j->row0) * j->P;
        for (int64_t p = 0; p < j->P; ++p) {
            double ar = 0.0, ai = 0.0;
            for (int64_t m = 0; m < j->T; ++m) {
                /* tap m of branch p: h[m*P + p] (correlation form, Sec. 4.3) or
                   h[(T-1-m)*P + p] (the convolution of the Sec. 5.2 equation) */
                int64_t mt = j->reverse ? (j->T - 1 - m) : m;
                double hv = j->h[mt * j->P + p];
                int64_t idx = s * j->D + m * j->P + p;
                ar += hv * j->xr[idx];
                ai += hv * j->xi[idx];
            }
            orow_r[p] = ar;
            orow_i[p] = ai;
        }
    }
    return NULL;
}

/* X[s - s0, k] for s in [s0, s0+ns) of the channeliser with hop D and the
 * given tap order: y[s,p] = sum_m h'[m*P+p] x[s*D + m*P + p], then the DFT
 * of each row (Sec. 4.1).  D = P with reverse = 0 is oracle_pfb. */
int oracle_pfb_hop(const double *xr, const double *xi, int64_t N, int64_t P, int64_t T, int64_t D,
                   int reverse, const double *h, int64_t s0, int64_t ns, double *Xr, double *Xi, int nthreads) {
    int64_t S = oracle_num_spectra_hop(N, P, T, D);
    if (S < 0 || s0 < 0 || ns < 0 || s0 + ns > S) return -1;
    if (ns == 0) return 0;
    double *yr = (double *)malloc(sizeof(double) * (size_t)(ns * P));
    double *yi = (double *)malloc(sizeof(double) * (size_t)(ns * P));
    if (!yr || !yi) { free(yr); free(yi); return -1; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ns) nthreads = (int)ns;
    fir_hop_job *jobs = (fir_hop_job *)calloc((size_t)nthreads, sizeof(fir_hop_job));
    if (!jobs) { free(yr); free(yi); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].xr = xr; jobs[t].xi = xi; jobs[t].h = h;
        jobs[t].P = P; jobs[t].T = T; jobs[t].D = D; jobs[t].reverse = reverse;
        jobs[t].s0 = s0 + ns * t / nthreads;
        jobs[t].s1 = s0 + ns * (t + 1) / nthreads;
        jobs[t].row0 = s0;
        jobs[t].yr = yr; jobs[t].yi = yi;
    }
    int rc = run_jobs(fir_hop_worker, jobs, sizeof(fir_hop_job), nthreads);
    free(jobs);
    if (rc == 0) rc = oracle_dft(yr, yi, ns, P, Xr, Xi, nthreads);
    free(yr); free(yi);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Synthesis (inverse) filter bank                                          */
/* ------------------------------------------------------------------------ */

/* The adjoint of the analysis channeliser, up to the IDFT's 1/P:
 *   y~[s,p] = (1/P) sum_{k<P} X[s,k] exp(+2 pi i (pk mod P)/P)  (the inverse
 *             Fourier-matrix product of Sec. 4.2);
 *   xh[f*P + p] = sum_{m<T} h[m*P + p] y~[f - m, p],  f < S + T - 1,
 *             with y~[s,p] = 0 outside 0 <= s < S (each spectrum s spreads its
 *             branch values over the T frames it was analysed from).
 * Frames [f0, f0 + nf) are written to xh (nf*P complex samples). */
int oracle_synth(const double *Xr, const double *Xi, int64_t S, int64_t P, int64_t T, const double *h,
                 int64_t f0, int64_t nf, double *xr, double *xi) {
    if (P < 1 || T < 1 || S < 0 || f0 < 0 || nf < 0 || f0 + nf > (S > 0 ? S + T - 1 : 0)) return -1;
    if (nf == 0) return 0;
    /* rows s in [f0 - T + 1, f0 + nf) intersect [0, S): their IDFTs */
    int64_t sa = f0 - T + 1 < 0 ? 0 : f0 - T + 1;
    int64_t sb = f0 + nf < S ? f0 + nf : S;
    int64_t nr = sb > sa ? sb - sa : 0;
    double *cr = (double *)malloc(sizeof(double) * (size_t)P);
    double *ci = (double *)malloc(sizeof(double) * (size_t)P);
    double *yr = (double *)calloc((size_t)(nr * P + 1), sizeof(double));
    double *yi = (double *)calloc((size_t)(nr * P + 1), sizeof(double));
    if (!cr || !ci || !yr || !yi) { free(cr); free(ci); free(yr); free(yi); return -1; }
    for (int64_t r = 0; r < P; ++r) {
        double a = 2.0 * ORACLE_PI * (double)r / (double)P;
        cr[r] = cos(a);
        ci[r] = sin(a);
    }
    for (int64_t s = sa; s < sb; ++s) {
        const double *ar = Xr + s * P, *ai = Xi + s * P;
        for (int64_t p = 0; p < P; ++p) {
            double accr = 0.0, acci = 0.0;
            for (int64_t k = 0; k < P; ++k) {
                int64_t r = (p * k) % P;
                /* (ar + i ai) * (cos + i sin) */
                accr += ar[k] * cr[r] - ai[k] * ci[r];
                acci += ai[k] * cr[r] + ar[k] * ci[r];
            }
            yr[(s - sa) * P + p] = accr / (double)P;
            yi[(s - sa) * P + p] = acci / (double)P;
        }
    }
    for (int64_t f = f0; f < f0 + nf; ++f) {
        for (int64_t p = 0; p < P; ++p) {
            double accr = 0.0, acci = 0.0;
            for (int64_t m = 0; m < T; ++m) {
                int64_t s = f - m;
                if (s < sa || s >= sb) continue;
                double hv = h[m * P + p];
                accr += hv * yr[(s - sa) * P + p];
                acci += hv * yi[(s - sa) * P + p];
            }
            xr[(f - f0) * P + p] = accr;
            xi[(f - f0) * P + p] = acci;
        }
    }
    free(cr); free(ci); free(yr); free(yi);
    return 0;
}
