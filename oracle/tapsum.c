/*
 * FP64 direct tap-sum correlation -- part of the FDAS test oracle.
 *
 * TEST INFRASTRUCTURE ONLY: linked by the oracle's Python module, which only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load.
 *
 * Computes the matched-filter correlation of Eq. 23 (Section 2) by its plain
 * definition, with no FFT and no overlap-save:
 *
 *     F_k(r) = sum_{d=-h_k}^{h_k} A[r + d] * conj(R_k[d]),
 *
 * where A is the complex spectrum (A[q] = 0 for q outside [0, nb), the zero
 * padding of Section 3) and R_k[d] the k-th template's response at integer
 * offset d from the bin being recovered (the "frequency reversed and complex
 * conjugated template" of Eq. 23).  Complex values are interleaved (re, im).
 */
#include <stdint.h>

static void one_point(const double *A, int64_t nb, const double *Rk, int32_t hk,
                      int32_t hmax, int64_t r, double *out)
{
    double fr = 0.0, fi = 0.0;
    for (int32_t d = -hk; d <= hk; ++d) {
        int64_t q = r + d;
        if (q < 0 || q >= nb)
            continue;
        double ar = A[2 * q], ai = A[2 * q + 1];
        double tr = Rk[2 * (hmax + d)], ti = Rk[2 * (hmax + d) + 1];
        /* A * conj(R) */
        fr += ar * tr + ai * ti;
        fi += ai * tr - ar * ti;
    }
    out[0] = fr;
    out[1] = fi;
}

/* F[k][i] for k < K, i < nr (bins r = r0 + i).  R is K x (2*hmax+1) complex,
 * row k holding offsets d = -hmax..hmax; h[k] <= hmax taps are used. */
void oracle_tapsum(const double *A, int64_t nb, const double *R, const int32_t *h,
                   int32_t K, int32_t hmax, int64_t r0, int64_t nr, double *F)
{
    const int64_t width = 2 * (int64_t)hmax + 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int32_t k = 0; k < K; ++k)
        for (int64_t i = 0; i < nr; ++i)
            one_point(A, nb, R + 2 * width * k, h[k], hmax, r0 + i,
                      F + 2 * ((int64_t)k * nr + i));
}

/* F[p] at npts scattered points (template index zi[p], bin r[p]). */
void oracle_tapsum_points(const double *A, int64_t nb, const double *R, const int32_t *h,
                          int32_t hmax, const int32_t *zi, const int64_t *r,
                          int64_t npts, double *F)
{
    const int64_t width = 2 * (int64_t)hmax + 1;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p)
        one_point(A, nb, R + 2 * width * zi[p], h[zi[p]], hmax, r[p], F + 2 * p);
}

int oracle_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
