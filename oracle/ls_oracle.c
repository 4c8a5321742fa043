/*
 * Oracle: direct FP64 evaluation of the floating-mean Lomb-Scargle periodogram.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct CPU
 * definition that the GPU path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may build, load or call it;
 * the library under paper_2409_08090_gb300/ never does, and nothing here is
 * shared with it.
 *
 * What it computes (nifty-ls, arXiv 2409.08090):
 *   - Eq. 1 (Sec. 1): the weighted trigonometric sums
 *         S_k = sum_j h_j sin(2 pi f_k t_j),   C_k = sum_j h_j cos(2 pi f_k t_j)
 *     evaluated directly, O(N_d N_f), for f_k = f0 + k df.  Sec. 2 ("Accuracy")
 *     names exactly this direct evaluation as the reference result.
 *   - The sums are taken for three weight vectors, as the floating-mean
 *     ("generalised") model needs: h = w^ (y - ybar) and h = w^ at f_k, and
 *     h = w^ at 2 f_k, with w_j = 1/dy_j^2, w^_j = w_j / sum w, ybar = sum w^ y.
 *     The paper cites VanderPlas (2018) for the periodogram itself and states
 *     none of these formulas; the model, tau and the standard normalisation
 *     below are that reference's generalised periodogram.
 *   - tau:  tan(2 w tau) = (S2 - 2 C S) / (C2 - (C^2 - S^2)),  w = 2 pi f.
 *   - P = (YC_tau^2 / CC_tau + YS_tau^2 / SS_tau) / YY  (standard normalisation),
 *     with YC_tau = Ch cos + Sh sin, YS_tau = Sh cos - Ch sin,
 *     C_tau = C cos + S sin, S_tau = S cos - C sin,
 *     CC_tau = (1 + C2 cos2 + S2 sin2)/2 - C_tau^2,
 *     SS_tau = (1 - C2 cos2 - S2 sin2)/2 - S_tau^2,  YY = sum w^ (y-ybar)^2.
 *
 *
 * Model variants (ls_oracle_power_ex).  The package is a backend of the Astropy
 * Lomb-Scargle interface (Sec. 1), whose options select the model and the
 * normalisation.  With p = YC_tau^2/CC_tau + YS_tau^2/SS_tau:
 *   - fit_mean = 0: no offset in the model, so C and S drop out:
 *     tan(2 w tau) = S2 / C2, CC_tau = (1 + C2 cos2 + S2 sin2)/2,
 *     SS_tau = (1 - C2 cos2 - S2 sin2)/2.
 *   - center = 0 (meaningful only with fit_mean = 0; a fitted offset always
 *     works on centred data): y' = y and YY = sum w^ y^2.
 *   - normalisation 0 standard p / YY; 1 model p / (YY - p);
 *     2 log -ln(1 - p / YY); 3 psd p W / 2 with W = sum w (unnormalised).
 *   In least-squares terms (chi2 with the unnormalised weights w, chi2_ref of
 *   the model without its sinusoid): standard 1 - chi2/chi2_ref, model
 *   chi2_ref/chi2 - 1, log ln(chi2_ref/chi2), psd (chi2_ref - chi2)/2.
 *
 * Arithmetic: FP64 throughout.  The inputs are treated as exact reals: the
 * phase f_k t_j (in cycles) is formed with error-free products (fma) in
 * double-double and reduced modulo 1 before sin/cos, so the long-baseline
 * phases of large configurations lose nothing to the product's rounding.
 * Summation is plain left-to-right over j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

/* Phase of frequency f0 + k df at time t, in cycles, reduced to [-1/2, 1/2].
 * f0 t and df t are split exactly into hi + lo with fma; k (df t)_hi is split
 * the same way; the integer parts are dropped before the small parts are
 * added, so the result is accurate to a few units of 1e-16 cycles. */
static double phase_cycles(double f0, double df, int64_t k, double t)
{
    double a_hi = f0 * t, a_lo = fma(f0, t, -a_hi);
    double b_hi = df * t, b_lo = fma(df, t, -b_hi);
    double kd = (double)k;
    double c_hi = kd * b_hi, c_lo = fma(kd, b_hi, -c_hi);
    double s = (a_hi - rint(a_hi)) + (c_hi - rint(c_hi));
    s += a_lo + c_lo + kd * b_lo;
    return s - rint(s);
}

/* Weighted mean and normalised weights (shared by every frequency); y' = y - ybar
 * when centring, else y.  Returns 0 on success, -1 if the inputs are unusable. */
static int prepare(int64_t nd, const double *y, const double *dy, int center,
                   double *what, double *yc, double *yy_out, double *W_out)
{
    double W = 0.0;
    for (int64_t j = 0; j < nd; ++j) {
        double d = dy ? dy[j] : 1.0;
        if (!(d > 0.0)) return -1;
        what[j] = 1.0 / (d * d);
        W += what[j];
    }
    double ybar = 0.0;
    for (int64_t j = 0; j < nd; ++j) {
        what[j] /= W;
        ybar += what[j] * y[j];
    }
    if (!center) ybar = 0.0;
    double yy = 0.0, y2 = 0.0;
    for (int64_t j = 0; j < nd; ++j) {
        yc[j] = y[j] - ybar;
        yy += what[j] * yc[j] * yc[j];
        y2 += what[j] * y[j] * y[j];
    }
    /* A constant series (variance zero up to the rounding of the mean) has no
     * periodogram. */
    if (!(yy > 1e-24 * y2)) return -1;
    *yy_out = yy;
    *W_out = W;
    return 0;
}

/* Power from the six sums, YY and W (see the file header). */
static double power_from_sums(double Ch, double Sh, double C, double S,
                              double C2, double S2, double YY, double W,
                              int fit_mean, int norm)
{
    double two_wtau = fit_mean ? atan2(S2 - 2.0 * C * S, C2 - (C * C - S * S))
                               : atan2(S2, C2);
    double wtau = 0.5 * two_wtau;
    double c = cos(wtau), s = sin(wtau);
    double c2 = cos(two_wtau), s2 = sin(two_wtau);
    double YC = Ch * c + Sh * s;
    double YS = Sh * c - Ch * s;
    double CC = 0.5 * (1.0 + C2 * c2 + S2 * s2);
    double SS = 0.5 * (1.0 - C2 * c2 - S2 * s2);
    if (fit_mean) {
        double Ct = C * c + S * s;
        double St = S * c - C * s;
        CC -= Ct * Ct;
        SS -= St * St;
    }
    /* A vanishing CC or SS (all phases equal mod pi) carries no information:
     * that term of the fit is absent. */
    double p = 0.0;
    if (CC > 1e-15) p += YC * YC / CC;
    if (SS > 1e-15) p += YS * YS / SS;
    switch (norm) {
    case 1: return p / (YY - p);
    case 2: return -log(1.0 - p / YY);
    case 3: return 0.5 * W * p;
    default: return p / YY;
    }
}

/*
 * ls_oracle_power_ex: periodogram at the frequencies f0 + k[i] df, i < nk.
 *   t, y: nd FP64 values; dy: nd FP64 values or NULL (all ones).
 *   fit_mean, center, norm: the model variant (file header); fit_mean = 1
 *   always centres.
 *   power: nk outputs.  sums: NULL or nk*7 outputs, per frequency
 *   (Ch, Sh, C, S, C2, S2, YY) as defined in the file header.
 * Returns 0, or -1 for nd < 1, a non-positive dy, an unknown norm, or a
 * vanishing YY (YY <= 1e-24 sum w^ y^2, i.e. zero up to rounding).
 */
int ls_oracle_power_ex(int64_t nd, const double *t, const double *y, const double *dy,
                       double f0, double df, int64_t nk, const int64_t *k,
                       int fit_mean, int center, int norm, double *power, double *sums)
{
    if (nd < 1 || nk < 0 || norm < 0 || norm > 3) return -1;
    if (fit_mean) center = 1;
    double *what = (double *)malloc(sizeof(double) * (size_t)nd);
    double *yc = (double *)malloc(sizeof(double) * (size_t)nd);
    if (!what || !yc) { free(what); free(yc); return -1; }
    double YY, W;
    int rc = prepare(nd, y, dy, center, what, yc, &YY, &W);
    if (rc == 0) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t i = 0; i < nk; ++i) {
            double Ch = 0, Sh = 0, C = 0, S = 0, C2 = 0, S2 = 0;
            for (int64_t j = 0; j < nd; ++j) {
                double ph = phase_cycles(f0, df, k[i], t[j]);
                double ph2 = 2.0 * ph;            /* exact doubling */
                ph2 -= rint(ph2);
                double sn = sin(TWO_PI * ph), cs = cos(TWO_PI * ph);
                double sn2 = sin(TWO_PI * ph2), cs2 = cos(TWO_PI * ph2);
                Ch += what[j] * yc[j] * cs;
                Sh += what[j] * yc[j] * sn;
                C += what[j] * cs;
                S += what[j] * sn;
                C2 += what[j] * cs2;
                S2 += what[j] * sn2;
            }
            power[i] = power_from_sums(Ch, Sh, C, S, C2, S2, YY, W, fit_mean, norm);
            if (sums) {
                double *o = sums + 7 * i;
                o[0] = Ch; o[1] = Sh; o[2] = C; o[3] = S; o[4] = C2; o[5] = S2; o[6] = YY;
            }
        }
    }
    free(what);
    free(yc);
    return rc;
}

/* The default model: floating mean, standard normalisation. */
int ls_oracle_power(int64_t nd, const double *t, const double *y, const double *dy,
                    double f0, double df, int64_t nk, const int64_t *k,
                    double *power, double *sums)
{
    return ls_oracle_power_ex(nd, t, y, dy, f0, df, nk, k, 1, 1, 0, power, sums);
}

/* Number of threads the parallel loop above uses. */
int ls_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
