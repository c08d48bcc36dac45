/*
 * oracle.c -- FP64 CPU oracle for the road-surface stereo hot path of
 * Fan et al., "Real-Time Stereo Vision for Road Surface 3-D Reconstruction"
 * (arXiv 1807.07433).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline / reference arm may load this
 * library.  The CUDA path shares no code, header, table or helper with it.
 *
 * Every quantity is computed by its direct definition in double precision:
 * explicit window sums (no running sums, no integral images), explicit
 * neighbourhood sums for the bilateral filter, a linear scan for the argmax.
 * Where the paper is silent the reading used is stated at the function.
 *
 * Layouts: images are row-major [H][W] (index v*W+u); cost volumes and
 * aggregated volumes are [H][W][D] (index (v*W+u)*D+d); XYZ is three planes
 * [3][H][W].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int W, H;          /* image size */
    int D;             /* number of residual disparities searched: 0..D-1 */
    int ncc_r;         /* NCC block radius (rho-script in Eq. 3); n = (2r+1)^2 */
    int agg_r;         /* bilateral window radius (rho in Eq. 8) */
    double gamma_d;    /* Eq. 9 */
    double gamma_r;    /* Eq. 10 */
    double lr_thresh;  /* L-R consistency tolerance in pixels (Eq. 11 is 0) */
    double alpha0, alpha1, delta; /* Eq. 2 plane and the offset of Sec. II-A */
    double f_px, baseline, u0, v0; /* camera for Sec. II-D */
} orc_params;

/* Optional outputs; any pointer may be NULL.  Arrays are full-frame sized
 * even when only a band of rows is computed (rows outside are untouched). */
typedef struct {
    double *warped;           /* [H][W] i_r' after the perspective transform */
    double *mu_l, *sig_l;     /* [H][W] block mean / std of i_l  (Eq. 4) */
    double *mu_r, *sig_r;     /* [H][W] block mean / std of i_r' (Eq. 5) */
    double *cost_l, *cost_r;  /* [H][W][D] raw NCC volumes (Eq. 3) */
    double *agg_l, *agg_r;    /* [H][W][D] aggregated volumes (Eq. 8) */
    int32_t *lbl_l, *lbl_r;   /* [H][W] WTA maps l_ref, l_tar */
    double *gap_l, *gap_r;    /* [H][W] best minus second-best aggregated cost */
    double *den_l;            /* [H][W] parabola denominator of Eq. 12 (0 at ends) */
    double *dsub;             /* [H][W] subpixel residual disparity d^s */
    uint8_t *valid;           /* [H][W] 1 where the L-R check passes */
    double *dfull;            /* [H][W] post-processed disparity, NaN if rejected */
    double *xyz;              /* [3][H][W] reconstructed points, NaN if rejected */
} orc_outputs;

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Planted mistakes for the pin tests' own test (tests/test_oracle_mutants.py):
 * built with -DORC_MUTANT=k, the library carries mistake k, one plausible
 * slip each (a flipped sign or direction, a dropped term, an off-by-one, a
 * wrong normaliser); the pins must catch every one.  The default build
 * (ORC_MUTANT 0) has none. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#define MUT(k) (ORC_MUTANT == (k))

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Sec. II-A: every point of target row v is shifted alpha0 + alpha1*v - delta
 * pixels to the right (Eq. 2 gives the road-plane disparity alpha0+alpha1*v). */
double orc_row_shift(const orc_params *p, int v) {
    return p->alpha0 + p->alpha1 * (double)v - p->delta;
}

/* Sec. II-A perspective transformation of the target image.
 * Reading: a shift by s to the right means i_r'(x,v) = i_r(x - s, v); a
 * non-integer shift is linear interpolation along x (what bilinear resampling
 * reduces to for a pure row shift); source columns outside the image are
 * clamped to the edge.  With k = floor(s), w = s - k:
 *     i_r'(x,v) = (1-w) i_r(x-k, v) + w i_r(x-k-1, v). */
void orc_warp(const orc_params *p, const uint8_t *ir, double *out) {
    const int W = p->W, H = p->H;
    for (int v = 0; v < H; ++v) {
        const double s = orc_row_shift(p, v);
        const double k = floor(s);
        const double w = s - k;
        const int ki = (int)k;
        for (int x = 0; x < W; ++x) {
            const int xa = MUT(1) ? x + ki : x - ki, xb = MUT(1) ? x + ki + 1 : x - ki - 1;
            const double a = ir[(size_t)v * W + clampi(xa, 0, W - 1)];
            const double b = ir[(size_t)v * W + clampi(xb, 0, W - 1)];
            out[(size_t)v * W + x] = MUT(2) ? w * a + (1.0 - w) * b : (1.0 - w) * a + w * b;
        }
    }
}

/* Eqs. 4-5: mean and population standard deviation of the (2r+1)x(2r+1)
 * block centred at (u,v).  Reading: pixels outside the image are read
 * clamp-to-edge, so a block is defined for any integer centre.
 * Returns the variance; writes mu and sigma. */
double orc_block_stats(const double *img, int W, int H, int r, int u, int v,
                       double *mu, double *sigma) {
    const double n = (double)((2 * r + 1) * (2 * r + 1));
    double s = 0.0, s2 = 0.0;
    for (int j = -r; j <= r; ++j) {
        const int y = clampi(v + j, 0, H - 1);
        for (int i = -r; i <= r; ++i) {
            const double val = img[(size_t)y * W + clampi(u + i, 0, W - 1)];
            s += val;
            s2 += val * val;
        }
    }
    const double m = s / n;
    double var = s2 / n - m * m;          /* Eq. 4 / Eq. 5 under the root */
    if (MUT(4)) var *= n / (n - 1.0);
    if (var < 0.0) var = 0.0;
    if (mu) *mu = m;
    if (sigma) *sigma = sqrt(var);
    return var;
}

/* Variance below which a block is treated as flat and its NCC is 0
 * (reading: Eq. 3 divides by n*sigma_l*sigma_r, undefined for a flat block). */
#define ORC_FLAT_VAR 1e-6

/* Eq. 3: normalised cross-correlation between the left block centred at
 * (ul, v) and the right block centred at (ur, v) of the warped target.
 * In the paper's notation ul = u and ur = u - d. */
double orc_ncc(const double *L, const double *R, int W, int H, int r,
               int ul, int ur, int v) {
    double mu_l, sig_l, mu_r, sig_r;
    const double var_l = orc_block_stats(L, W, H, r, ul, v, &mu_l, &sig_l);
    const double var_r = orc_block_stats(R, W, H, r, ur, v, &mu_r, &sig_r);
    if (var_l < ORC_FLAT_VAR || var_r < ORC_FLAT_VAR) return 0.0;
    const double n = (double)((2 * r + 1) * (2 * r + 1));
    double dot = 0.0;
    for (int j = -r; j <= r; ++j) {
        const int y = clampi(v + j, 0, H - 1);
        for (int i = -r; i <= r; ++i) {
            dot += L[(size_t)y * W + clampi(ul + i, 0, W - 1)] *
                   R[(size_t)y * W + clampi(ur + i, 0, W - 1)];
        }
    }
    return ((MUT(3) ? dot : dot - n * mu_l * mu_r)) / (n * sig_l * sig_r);
}

/* Eqs. 8-10: bilateral aggregation of cost slice d at (u,v).
 * vol is [H][W][D]; g is the guide image whose intensities drive omega_r.
 * Readings: Eqs. 9-10 carry no factor 2; neighbours outside the image are
 * left out of both sums. */
double orc_bilateral(const double *vol, int D, int d, const double *g, int W, int H,
                     int rho, double gamma_d, double gamma_r, int u, int v) {
    const double gc = g[(size_t)v * W + u];
    double num = 0.0, den = 0.0;
    for (int dy = -rho; dy <= rho; ++dy) {
        const int y = MUT(6) ? clampi(v + dy, 0, H - 1) : v + dy;
        if (y < 0 || y >= H) continue;
        for (int dx = -rho; dx <= rho; ++dx) {
            const int x = MUT(6) ? clampi(u + dx, 0, W - 1) : u + dx;
            if (x < 0 || x >= W) continue;
            const double wd = exp(-(double)(dx * dx + dy * dy) / ((MUT(5) ? 2.0 : 1.0) * gamma_d * gamma_d)); /* Eq. 9 */
            const double di = g[(size_t)y * W + x] - gc;
            const double wr = exp(-(di * di) / ((MUT(5) ? 2.0 : 1.0) * gamma_r * gamma_r));                  /* Eq. 10 */
            num += wd * wr * vol[((size_t)y * W + x) * D + d];
            den += wd * wr;
        }
    }
    return num / den;
}

/* Bilateral aggregation of every disparity at (u,v): out[d] for d in [0,D).
 * Each out[d] is exactly the sum of orc_bilateral (same terms, same order);
 * the weights are simply evaluated once per neighbour. */
static void bilateral_all_d(const double *vol, int D, const double *g, int W, int H,
                            int rho, double gamma_d, double gamma_r, int u, int v,
                            double *num, double *out) {
    const double gc = g[(size_t)v * W + u];
    double den = 0.0;
    for (int d = 0; d < D; ++d) num[d] = 0.0;
    for (int dy = -rho; dy <= rho; ++dy) {
        const int y = MUT(6) ? clampi(v + dy, 0, H - 1) : v + dy;
        if (y < 0 || y >= H) continue;
        for (int dx = -rho; dx <= rho; ++dx) {
            const int x = MUT(6) ? clampi(u + dx, 0, W - 1) : u + dx;
            if (x < 0 || x >= W) continue;
            const double wd = exp(-(double)(dx * dx + dy * dy) / ((MUT(5) ? 2.0 : 1.0) * gamma_d * gamma_d));
            const double di = g[(size_t)y * W + x] - gc;
            const double wr = exp(-(di * di) / ((MUT(5) ? 2.0 : 1.0) * gamma_r * gamma_r));
            const double *c = vol + ((size_t)y * W + x) * D;
            for (int d = 0; d < D; ++d) num[d] += wd * wr * c[d];
            den += wd * wr;
        }
    }
    for (int d = 0; d < D; ++d) out[d] = num[d] / den;
}

/* Bilateral filter of one 2-D slice (tests use it with synthetic slices). */
void orc_bilateral_slice(const double *slice, const double *g, int W, int H, int rho,
                         double gamma_d, double gamma_r, double *out) {
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u)
            out[(size_t)v * W + u] = orc_bilateral(slice, 1, 0, g, W, H, rho, gamma_d, gamma_r, u, v);
}

/* Sec. II-B-3: winner-take-all on a correlation (higher is better).
 * Reading: ties go to the smallest d.  *gap (optional) = best - second best. */
int orc_wta(const double *c, int D, double *gap) {
    int best = 0;
    for (int d = 1; d < D; ++d)
        if (MUT(7) ? c[d] >= c[best] : c[d] > c[best]) best = d;
    if (gap) {
        double second = -INFINITY;
        for (int d = 0; d < D; ++d)
            if (d != best && c[d] > second) second = c[d];
        *gap = (D > 1) ? c[best] - second : INFINITY;
    }
    return best;
}

/* Eq. 12: parabola through (d-1, d, d+1) of the aggregated left costs.
 * Reading: at d = 0 or d = D-1, or when the denominator is not negative
 * (no strict interior maximum), d^s = d.  *den (optional) receives the
 * denominator (0 at the ends). */
double orc_parabola(const double *c, int D, int d, double *den) {
    if (d <= 0 || d >= D - 1) {
        if (den) *den = 0.0;
        return (double)d;
    }
    const double cm = c[d - 1], c0 = c[d], cp = c[d + 1];
    const double q = 2.0 * cm + 2.0 * cp - 4.0 * c0;
    if (den) *den = q;
    if (!(q < 0.0)) return (double)d;
    return (double)d + (MUT(8) ? -1.0 : 1.0) * (cm - cp) / q;
}

/* Restricted search (the paper's Sec. IV plan: filter only the space around
 * previously calculated disparities).  Pixel p searches the window
 * [max(0, c - r), min(D - 1, c + r)] around its centre c (clamped to
 * 0..D-1) instead of 0..D-1: WTA and Eq. 12 as above with the window's ends
 * in the role of 0 and D - 1.  The aggregated costs are those of Eq. 8. */
static void search_window(int D, int centre, int radius, int *lo, int *hi) {
    const int c = clampi(centre, 0, D - 1);
    *lo = c - radius < 0 ? 0 : c - radius;
    *hi = c + radius - (MUT(16) ? 1 : 0) > D - 1 ? D - 1 : c + radius - (MUT(16) ? 1 : 0);
}

int orc_wta_window(const double *c, int lo, int hi, double *gap) {
    int best = lo;
    for (int d = lo + 1; d <= hi; ++d)
        if (MUT(7) ? c[d] >= c[best] : c[d] > c[best]) best = d;
    if (gap) {
        double second = -INFINITY;
        for (int d = lo; d <= hi; ++d)
            if (d != best && c[d] > second) second = c[d];
        *gap = (hi > lo) ? c[best] - second : INFINITY;
    }
    return best;
}

double orc_parabola_window(const double *c, int lo, int hi, int d, double *den) {
    if (d <= lo || d >= hi) {
        if (den) *den = 0.0;
        return (double)d;
    }
    const double cm = c[d - 1], c0 = c[d], cp = c[d + 1];
    const double q = 2.0 * cm + 2.0 * cp - 4.0 * c0;
    if (den) *den = q;
    if (!(q < 0.0)) return (double)d;
    return (double)d + (MUT(8) ? -1.0 : 1.0) * (cm - cp) / q;
}

/* Eq. 11 with a tolerance: pixel u of a row passes iff its match u - l_ref
 * lies in the image and the target map agrees there within lr_thresh. */
int orc_lr_valid(int u, int lref, const int32_t *ltar_row, double lr_thresh) {
    const int ur = u - lref;
    if (ur < 0) return 0;
    return fabs((double)(MUT(9) ? lref + ltar_row[ur] : lref - ltar_row[ur])) <= lr_thresh;
}

/* Sec. II-C: undo the perspective transform, d = d^s + alpha0 + alpha1*v - delta. */
double orc_postprocess(const orc_params *p, double ds, int v) {
    return MUT(10) ? ds - orc_row_shift(p, v) : ds + orc_row_shift(p, v);
}

/* Sec. II-D: 3-D point of left pixel (u,v) with disparity dfull.
 * Reading (the paper prints no formula): rectified pinhole pair in the left
 * camera frame, Z = f T / d, X = (u - u0) Z / f, Y = (v - v0) Z / f.
 * NaN when d is not finite or not positive. */
void orc_reconstruct(const orc_params *p, double dfull, int u, int v, double *X, double *Y, double *Z) {
    if (!isfinite(dfull) || dfull <= 0.0) {
        *X = *Y = *Z = NAN;
        return;
    }
    const double z = p->f_px * p->baseline / dfull;
    *Z = z;
    *X = ((double)u - p->u0) * z / p->f_px;
    *Y = ((double)(MUT(11) ? u : v) - p->v0) * z / p->f_px;
}

/* Raw NCC volumes for rows [y0, y1).
 * Left (reference) volume: cost_l(u,v,d) = NCC(left block u, right block u-d).
 * Right (target) volume:   cost_r(u,v,d) = NCC(left block u+d, right block u).
 * Both are evaluated from Eq. 3 directly; the identity of Sec. II-B-1,
 * cost_r(u-d,v,d) = cost_l(u,v,d), is a property tests check. */
static void cost_rows(const orc_params *p, const double *L, const double *R, int y0, int y1,
                      double *cl, double *cr, int row_base) {
    const int W = p->W, H = p->H, D = p->D;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int v = y0; v < y1; ++v) {
        for (int u = 0; u < W; ++u) {
            const size_t o = ((size_t)(v - row_base) * W + u) * D;
            for (int d = 0; d < D; ++d) {
                if (cl) cl[o + d] = orc_ncc(L, R, W, H, p->ncc_r, u, u - d, v);
                if (cr) cr[o + d] = orc_ncc(L, R, W, H, p->ncc_r, MUT(12) ? u - d : u + d, u, v);
            }
        }
    }
}

/* Full pipeline (Fig. 1 order) for output rows [row_begin, row_end); with
 * centre != NULL, every pixel of both views searches only its window around
 * centre[v*W+u] (see search_window).
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure. */
static int match_impl(const orc_params *p, const uint8_t *il, const uint8_t *ir,
                      const int32_t *centre, int radius, int row_begin, int row_end,
                      orc_outputs *out) {
    const int W = p->W, H = p->H, D = p->D, rho = p->agg_r;
    if (W < 1 || H < 1 || D < 1 || p->ncc_r < 0 || rho < 0) return -1;
    if (row_begin < 0) row_begin = 0;
    if (row_end > H) row_end = H;
    if (row_begin >= row_end) return 0;

    const size_t npx = (size_t)W * H;
    double *L = (double *)malloc(npx * sizeof(double));
    double *R = (double *)malloc(npx * sizeof(double));
    if (!L || !R) { free(L); free(R); return -2; }
    for (size_t i = 0; i < npx; ++i) L[i] = il[i];
    orc_warp(p, ir, R);
    if (out->warped) memcpy(out->warped, R, npx * sizeof(double));

    /* Block statistics (reported only; orc_ncc recomputes them by definition). */
    if (out->mu_l || out->sig_l || out->mu_r || out->sig_r) {
        #pragma omp parallel for schedule(static)
        for (int v = row_begin; v < row_end; ++v)
            for (int u = 0; u < W; ++u) {
                double m, s;
                const size_t i = (size_t)v * W + u;
                orc_block_stats(L, W, H, p->ncc_r, u, v, &m, &s);
                if (out->mu_l) out->mu_l[i] = m;
                if (out->sig_l) out->sig_l[i] = s;
                orc_block_stats(R, W, H, p->ncc_r, u, v, &m, &s);
                if (out->mu_r) out->mu_r[i] = m;
                if (out->sig_r) out->sig_r[i] = s;
            }
    }

    /* Cost rows needed by the aggregation window of the requested band. */
    const int cy0 = row_begin - rho < 0 ? 0 : row_begin - rho;
    const int cy1 = row_end + rho > H ? H : row_end + rho;
    double *cl, *cr;
    int base;
    if (out->cost_l && out->cost_r) {
        cl = out->cost_l; cr = out->cost_r; base = 0;
    } else {
        const size_t n = (size_t)(cy1 - cy0) * W * D;
        cl = (double *)malloc(n * sizeof(double));
        cr = (double *)malloc(n * sizeof(double));
        if (!cl || !cr) { free(cl); free(cr); free(L); free(R); return -2; }
        base = cy0;
    }
    cost_rows(p, L, R, cy0, cy1, cl, cr, base);
    if (base != 0) {
        /* Copy the band back if the caller asked for one of the volumes. */
        for (int v = cy0; v < cy1; ++v) {
            const size_t src = (size_t)(v - base) * W * D, dst = (size_t)v * W * D;
            if (out->cost_l) memcpy(out->cost_l + dst, cl + src, (size_t)W * D * sizeof(double));
            if (out->cost_r) memcpy(out->cost_r + dst, cr + src, (size_t)W * D * sizeof(double));
        }
    }

    /* Aggregation (Eqs. 8-10), WTA (Sec. II-B-3), parabola (Eq. 12). */
    int32_t *lbl_l = out->lbl_l ? out->lbl_l : (int32_t *)malloc(npx * sizeof(int32_t));
    int32_t *lbl_r = out->lbl_r ? out->lbl_r : (int32_t *)malloc(npx * sizeof(int32_t));
    double *dsub = out->dsub ? out->dsub : (double *)malloc(npx * sizeof(double));
    int err = (!lbl_l || !lbl_r || !dsub);
    if (!err) {
        /* Shift the volume pointers so that row v is addressed as v. */
        const double *vl = cl - (size_t)base * W * D;
        const double *vr = cr - (size_t)base * W * D;
        #pragma omp parallel
        {
            double *num = (double *)malloc((size_t)D * sizeof(double));
            double *al = (double *)malloc((size_t)D * sizeof(double));
            double *ar = (double *)malloc((size_t)D * sizeof(double));
            #pragma omp for schedule(dynamic, 1)
            for (int v = row_begin; v < row_end; ++v) {
                for (int u = 0; u < W; ++u) {
                    const size_t i = (size_t)v * W + u;
                    bilateral_all_d(vl, D, L, W, H, rho, p->gamma_d, p->gamma_r, u, v, num, al);
                    bilateral_all_d(vr, D, R, W, H, rho, p->gamma_d, p->gamma_r, u, v, num, ar);
                    if (out->agg_l) memcpy(out->agg_l + i * D, al, (size_t)D * sizeof(double));
                    if (out->agg_r) memcpy(out->agg_r + i * D, ar, (size_t)D * sizeof(double));
                    int lo = 0, hi = D - 1;
                    if (centre) search_window(D, centre[i], radius, &lo, &hi);
                    double g;
                    lbl_l[i] = orc_wta_window(al, lo, hi, &g);
                    if (out->gap_l) out->gap_l[i] = g;
                    lbl_r[i] = orc_wta_window(ar, lo, hi, &g);
                    if (out->gap_r) out->gap_r[i] = g;
                    double q;
                    dsub[i] = orc_parabola_window(al, lo, hi, lbl_l[i], &q);
                    if (out->den_l) out->den_l[i] = q;
                }
            }
            free(num); free(al); free(ar);
        }
        /* L-R check (Eq. 11), post-processing (Sec. II-C), 3-D (Sec. II-D). */
        for (int v = row_begin; v < row_end; ++v) {
            for (int u = 0; u < W; ++u) {
                const size_t i = (size_t)v * W + u;
                const int ok = orc_lr_valid(u, lbl_l[i], lbl_r + (size_t)v * W, p->lr_thresh);
                const double df = ok ? orc_postprocess(p, dsub[i], v) : NAN;
                if (out->valid) out->valid[i] = (uint8_t)ok;
                if (out->dfull) out->dfull[i] = df;
                if (out->xyz) {
                    double X, Y, Z;
                    orc_reconstruct(p, df, u, v, &X, &Y, &Z);
                    out->xyz[i] = X; out->xyz[npx + i] = Y; out->xyz[2 * npx + i] = Z;
                }
            }
        }
    }
    if (!out->lbl_l) free(lbl_l);
    if (!out->lbl_r) free(lbl_r);
    if (!out->dsub) free(dsub);
    if (base != 0) { free(cl); free(cr); }
    free(L); free(R);
    return err ? -2 : 0;
}

int orc_match(const orc_params *p, const uint8_t *il, const uint8_t *ir,
              int row_begin, int row_end, orc_outputs *out) {
    return match_impl(p, il, ir, NULL, 0, row_begin, row_end, out);
}

int orc_match_restricted(const orc_params *p, const uint8_t *il, const uint8_t *ir,
                         const int32_t *centre, int radius, int row_begin, int row_end,
                         orc_outputs *out) {
    if (!centre || radius < 0) return -1;
    return match_impl(p, il, ir, centre, radius, row_begin, row_end, out);
}

/* Aggregated cost vector at one pixel, every NCC value evaluated on demand
 * from Eq. 3 (no volume).  right = 0: reference view; right = 1: target view. */
static void agg_vector_direct(const orc_params *p, const double *L, const double *R, int right,
                              int u, int v, double *out) {
    const int W = p->W, H = p->H, D = p->D, rho = p->agg_r;
    const double *g = right ? R : L;
    const double gc = g[(size_t)v * W + u];
    double den = 0.0;
    for (int d = 0; d < D; ++d) out[d] = 0.0;
    for (int dy = -rho; dy <= rho; ++dy) {
        const int y = v + dy;
        if (y < 0 || y >= H) continue;
        for (int dx = -rho; dx <= rho; ++dx) {
            const int x = u + dx;
            if (x < 0 || x >= W) continue;
            const double wd = exp(-(double)(dx * dx + dy * dy) / (p->gamma_d * p->gamma_d));
            const double di = g[(size_t)y * W + x] - gc;
            const double wr = exp(-(di * di) / (p->gamma_r * p->gamma_r));
            for (int d = 0; d < D; ++d) {
                const double c = right ? orc_ncc(L, R, W, H, p->ncc_r, x + d, x, y)
                                       : orc_ncc(L, R, W, H, p->ncc_r, x, x - d, y);
                out[d] += wd * wr * c;
            }
            den += wd * wr;
        }
    }
    for (int d = 0; d < D; ++d) out[d] /= den;
}

/* The pipeline at n sampled pixels (us[i], vs[i]), each computed on its own
 * from the definitions (for checks at sizes where a full frame is slow).
 * Outputs (any may be NULL) are per sample: l_ref, l_tar at the matched
 * target pixel (or -1 if it lies outside), gaps, denominator, d^s, validity,
 * post-processed disparity.  Returns 0, or -1/-2 as orc_match. */
int orc_match_pixels(const orc_params *p, const uint8_t *il, const uint8_t *ir, int n,
                     const int32_t *us, const int32_t *vs, int32_t *lbl_l, int32_t *lbl_r_match,
                     double *gap_l, double *gap_r_match, double *den_l, double *dsub,
                     uint8_t *valid, double *dfull) {
    const int W = p->W, H = p->H, D = p->D;
    if (W < 1 || H < 1 || D < 1) return -1;
    const size_t npx = (size_t)W * H;
    double *L = (double *)malloc(npx * sizeof(double));
    double *R = (double *)malloc(npx * sizeof(double));
    if (!L || !R) { free(L); free(R); return -2; }
    for (size_t i = 0; i < npx; ++i) L[i] = il[i];
    orc_warp(p, ir, R);
    #pragma omp parallel
    {
        double *al = (double *)malloc((size_t)D * sizeof(double));
        double *ar = (double *)malloc((size_t)D * sizeof(double));
        #pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n; ++i) {
            const int u = us[i], v = vs[i];
            double g, q;
            agg_vector_direct(p, L, R, 0, u, v, al);
            const int ll = orc_wta(al, D, &g);
            if (gap_l) gap_l[i] = g;
            const double ds = orc_parabola(al, D, ll, &q);
            if (den_l) den_l[i] = q;
            if (lbl_l) lbl_l[i] = ll;
            if (dsub) dsub[i] = ds;
            int lr = -1, ok = 0;
            double gr = INFINITY;
            if (u - ll >= 0) {
                agg_vector_direct(p, L, R, 1, u - ll, v, ar);
                lr = orc_wta(ar, D, &gr);
                ok = fabs((double)(ll - lr)) <= p->lr_thresh;
            }
            if (lbl_r_match) lbl_r_match[i] = lr;
            if (gap_r_match) gap_r_match[i] = gr;
            if (valid) valid[i] = (uint8_t)ok;
            if (dfull) dfull[i] = ok ? orc_postprocess(p, ds, v) : NAN;
        }
        free(al); free(ar);
    }
    free(L); free(R);
    return 0;
}

/* ------------------------------------------------------------------------
 * Objective and gradient for refining the road plane (Sec. II-A, Eq. 2).
 *
 * L(alpha) = sum over pixels p with dstar[p] >= 0 of the aggregated reference
 * cost c_agg(p, dstar[p]) (Eq. 8), the disparities dstar held fixed.  Images
 * are real-valued here (double), so that derivatives with respect to pixel
 * values exist; ir is the original target image, warped inside.
 * ------------------------------------------------------------------------ */

/* Sec. II-A warp of a real-valued target image; also d(warped)/ds per pixel. */
static void warp_real(const orc_params *p, const double *ir, double *out, double *dds) {
    const int W = p->W, H = p->H;
    for (int v = 0; v < H; ++v) {
        const double s = orc_row_shift(p, v);
        const double k = floor(s);
        const double w = s - k;
        const int ki = (int)k;
        for (int x = 0; x < W; ++x) {
            const double a = ir[(size_t)v * W + clampi(x - ki, 0, W - 1)];
            const double b = ir[(size_t)v * W + clampi(x - ki - 1, 0, W - 1)];
            out[(size_t)v * W + x] = (1.0 - w) * a + w * b;
            if (dds) dds[(size_t)v * W + x] = b - a;   /* d/ds of (1-w) a + w b, w = s - k */
        }
    }
}

double orc_objective(const orc_params *p, const double *il, const double *ir, const int32_t *dstar) {
    const int W = p->W, H = p->H, rho = p->agg_r;
    double *R = (double *)malloc((size_t)W * H * sizeof(double));
    if (!R) return NAN;
    warp_real(p, ir, R, NULL);
    double L = 0.0;
    #pragma omp parallel for reduction(+ : L) schedule(dynamic, 1)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            const int d = dstar[(size_t)v * W + u];
            if (d < 0) continue;
            const double gc = il[(size_t)v * W + u];
            double num = 0.0, den = 0.0;
            for (int dy = -rho; dy <= rho; ++dy) {
                const int y = v + dy;
                if (y < 0 || y >= H) continue;
                for (int dx = -rho; dx <= rho; ++dx) {
                    const int x = u + dx;
                    if (x < 0 || x >= W) continue;
                    const double wd = exp(-(double)(dx * dx + dy * dy) / (p->gamma_d * p->gamma_d));
                    const double di = il[(size_t)y * W + x] - gc;
                    const double wr = exp(-(di * di) / (p->gamma_r * p->gamma_r));
                    num += wd * wr * orc_ncc(il, R, W, H, p->ncc_r, x, x - d, y);
                    den += wd * wr;
                }
            }
            L += num / den;
        }
    }
    free(R);
    return L;
}

/* Analytic gradient of orc_objective by the chain rule, in FP64:
 *   c_agg = sum_k w_k c_k / sum_k w_k, w_k = omega_d omega_r(i_l(n_k) - i_l(p))
 *     d c_agg / d c_k = w_k / W;  d c_agg / d w_k = (c_k - c_agg) / W;
 *     d omega_r / d delta = -2 delta / gamma_r^2 * omega_r            (Eq. 10)
 *   c = sum a b / (n sig_l sig_r), a, b the centred blocks            (Eq. 3)
 *     d c / d r_j = (a_j - c (sig_l / sig_r) b_j) / (n sig_l sig_r)
 *     d c / d l_j = (b_j - c (sig_r / sig_l) a_j) / (n sig_l sig_r)
 *   r = i_r'(x, v) = (1-w) i_r(x-k) + w i_r(x-k-1), s = alpha0 + alpha1 v - delta
 *     d r / d s = i_r(x-k-1) - i_r(x-k);  d s / d alpha = (1, v)
 * Writes L, dL/dalpha (2 values) and, when not NULL, dL/d i_l and dL/d i_r
 * (H*W each).  Returns 0, or -2 on allocation failure. */
int orc_grad(const orc_params *p, const double *il, const double *ir, const int32_t *dstar,
             double *L_out, double *dalpha, double *gl, double *gr) {
    const int W = p->W, H = p->H, rho = p->agg_r, r = p->ncc_r;
    const size_t npx = (size_t)W * H;
    const double n = (double)((2 * r + 1) * (2 * r + 1));
    double *R = (double *)malloc(npx * sizeof(double));
    double *dds = (double *)malloc(npx * sizeof(double));
    double *gR = (double *)calloc(npx, sizeof(double));     /* dL / d i_r' */
    double *gL = (double *)calloc(npx, sizeof(double));     /* dL / d i_l  */
    if (!R || !dds || !gR || !gL) { free(R); free(dds); free(gR); free(gL); return -2; }
    warp_real(p, ir, R, dds);
    double L = 0.0;
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            const int d = dstar[(size_t)v * W + u];
            if (d < 0) continue;
            const double gc = il[(size_t)v * W + u];
            /* weights and costs of the window */
            double wk[256], ck[256], dk[256];
            int xk[256], yk[256], m = 0;
            double Wsum = 0.0, num = 0.0;
            for (int dy = -rho; dy <= rho; ++dy) {
                const int y = v + dy;
                if (y < 0 || y >= H) continue;
                for (int dx = -rho; dx <= rho; ++dx) {
                    const int x = u + dx;
                    if (x < 0 || x >= W) continue;
                    const double wd = exp(-(double)(dx * dx + dy * dy) / (p->gamma_d * p->gamma_d));
                    const double di = il[(size_t)y * W + x] - gc;
                    const double wr = exp(-(di * di) / (p->gamma_r * p->gamma_r));
                    wk[m] = wd * wr;
                    dk[m] = di;
                    ck[m] = orc_ncc(il, R, W, H, r, x, x - d, y);
                    xk[m] = x;
                    yk[m] = y;
                    Wsum += wk[m];
                    num += wk[m] * ck[m];
                    ++m;
                }
            }
            const double cagg = num / Wsum;
            L += cagg;
            for (int k = 0; k < m; ++k) {
                /* through the weight w_k (guide = left image) */
                const double gw = (ck[k] - cagg) / Wsum * wk[k] *
                                  (-2.0 * dk[k] / (p->gamma_r * p->gamma_r));
                gL[(size_t)yk[k] * W + xk[k]] += MUT(13) ? -gw : gw;
                gL[(size_t)v * W + u] -= gw;
                /* through the cost c_k = NCC(left block n_k, right block n_k - d) */
                const double beta = wk[k] / Wsum;
                double mu_l, sg_l, mu_r, sg_r;
                const double var_l = orc_block_stats(il, W, H, r, xk[k], yk[k], &mu_l, &sg_l);
                const double var_r = orc_block_stats(R, W, H, r, xk[k] - d, yk[k], &mu_r, &sg_r);
                if (var_l < ORC_FLAT_VAR || var_r < ORC_FLAT_VAR) continue;   /* c == 0 */
                const double c = ck[k], den = n * sg_l * sg_r;
                for (int j = -r; j <= r; ++j) {
                    const int y = clampi(yk[k] + j, 0, H - 1);
                    for (int i = -r; i <= r; ++i) {
                        const size_t li = (size_t)y * W + clampi(xk[k] + i, 0, W - 1);
                        const size_t ri = (size_t)y * W + clampi(xk[k] - d + i, 0, W - 1);
                        const double a = il[li] - mu_l, b = R[ri] - mu_r;
                        gR[ri] += beta * (a - c * (sg_l / sg_r) * b) / den;
                        gL[li] += beta * (b - c * (sg_r / sg_l) * a) / den;
                    }
                }
            }
        }
    }
    double g0 = 0.0, g1 = 0.0;
    for (int v = 0; v < H; ++v)
        for (int x = 0; x < W; ++x) {
            const double t = gR[(size_t)v * W + x] * dds[(size_t)v * W + x];
            g0 += t;
            g1 += t * (double)v;
        }
    if (L_out) *L_out = L;
    if (dalpha) { dalpha[0] = g0; dalpha[1] = g1; }
    if (gl) memcpy(gl, gL, npx * sizeof(double));
    if (gr) {
        /* adjoint of the warp: i_r'(x) = (1-w) i_r(x-k) + w i_r(x-k-1) */
        memset(gr, 0, npx * sizeof(double));
        for (int v = 0; v < H; ++v) {
            const double s = orc_row_shift(p, v);
            const double k = floor(s), w = s - k;
            const int ki = (int)k;
            for (int x = 0; x < W; ++x) {
                const double g = gR[(size_t)v * W + x];
                gr[(size_t)v * W + clampi(x - ki, 0, W - 1)] += (1.0 - w) * g;
                gr[(size_t)v * W + clampi(x - ki - 1, 0, W - 1)] += w * g;
            }
        }
    }
    free(R); free(dds); free(gR); free(gL);
    return 0;
}

/* ------------------------------------------------------------------------
 * Road-plane fitting from a disparity map (Sec. II-A): alpha of Eq. 2 by
 * least squares with RANSAC, and the roll angle from a linear plane fitted
 * to a near-field patch.  The correspondences are the valid pixels of a
 * full-disparity map d[H][W] (NaN = rejected) instead of ORB matches.
 * ------------------------------------------------------------------------ */

/* Two-point model of hypothesis (i1, i2) (pixel indices v*W+u): the line
 * d = a0 + a1 v through both points, in double.  Returns 0 if either point is
 * invalid or both lie on one row. */
static int line_through(const float *disp, int W, int i1, int i2, double *a0, double *a1) {
    const double d1 = disp[i1], d2 = disp[i2];
    const int v1 = i1 / W, v2 = i2 / W;
    if (isnan(d1) || isnan(d2) || v1 == v2) return 0;
    *a1 = (d2 - d1) / (double)(v2 - v1);
    *a0 = d1 - *a1 * (double)v1;
    return 1;
}

/* Inlier test of pixel (v, d) against the model d = a0 + a1 v, in double
 * precision: |d - (a0 + a1 v)| <= tau (the definition; the disparity map
 * itself is float). */
static int is_inlier(float d, int v, double a0, double a1, double tau) {
    return !isnan(d) && fabs((double)d - (a0 + a1 * (double)v)) <= tau;
}

/* RANSAC over n_hyp given point pairs (pairs[2h], pairs[2h+1]): counts[h] =
 * inliers of hypothesis h (-1 if it has no model); the best hypothesis has
 * the most inliers (ties: the smallest h); alpha = least-squares line through
 * its inliers (normal equations in double).  Returns the best h, or -1 if no
 * hypothesis has a model or the inliers span fewer than two rows. */
int orc_fit_alpha(const float *disp, int W, int H, int n_hyp, const int32_t *pairs, float tau,
                  int32_t *counts, double *alpha, int32_t *n_inliers) {
    const size_t npx = (size_t)W * H;
    int best = -1, best_n = -1;
    for (int h = 0; h < n_hyp; ++h) {
        double a0, a1;
        const int i1 = pairs[2 * h], i2 = pairs[2 * h + 1];
        if (i1 < 0 || i2 < 0 || (size_t)i1 >= npx || (size_t)i2 >= npx ||
            !line_through(disp, W, i1, i2, &a0, &a1)) {
            counts[h] = -1;
            continue;
        }
        int32_t c = 0;
        for (size_t i = 0; i < npx; ++i) c += is_inlier(disp[i], (int)(i / W), a0, a1, tau);
        counts[h] = c;
        if (c > best_n) { best_n = c; best = h; }
    }
    if (n_inliers) *n_inliers = best_n < 0 ? 0 : best_n;
    if (best < 0) return -1;
    double a0, a1;
    line_through(disp, W, pairs[2 * best], pairs[2 * best + 1], &a0, &a1);
    double s0 = 0, s1 = 0, s2 = 0, t0 = 0, t1 = 0;   /* n, sum v, sum v^2, sum d, sum v d */
    for (size_t i = 0; i < npx; ++i) {
        const int v = (int)(i / W);
        if (!is_inlier(disp[i], v, a0, a1, tau)) continue;
        const double d = disp[i];
        s0 += 1.0; s1 += v; s2 += (double)v * v; t0 += d; t1 += (double)v * d;
    }
    const double det = s0 * s2 - s1 * s1;
    if (det == 0.0) return -1;
    alpha[1] = (MUT(14) ? s1 * t0 - s0 * t1 : s0 * t1 - s1 * t0) / det;
    alpha[0] = (t0 - alpha[1] * s1) / s0;
    return best;
}

/* Roll: least-squares plane d = g0 + g1 u + g2 v over the valid pixels of the
 * patch [u_lo, u_hi) x [v_lo, v_hi); gamma = atan(-g1 / g2).  Solves the 3x3
 * normal equations by Gaussian elimination with partial pivoting.  Returns
 * the number of pixels used, or -1 if the system is singular. */
int orc_fit_roll(const float *disp, int W, int H, int u_lo, int v_lo, int u_hi, int v_hi,
                 double *g, double *roll) {
    double A[3][4] = {{0}};
    int n = 0;
    for (int v = v_lo < 0 ? 0 : v_lo; v < v_hi && v < H; ++v)
        for (int u = u_lo < 0 ? 0 : u_lo; u < u_hi && u < W; ++u) {
            const float df = disp[(size_t)v * W + u];
            if (isnan(df)) continue;
            const double x[3] = {1.0, (double)u, (double)v}, d = df;
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c) A[r][c] += x[r] * x[c];
                A[r][3] += x[r] * d;
            }
            ++n;
        }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int k = 0; k < 4; ++k) { const double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        for (int r = c + 1; r < 3; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = A[r][3];
        for (int k = r + 1; k < 3; ++k) s -= A[r][k] * g[k];
        g[r] = s / A[r][r];
    }
    *roll = atan((MUT(15) ? g[1] : -g[1]) / g[2]);
    return n;
}
