/*
 * FP64 CPU oracle of the adaptive-denoising event simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library, and nothing in the library calls it.  It is written
 * for clarity, not speed: plain loops in double precision, with OpenMP over
 * pixels so that full-size frames finish in reasonable time.
 *
 * What it computes (paper sections and equations):
 *   Eq. 1        event when Delta L = L(t) - L(t_last) reaches p*C;
 *                n = floor(|Delta L| / C) events per frame, L_last += p*n*C.
 *   Sec. 1.1     L = log E, here y = ln(Y + eps), Y luminance (Rec.709 for RGB).
 *   Eqs. 3-5     first-order weighted local regression around the centre
 *                feature x^c: minimise (1/W) sum_i w^i (y^i - alpha -
 *                beta^T (x^i - x^c))^2 with a product Gaussian kernel
 *                w^i = prod_j exp(-((x^i_j - x^c_j) / (h b_j))^2 / 2).
 *                A ridge lambda * |beta|^2 is added to that normalised
 *                objective (the paper leaves the Gram matrix unregularised;
 *                flat regions make feature columns vanish).  The solve is a
 *                Householder QR of the sqrt(w)-weighted design matrix stacked
 *                on sqrt(lambda W) [0 | I].
 *   Sec. 3       9-D feature: image coordinate (2), normal (3), depth (1),
 *                texture colour (3).  Brightness is not a feature.
 *   Eqs. 6-9     Proposition 1: with the model (alpha, beta, x^c) kept from the
 *                last event, Delta R = (beta^T (x^c - xhat^c))^2; the pixel is
 *                flagged for a new regression when Delta R >= C^2.
 *   Fig. 1, Sec. 3  the model is kept until a new event is detected.
 *
 * Windows: spatial |q - c|_inf <= r clipped to the image, temporal frames
 * max(0, t-T+1) .. t; the coordinate offset is (q - c) / r unless raw pixel
 * units are requested.  Frame 0 regresses every pixel and only initialises
 * L_last and the model.
 */
#include "esim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF 7          /* feature dimensions besides the image coordinate */
#define ND 9          /* regressors: dx, dy, 7 features                  */
#define NP 10         /* unknowns: alpha, beta_1..beta_9                   */

struct or_sim {
    or_config cfg;
    int64_t n;            /* pixels                                        */
    int32_t t;            /* frames pushed                                 */
    double* y;            /* ring [T][n] log brightness                    */
    double* x;            /* ring [T][NF][n] features                      */
    double* l_last;       /* [n]                                           */
    double* beta;         /* [n][ND]                                       */
    double* xc;           /* [n][NF]                                       */
    double* alpha_o;      /* [n] outputs of the last frame                 */
    double* stat_o;
    double* dl_o;
    int32_t* nev_o;
    uint8_t* flag_o;
    int32_t* ev;          /* events [ev_n][4]                              */
    int64_t ev_n, ev_cap;
};

int32_t or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

or_sim* or_create(const or_config* cfg)
{
    if (!cfg || cfg->width <= 0 || cfg->height <= 0 || cfg->radius < 1 || cfg->frames < 1 ||
        !(cfg->contrast > 0) || !(cfg->h > 0) || cfg->ridge < 0 ||
        (cfg->channels != 0 && cfg->channels != 1 && cfg->channels != 3))
        return NULL;
    for (int j = 0; j < NF; ++j)
        if (!(cfg->bandwidth[j] > 0)) return NULL;
    or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
    s->cfg = *cfg;
    s->n = (int64_t)cfg->width * cfg->height;
    int64_t n = s->n, T = cfg->frames;
    s->y = (double*)calloc((size_t)(T * n), sizeof(double));
    s->x = (double*)calloc((size_t)(T * NF * n), sizeof(double));
    s->l_last = (double*)calloc((size_t)n, sizeof(double));
    s->beta = (double*)calloc((size_t)(n * ND), sizeof(double));
    s->xc = (double*)calloc((size_t)(n * NF), sizeof(double));
    s->alpha_o = (double*)calloc((size_t)n, sizeof(double));
    s->stat_o = (double*)calloc((size_t)n, sizeof(double));
    s->dl_o = (double*)calloc((size_t)n, sizeof(double));
    s->nev_o = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    s->flag_o = (uint8_t*)calloc((size_t)n, sizeof(uint8_t));
    return s;
}

void or_destroy(or_sim* s)
{
    if (!s) return;
    free(s->y); free(s->x); free(s->l_last); free(s->beta); free(s->xc);
    free(s->alpha_o); free(s->stat_o); free(s->dl_o); free(s->nev_o); free(s->flag_o);
    free(s->ev);
    free(s);
}

/* y and x of frame tau (tau in the ring) at pixel p */
static double ring_y(const or_sim* s, int32_t tau, int64_t p)
{
    return s->y[(int64_t)(tau % s->cfg.frames) * s->n + p];
}

static double ring_x(const or_sim* s, int32_t tau, int j, int64_t p)
{
    return s->x[((int64_t)(tau % s->cfg.frames) * NF + j) * s->n + p];
}

/*
 * Householder QR least squares: minimise |A theta - b| for A (m x NP) stored
 * row-major in a[m][NP], b[m].  A and b are overwritten.  Returns 0, or -1 if
 * a column is (numerically) zero.
 */
static int qr_solve(double* a, double* b, int64_t m, double* theta)
{
    for (int k = 0; k < NP; ++k) {
        double norm = 0.0;
        for (int64_t i = k; i < m; ++i) norm += a[i * NP + k] * a[i * NP + k];
        norm = sqrt(norm);
        if (norm == 0.0) return -1;
        double akk = a[k * NP + k];
        double alpha = akk > 0 ? -norm : norm;          /* R_kk */
        /* v = x - alpha e_k, stored in column k rows k..m-1 */
        a[k * NP + k] = akk - alpha;
        double vtv = 0.0;
        for (int64_t i = k; i < m; ++i) vtv += a[i * NP + k] * a[i * NP + k];
        /* apply H = I - 2 v v^T / v^T v to columns k+1.. and to b */
        for (int c = k + 1; c < NP; ++c) {
            double dot = 0.0;
            for (int64_t i = k; i < m; ++i) dot += a[i * NP + k] * a[i * NP + c];
            double f = 2.0 * dot / vtv;
            for (int64_t i = k; i < m; ++i) a[i * NP + c] -= f * a[i * NP + k];
        }
        double dot = 0.0;
        for (int64_t i = k; i < m; ++i) dot += a[i * NP + k] * b[i];
        double f = 2.0 * dot / vtv;
        for (int64_t i = k; i < m; ++i) b[i] -= f * a[i * NP + k];
        a[k * NP + k] = alpha;                          /* keep R_kk on the diagonal */
    }
    /* back substitution R theta = (Q^T b)[0..NP) */
    for (int k = NP - 1; k >= 0; --k) {
        double acc = b[k];
        for (int c = k + 1; c < NP; ++c) acc -= a[k * NP + c] * theta[c];
        theta[k] = acc / a[k * NP + k];
    }
    return 0;
}

/*
 * Weighted local regression (Eqs. 3-5) at centre (cx, cy) of frame t (the last
 * pushed frame).  Workspace a[(m + ND) * NP], b[m + ND], z[m * NP], yw[m], w[m]
 * with m >= (2r+1)^2 T.  Returns 0 and fills theta, R, W.
 */
static int wlr(const or_sim* s, int32_t cx, int32_t cy, double* a, double* b, double* zs,
               double* ys, double* ws, double* theta, double* R_out, double* W_out)
{
    const or_config* c = &s->cfg;
    const int32_t t = s->t - 1;
    const int32_t r = c->radius;
    const double unit = c->pixel_units ? 1.0 : (double)r;
    const int64_t pc = (int64_t)cy * c->width + cx;
    double xcen[NF];
    for (int j = 0; j < NF; ++j) xcen[j] = ring_x(s, t, j, pc);
    double hb[ND];
    hb[0] = c->h;                                   /* coordinate bandwidths b = 1 */
    hb[1] = c->h;
    for (int j = 0; j < NF; ++j) hb[2 + j] = c->h * c->bandwidth[j];

    int32_t tau0 = t - c->frames + 1;
    if (tau0 < 0) tau0 = 0;
    int64_t m = 0;
    double W = 0.0;
    for (int32_t tau = tau0; tau <= t; ++tau) {
        for (int32_t qy = cy - r; qy <= cy + r; ++qy) {
            if (qy < 0 || qy >= c->height) continue;
            for (int32_t qx = cx - r; qx <= cx + r; ++qx) {
                if (qx < 0 || qx >= c->width) continue;
                int64_t q = (int64_t)qy * c->width + qx;
                double d[ND];
                d[0] = (qx - cx) / unit;
                d[1] = (qy - cy) / unit;
                for (int j = 0; j < NF; ++j) d[2 + j] = ring_x(s, tau, j, q) - xcen[j];
                double u = 0.0;
                for (int j = 0; j < ND; ++j) u += (d[j] / hb[j]) * (d[j] / hb[j]);
                double w = exp(-0.5 * u);               /* product of Gaussians, Eq. 5 */
                double sw = sqrt(w);
                double* z = zs + m * NP;
                z[0] = 1.0;
                for (int j = 0; j < ND; ++j) z[1 + j] = d[j];
                ys[m] = ring_y(s, tau, q);
                ws[m] = w;
                for (int k = 0; k < NP; ++k) a[m * NP + k] = sw * z[k];
                b[m] = sw * ys[m];
                W += w;
                ++m;
            }
        }
    }
    /* ridge rows: sqrt(lambda W) e_k for the slope unknowns k = 1..9 */
    int64_t rows = m;
    if (c->ridge > 0) {
        double sr = sqrt(c->ridge * W);
        for (int k = 1; k < NP; ++k) {
            for (int q = 0; q < NP; ++q) a[rows * NP + q] = (q == k) ? sr : 0.0;
            b[rows] = 0.0;
            ++rows;
        }
    }
    if (qr_solve(a, b, rows, theta) != 0) return -1;
    double R = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double f = 0.0;
        for (int k = 0; k < NP; ++k) f += zs[i * NP + k] * theta[k];
        R += ws[i] * (ys[i] - f) * (ys[i] - f);
    }
    *R_out = R / W;
    *W_out = W;
    return 0;
}

static int64_t window_rows(const or_config* c)
{
    int64_t side = 2 * (int64_t)c->radius + 1;
    return side * side * c->frames;
}

int or_wlr_at(const or_sim* s, int32_t cx, int32_t cy, double* theta10, double* R, double* W)
{
    if (!s || s->t < 1 || cx < 0 || cy < 0 || cx >= s->cfg.width || cy >= s->cfg.height) return -1;
    int64_t m = window_rows(&s->cfg);
    double* a = (double*)malloc(sizeof(double) * (size_t)((m + ND) * NP));
    double* b = (double*)malloc(sizeof(double) * (size_t)(m + ND));
    double* z = (double*)malloc(sizeof(double) * (size_t)(m * NP));
    double* yv = (double*)malloc(sizeof(double) * (size_t)m);
    double* wv = (double*)malloc(sizeof(double) * (size_t)m);
    int rc = wlr(s, cx, cy, a, b, z, yv, wv, theta10, R, W);
    free(a); free(b); free(z); free(yv); free(wv);
    return rc;
}

static void ingest(or_sim* s, const float* radiance, const float* normal, const float* albedo,
                   const float* depth)
{
    const or_config* c = &s->cfg;
    const int64_t n = s->n;
    const int32_t slot = s->t % c->frames;
    double* y = s->y + (int64_t)slot * n;
    double* x = s->x + (int64_t)slot * NF * n;
    for (int64_t p = 0; p < n; ++p) {
        if (c->channels == 0) {
            y[p] = (double)radiance[p];
        } else {
            double Y = (c->channels == 3)
                ? 0.2126 * radiance[p] + 0.7152 * radiance[n + p] + 0.0722 * radiance[2 * n + p]
                : (double)radiance[p];
            y[p] = log(Y + c->log_eps);
        }
        x[0 * n + p] = normal[p];
        x[1 * n + p] = normal[n + p];
        x[2 * n + p] = normal[2 * n + p];
        x[3 * n + p] = depth[p];
        x[4 * n + p] = albedo[p];
        x[5 * n + p] = albedo[n + p];
        x[6 * n + p] = albedo[2 * n + p];
    }
}

static void push_event(or_sim* s, int32_t t, int32_t x, int32_t y, int32_t p)
{
    if (s->ev_n == s->ev_cap) {
        s->ev_cap = s->ev_cap ? 2 * s->ev_cap : 1024;
        s->ev = (int32_t*)realloc(s->ev, sizeof(int32_t) * 4 * (size_t)s->ev_cap);
    }
    int32_t* e = s->ev + 4 * s->ev_n++;
    e[0] = t; e[1] = x; e[2] = y; e[3] = p;
}

int or_push(or_sim* s, const float* radiance, const float* normal, const float* albedo,
            const float* depth, int32_t row0, int32_t row1)
{
    return or_push_var(s, radiance, NULL, normal, albedo, depth, row0, row1);
}

int or_push_var(or_sim* s, const float* radiance, const float* variance, const float* normal,
                const float* albedo, const float* depth, int32_t row0, int32_t row1)
{
    if (!s || !radiance || !normal || !albedo || !depth) return -1;
    const or_config* c = &s->cfg;
    if (row1 < 0 || row1 > c->height) row1 = c->height;
    if (row0 < 0) row0 = 0;
    ingest(s, radiance, normal, albedo, depth);
    const int32_t t = s->t;
    s->t += 1;
    const int64_t n = s->n;
    const int32_t W = c->width;
    const double C = c->contrast;
    const double nan = NAN;
    for (int64_t p = 0; p < n; ++p) {
        s->alpha_o[p] = nan; s->stat_o[p] = nan; s->dl_o[p] = nan;
        s->nev_o[p] = 0; s->flag_o[p] = 0;
    }
    const int64_t m = window_rows(c);
    int failed = 0;
#pragma omp parallel reduction(|:failed)
    {
        double* a = (double*)malloc(sizeof(double) * (size_t)((m + ND) * NP));
        double* b = (double*)malloc(sizeof(double) * (size_t)(m + ND));
        double* z = (double*)malloc(sizeof(double) * (size_t)(m * NP));
        double* yv = (double*)malloc(sizeof(double) * (size_t)m);
        double* wv = (double*)malloc(sizeof(double) * (size_t)m);
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = (int64_t)row0 * W; p < (int64_t)row1 * W; ++p) {
            int32_t cx = (int32_t)(p % W), cy = (int32_t)(p / W);
            double xnow[NF];
            for (int j = 0; j < NF; ++j) xnow[j] = ring_x(s, t, j, p);
            int run = 1;
            if (t > 0 && c->mode == 0) {
                /* Proposition 1: Delta R = (beta^T (x^c - xhat^c))^2 against C^2;
                 * the coordinate part of x^c - xhat^c is zero (same pixel). */
                double st = 0.0;
                for (int j = 0; j < NF; ++j) st += s->beta[p * ND + 2 + j] * (s->xc[p * NF + j] - xnow[j]);
                s->stat_o[p] = st;
                run = (st * st >= C * C);
                if (!run && c->guard_kappa > 0) {
                    /* guard: the log brightness itself moved past C by more than
                     * guard_kappa deviations; sigma_y = sqrt(Var[Y]) / (Y + eps)
                     * with Y + eps = exp(y) */
                    const double yc = ring_y(s, t, p);
                    const double sig = variance ? sqrt(fmax((double)variance[p], 0.0)) / exp(yc) : 0.0;
                    run = fabs(yc - s->l_last[p]) >= C + c->guard_kappa * sig;
                }
            }
            if (!run) continue;
            double theta[NP], R, Wsum;
            if (wlr(s, cx, cy, a, b, z, yv, wv, theta, &R, &Wsum) != 0) { failed = 1; continue; }
            s->flag_o[p] = 1;
            s->alpha_o[p] = theta[0];
            if (t == 0) {
                /* initialisation: brightness reference and model, no events */
                s->l_last[p] = theta[0];
                for (int j = 0; j < ND; ++j) s->beta[p * ND + j] = theta[1 + j];
                for (int j = 0; j < NF; ++j) s->xc[p * NF + j] = xnow[j];
                continue;
            }
            /* Eq. 1 at a fixed frame time: n = floor(|dL| / C) crossings */
            double dl = theta[0] - s->l_last[p];
            s->dl_o[p] = dl;
            double k = floor(fabs(dl) / C);
            if (k >= 1.0) {
                int32_t pol = dl > 0 ? 1 : -1;
                s->nev_o[p] = pol * (int32_t)k;
                s->l_last[p] += pol * k * C;
                for (int j = 0; j < ND; ++j) s->beta[p * ND + j] = theta[1 + j];
                for (int j = 0; j < NF; ++j) s->xc[p * NF + j] = xnow[j];
            }
        }
        free(a); free(b); free(z); free(yv); free(wv);
    }
    if (failed) return -2;
    /* canonical event order: frame, row, column, repeat */
    for (int64_t p = 0; p < n; ++p) {
        int32_t k = s->nev_o[p];
        int32_t pol = k > 0 ? 1 : -1;
        for (int32_t i = 0; i < abs(k); ++i) push_event(s, t, (int32_t)(p % W), (int32_t)(p / W), pol);
    }
    return 0;
}

void or_frame_outputs(const or_sim* s, double* alpha, double* stat, double* dl, int32_t* nev,
                      uint8_t* flag)
{
    size_t n = (size_t)s->n;
    if (alpha) memcpy(alpha, s->alpha_o, n * sizeof(double));
    if (stat) memcpy(stat, s->stat_o, n * sizeof(double));
    if (dl) memcpy(dl, s->dl_o, n * sizeof(double));
    if (nev) memcpy(nev, s->nev_o, n * sizeof(int32_t));
    if (flag) memcpy(flag, s->flag_o, n * sizeof(uint8_t));
}

int64_t or_event_count(const or_sim* s) { return s->ev_n; }

int64_t or_take_events(or_sim* s, int32_t* dst, int64_t cap)
{
    int64_t k = s->ev_n < cap ? s->ev_n : cap;
    memcpy(dst, s->ev, sizeof(int32_t) * 4 * (size_t)k);
    /* keep any events that did not fit */
    memmove(s->ev, s->ev + 4 * k, sizeof(int32_t) * 4 * (size_t)(s->ev_n - k));
    s->ev_n -= k;
    return k;
}

void or_get_state(const or_sim* s, double* l_last, double* beta9, double* xc7)
{
    size_t n = (size_t)s->n;
    if (l_last) memcpy(l_last, s->l_last, n * sizeof(double));
    if (beta9) memcpy(beta9, s->beta, n * ND * sizeof(double));
    if (xc7) memcpy(xc7, s->xc, n * NF * sizeof(double));
}

void or_set_state_pixel(or_sim* s, int64_t idx, double l_last, const double* beta9,
                        const double* xc7)
{
    if (idx < 0 || idx >= s->n) return;
    s->l_last[idx] = l_last;
    if (beta9) for (int j = 0; j < ND; ++j) s->beta[idx * ND + j] = beta9[j];
    if (xc7) for (int j = 0; j < NF; ++j) s->xc[idx * NF + j] = xc7[j];
}

void or_set_state(or_sim* s, const double* l_last, const double* beta9, const double* xc7)
{
    size_t n = (size_t)s->n;
    if (l_last) memcpy(s->l_last, l_last, n * sizeof(double));
    if (beta9) memcpy(s->beta, beta9, n * ND * sizeof(double));
    if (xc7) memcpy(s->xc, xc7, n * NF * sizeof(double));
}
