/*
 * FP64 CPU oracle of the adaptive-denoising event simulator (test
 * infrastructure only: it exists to check the CUDA path and is never part of
 * it).  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load it.
 *
 * It restates, step by step and in double precision, what the method computes
 * for each frame (Section 2 of the paper):
 *   - log brightness y = ln(Y + eps) (Section 1.1, Section 2.1),
 *   - the likelihood test of Proposition 1 / Eq. 9 on pixels that keep a model,
 *   - the weighted local regression of Eqs. 3-5 at flagged pixels, solved by
 *     Householder QR on the sqrt(w)-weighted, ridge-augmented design matrix,
 *   - DVS events by Eq. 1 at fixed frame times (Section 3 footnote).
 */
#ifndef ESIM_ORACLE_H
#define ESIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_config {
    int32_t width, height;
    int32_t radius;       /* spatial window half-size r: (2r+1)^2 pixels      */
    int32_t frames;       /* temporal window T: frames t-T+1 .. t            */
    int32_t channels;     /* radiance channels: 1 luminance, 3 RGB, 0 = log */
    int32_t mode;         /* 0 adaptive (Prop. 1 test), 1 exhaustive WLR     */
    int32_t pixel_units;  /* 0: coordinate offset / r ; 1: raw pixels         */
    int32_t pad_;
    double contrast;      /* C of Eq. 1                                      */
    double h;             /* global bandwidth h of Eq. 5                     */
    double bandwidth[7];  /* b_j of the 7 feature dimensions (coords: 1)     */
    double log_eps;       /* eps in y = ln(Y + eps)                          */
    double ridge;         /* lambda: objective gets + lambda * W * |beta|^2   */
    double guard_kappa;   /* optional variance guard (a project extension, not
                             in the paper): > 0 also regresses a pixel whose
                             |y_t(c) - L_last| >= C + guard_kappa * sigma_y,
                             sigma_y = sqrt(Var[Y]) / (Y + eps); <= 0: off   */
} or_config;

typedef struct or_sim or_sim;

or_sim* or_create(const or_config* cfg);
void    or_destroy(or_sim* s);

/* Push frame t (= number of frames pushed before).  Planar float32 inputs:
 * radiance [channels][H][W] (or [H][W] log brightness when channels == 0),
 * normal [3][H][W], albedo [3][H][W], depth [H][W].  Only pixels in rows
 * [row0, row1) are tested / regressed / emitted; row1 < 0 means all rows.
 * Returns 0, or -1 on a bad argument. */
int     or_push(or_sim* s, const float* radiance, const float* normal,
                const float* albedo, const float* depth, int32_t row0, int32_t row1);

/* or_push with the frame's luminance variance [H][W] for the guard (may be
 * NULL: sigma_y = 0). */
int     or_push_var(or_sim* s, const float* radiance, const float* variance, const float* normal,
                    const float* albedo, const float* depth, int32_t row0, int32_t row1);

/* Per-pixel results of the last pushed frame (any pointer may be NULL):
 * alpha (NaN where no regression ran), stat = beta^T (x^c - xhat^c) of the
 * test (NaN where not evaluated), dl = alpha - L_last before emission (NaN
 * where no regression ran), nev = signed event count p*n, flag = 1 where the
 * regression ran. */
void    or_frame_outputs(const or_sim* s, double* alpha, double* stat, double* dl,
                         int32_t* nev, uint8_t* flag);

/* Events accumulated since the last take, canonical order (t, y, x, repeat);
 * each as 4 int32: frame, x, y, polarity. Returns how many were copied. */
int64_t or_event_count(const or_sim* s);
int64_t or_take_events(or_sim* s, int32_t* dst, int64_t cap);

/* Per-pixel model: L_last, beta (9: dx, dy, 7 features), x^c (7 features). */
void    or_get_state(const or_sim* s, double* l_last, double* beta9, double* xc7);
void    or_set_state_pixel(or_sim* s, int64_t idx, double l_last, const double* beta9,
                           const double* xc7);
/* Overwrite the model of every pixel (any pointer may be NULL to keep that part). */
void    or_set_state(or_sim* s, const double* l_last, const double* beta9, const double* xc7);

/* The regression of Eqs. 4-5 at pixel (cx, cy) of the last pushed frame:
 * theta = (alpha, beta_1..beta_9), R of Eq. 4, W of Eq. 5. Returns 0 or -1. */
int     or_wlr_at(const or_sim* s, int32_t cx, int32_t cy, double* theta10, double* R,
                  double* W);

int32_t or_threads(void);
/* OpenMP threads for the calls that follow (n > 0); timing only. */
void    or_set_threads(int32_t n);

#ifdef __cplusplus
}
#endif
#endif
