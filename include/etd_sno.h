/*
 * etd_sno.h - C ABI of the spectral neural operator (SNO) and of the Parareal loop that uses it as
 * its coarse propagator, with batched ETDRK2 (eq. (2.14), the EIFE2 scheme) as the fine one.
 *
 * The paper has no learned component: this is an accelerator around its method. The SNO maps a
 * field u on the interior nodes of an N x N mesh (unit square, homogeneous Dirichlet) and the
 * diffusion coefficient D of u_t = D Lap u + u - u^3 to a prediction of u a fixed number of ETDRK2
 * steps later. It works in the sine eigenbasis of Section 4, truncated to the lowest M modes per
 * axis, S_M[p][j] = sqrt(2/N) sin((p+1)(j+1) pi / N):
 *   a = (ln D - ln 1e-3) / ln 100;  h_0[c] = Wl[c][0] u + Wl[c][1] a + bl[c]   (c < C)
 *   layers l < L:  hh = bf16(S_M h_l S_M^T);  gh[o][p][q] = sum_c bf16(Wm[l][p][q][o][c]) hh[c][p][q];
 *                  z = S_M^T gh S_M + sum_c Wp[l][o][c] h_l[c] + bp[l][o];  h_{l+1} = gelu(z)
 *   u_hat = u + sum_c Wq[c] h_L[c] + bq
 * (bf16: round to nearest even; gelu(z) = z (1 + erf(z / sqrt 2)) / 2). FP32 everywhere else.
 *
 * Conventions: fields are DEVICE float32 arrays of B x (N-1) x (N-1) values (x fastest), D arrays
 * are HOST doubles. Calls are asynchronous on `stream` unless stated. Errors as in etd.h
 * (etd_last_error() gives the detail); no call aborts.
 */
#ifndef ETD_SNO_H
#define ETD_SNO_H

#include <stdint.h>

#include "etd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etd_sno_s* etd_sno;

/* Create an operator for N intervals per axis (N even, 8 <= N <= 2048), C channels (1..256), M
 * modes per axis (1 <= M < N), L layers (1..16), for batches of up to max_batch fields. Allocates
 * the parameters (zeroed; set them with etd_sno_set_params), the Adam moments and the activations
 * for max_batch fields. ETD_ERR_INVALID_ARG, ETD_ERR_OOM, ETD_ERR_CUDA. */
etd_status etd_sno_create(etd_sno* out, int N, int C, int M, int L, int max_batch);

/* Number of float32 parameters, laid out as Wl[C][2], bl[C], Wm[L][M][M][C][C], Wp[L][C][C],
 * bp[L][C], Wq[C], bq[1]. */
int64_t etd_sno_param_count(etd_sno s);

/* Copy all parameters from / to HOST memory (param_count floats, the layout above); both
 * synchronise. set_params also resets the Adam state (moments and step count). */
etd_status etd_sno_set_params(etd_sno s, const float* host);
etd_status etd_sno_get_params(etd_sno s, float* host);

/* u_hat for B <= max_batch fields u (device) with coefficients D[B] (host); writes out (device,
 * may not alias u). */
etd_status etd_sno_forward(etd_sno s, const float* u, const double* D, int B, float* out, void* stream);

/* One training step on a batch: forward, the gradient of the mean squared error against target
 * (device, B fields), and an Adam update (b1 = 0.9, b2 = 0.999, eps = 1e-8, bias-corrected) with
 * learning rate lr. Synchronises the stream; *loss (host, may be NULL) receives the loss before the
 * update. grads_out (host, may be NULL) receives the gradient (param_count floats) and then the
 * update is skipped: a gradient-only call. */
etd_status etd_sno_train_step(etd_sno s, const float* u, const double* D, const float* target, int B, float lr,
                              double* loss, float* grads_out, void* stream);

etd_status etd_sno_destroy(etd_sno s);

/* Parareal over `windows` windows of `window_steps` ETDRK2 steps of size tau, for B problems at N x N
 * with coefficients D[B] (host): U_0 = u0, U_{n+1}^{k+1} = G(U_n^{k+1}) + F(U_n^k) - G(U_n^k) from the
 * coarse sweep U^0. F runs the windows not yet converged of every problem as one batched ETDRK2 launch
 * sequence; G is the SNO (sno != NULL, trained for window_steps steps) or, for
 * sno == NULL, one ETDRK2 step of size window_steps * tau. Creation builds (and autotunes) the
 * batched solvers, one fine solver per count of windows still to converge (an iteration propagates only
 * those); it allocates states for all windows. */
typedef struct etd_parareal_s* etd_parareal;
etd_status etd_parareal_create(etd_parareal* out, etd_sno sno, int N, int B, const double* D, double tau,
                               int window_steps, int windows);

typedef struct {
  int iterations;          /* Parareal iterations run (fine sweeps) */
  int fallbacks;           /* windows advanced by the plain solver after a rejected correction */
  double correction[32];   /* per iteration: max over problems and updated windows of the correction rel L2 */
} etd_parareal_stats;

/* Run from u0 (device, B fields) and write the final state to u_out (device). Iterates until the
 * largest per-window correction (rel L2, max over problems) falls below tol, every window is converged,
 * or `max_iter` fine sweeps ran. Windows whose start is already the fine solution (u0, then one more
 * window per iteration, and windows advanced by the fine solver from such a start) take F of that start
 * and keep it: the update's value in exact arithmetic, without the coarse propagator's rounding. A
 * window whose correction exceeds fallback_tol in an iteration after the first is recomputed by the
 * fine solver from its corrected start (counted in stats->fallbacks), so later windows start from
 * plain-solver states. Synchronises. */
etd_status etd_parareal_run(etd_parareal p, const float* u0, float* u_out, int max_iter, double tol,
                            double fallback_tol, etd_parareal_stats* stats, void* stream);

etd_status etd_parareal_destroy(etd_parareal p);

#ifdef __cplusplus
}
#endif
#endif /* ETD_SNO_H */
