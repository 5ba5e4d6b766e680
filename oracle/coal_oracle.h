/*
 * coal_oracle.h -- plain FP64 CPU oracle for the FSBM collision-coalescence step.
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, obviously-correct restatement of the
 * collision step that the CUDA library is checked against. Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or helper with the CUDA library under paper_2409_07232_gb300/.
 *
 * The paper (arXiv 2409.07232) names the routine (coal_bott_new, Sec. III and
 * Listing 1) and its cost structure (O(m n k b^2) per task, Sec. VI-A) but prints no
 * collision equations. The arithmetic here is Bott's (1998) flux method for the
 * stochastic collection equation, in the pairwise (Jacobi) form: every bin pair reads
 * start-of-step values, losses are limited by a per-bin ratio, and the combined mass
 * of a pair is split between the two mass bins that bracket it with Bott's
 * exponential-profile flux. Each reading taken where the paper is silent is marked
 * [reading] beside the code that implements it.
 *
 * Units are CGS: bin mass content M in g cm^-3, particle mass x in g, kernel K in
 * cm^3 s^-1, dt in s.
 */
#ifndef FSBM_COAL_ORACLE_H
#define FSBM_COAL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_PAIRWISE = 0, ORACLE_SWEEP = 1 };

/* Per-point status bits (the same meaning as the library's). */
enum {
  ORACLE_ST_LIMITED  = 1,   /* the loss limiter fired in some bin, some step        */
  ORACLE_ST_BADINPUT = 2,   /* negative / non-finite / inconsistent input: skipped  */
  ORACLE_ST_INACTIVE = 4    /* not cloudy, too cold, or no mass: left unchanged     */
};

typedef struct {
  int32_t n_species;              /* species index space S, 1..5                      */
  int32_t n_grids;                /* 1..4                                             */
  const int32_t* bins_per_grid;   /* [n_grids]                                        */
  const double* x0_g;             /* [n_grids] smallest bin mass (g)                  */
  const double* alpha;            /* [n_grids] mass ratio of adjacent bins            */
  const double* kernels;          /* [grid][pair a<=b][n][n], grids packed in order   */
  const int8_t* product;          /* [S][S] product species of a collision            */
  double t_min_K;                 /* collisions only where T > t_min_K                */
  double active_rel_threshold;    /* tau_act                                          */
  /* Pressure dependence of the kernels (Sec. VI-A, Listing 3: every collision array is
   * formed from a 750 mb and a 500 mb table). kernels_p2 == NULL: `kernels` is used as is.
   * Otherwise `kernels` holds the tables at pressure p1_hpa and kernels_p2 (same layout)
   * those at p2_hpa, and a point at pressure p uses
   *   K = K1 + w (K2 - K1),  w = (p1 - p) / (p1 - p2) clamped to [0, 1]
   * [reading: linear in pressure between the two levels, constant outside them; the
   * paper elides the formula]. A point without a pressure (pressure == NULL) is at p1. */
  const double* kernels_p2;
  double p1_hpa, p2_hpa;
} oracle_config;

typedef struct {
  double* spectra;                /* packed: per point [stored species][n], in/out    */
  const int64_t* offset;          /* [n_points+1] element offsets                     */
  const uint8_t* grid_id;         /* [n_points]                                       */
  const uint8_t* species_mask;    /* [n_points] bit a set: species a stored           */
  const uint8_t* cloudy;          /* [n_points] or NULL                               */
  const float* temperature;       /* [n_points] or NULL                               */
  const float* pressure;          /* [n_points] hPa, or NULL (see kernels_p2)         */
  double* mass_budget;            /* [n_points] out: B of the first step              */
  double* mass_error;             /* [n_points] out: max over steps of |sum M'-B|/B   */
  int32_t* status;                /* [n_points] out                                   */
  double* min_rel_preclamp;       /* [n_points] out or NULL: min over steps and bins of
                                     M'/B before negative round-off is clamped        */
} oracle_state;

/* Bin-pair product tables of one grid, straight from the definitions:
 * kidx[i*n+j] = floor(log_alpha((x_i+x_j)/x_0)) (tie-snapped), may be >= n;
 * cfrac[i*n+j] = (x_i+x_j-x_k)/(x_{k+1}-x_k). Returns 0 or -1 on bad arguments. */
int oracle_grid_tables(int32_t n, double x0, double alpha, int32_t* kidx, double* cfrac);

/* Advance every point n_steps steps of length dt. n_threads <= 0 means all cores.
 * Returns 0, or -1 on a bad argument (nothing is changed then). */
int oracle_coal_step(const oracle_config* cfg, const oracle_state* st, int64_t n_points,
                     double dt, int32_t n_steps, int32_t mode, int32_t n_threads);

/* Threads an OpenMP parallel region would use (1 when built without OpenMP). */
int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
