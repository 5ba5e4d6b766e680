/*
 * coal_oracle.c -- plain FP64 CPU oracle of the FSBM collision-coalescence step.
 *
 * TEST INFRASTRUCTURE ONLY (see coal_oracle.h). Written for a reader checking it against
 * the method by eye: no blocking, no fusion, no reordering beyond what the method states.
 * Compiled with -ffp-contract=off so that every product and sum rounds on its own.
 *
 * What the paper fixes: the routine is the per-grid-point collision-coalescence update
 * coal_bott_new (Sec. III, Listing 1), called only where T > 223.15 K (Listing 1), over
 * nkr = 33 mass bins extendable to a few hundred (Sec. I), whose cost is quadratic in the
 * bin count (Sec. VI-A). Each species pair has its own tabulated collection kernel such as
 * cwls, cwlg (Sec. VI-A, Listing 3), read one entry at a time (Listing 5). Grid points are
 * independent (Sec. VI-A, Codee's dependency analysis).
 *
 * What the paper leaves out is read from Bott (1998), whose flux method the routine's name
 * refers to, in the pairwise form; each reading is marked [reading] below.
 *
 * parity pins: mass conservation, positivity, number monotonicity, K = 0 identity, one-bin
 * constant kernel, single-pair cases, power-of-two scaling, Golovin and constant-kernel
 * closed forms, the active range with tau > 0 and one SWEEP step written out pair by pair
 * (tests/oracle_pins.py, tests/test_oracle_*.py).
 */
#include "coal_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAX_SPECIES 5
#define MAX_GRIDS 4
#define MAX_BINS 512

/* [reading] Bott's small constant added to the bin ratio before taking its logarithm. */
static const double BOTT_EPS = 1e-60;
/* [reading] A bin-sum whose log_alpha lies within this distance of an integer m is taken
 * to land exactly on bin m (c = 0); on the mass-doubling grid this is the i = j case. */
static const double TIE_SNAP = 1e-9;

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Mass of bin k on the geometric grid x_k = x0 * alpha^k. */
static double bin_mass(double x0, double alpha, int k) { return x0 * pow(alpha, (double)k); }

int oracle_grid_tables(int32_t n, double x0, double alpha, int32_t* kidx, double* cfrac) {
  if (n < 1 || n > MAX_BINS || !(x0 > 0.0) || !(alpha > 1.0) || !kidx || !cfrac) return -1;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      const double xs = bin_mass(x0, alpha, i) + bin_mass(x0, alpha, j);
      /* position of the pair's mass on the bin axis: log_alpha(xs / x0) */
      const double t = log(xs / x0) / log(alpha);
      const double m = floor(t + 0.5);
      int k;
      double c;
      if (fabs(t - m) < TIE_SNAP) {
        k = (int)m;
        c = 0.0;
      } else {
        k = (int)floor(t);
        const double xk = bin_mass(x0, alpha, k);
        const double xk1 = bin_mass(x0, alpha, k + 1);
        /* [reading] Bott's Courant number: the fraction of the way from x_k to x_{k+1},
         * linear in mass. */
        c = (xs - xk) / (xk1 - xk);
      }
      kidx[i * n + j] = k;
      cfrac[i * n + j] = c;
    }
  }
  return 0;
}

/* Index of the unordered species pair (a <= b) in the kernel table, upper-triangular
 * row-major: (0,0),(0,1),...,(0,S-1),(1,1),...,(S-1,S-1). */
static int pair_index(int S, int a, int b) { return a * S - a * (a - 1) / 2 + (b - a); }

typedef struct {
  int n;
  int S;                        /* species index space                          */
  int ns;                       /* species stored at this point                 */
  int sp[MAX_SPECIES];          /* their ids, ascending                         */
  const double* x;              /* [n] bin masses                               */
  const int32_t* kidx;          /* [n*n]                                        */
  const double* cfrac;          /* [n*n]                                        */
  const double* K;              /* this grid's kernels [pair][n][n]             */
  const double* K2;             /* ... at the second pressure level, or NULL    */
  double w;                     /* weight of K2 at this point's pressure        */
  const int8_t* product;        /* [S][S]                                       */
  double tau;
} point_ctx;

/* Collection kernel of particle (a, bin i) with particle (b, bin j).
 * a < b: K_ab[i][j]; a > b: K_ba[j][i]; a == b: the upper-triangle entry
 * K_aa[min(i,j)][max(i,j)] ([reading] a same-species table is read as symmetric). */
static double kern_table(const point_ctx* P, const double* K, int a, int i, int b, int j) {
  const size_t nn = (size_t)P->n * (size_t)P->n;
  if (a < b) return K[(size_t)pair_index(P->S, a, b) * nn + (size_t)i * P->n + j];
  if (a > b) return K[(size_t)pair_index(P->S, b, a) * nn + (size_t)j * P->n + i];
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  return K[(size_t)pair_index(P->S, a, a) * nn + (size_t)lo * P->n + hi];
}

/* The collection kernel of species a bin i with species b bin j at this point: the table
 * entry, or the two pressure levels' entries combined with the point's weight w. */
static double kern(const point_ctx* P, int a, int i, int b, int j) {
  const double k1 = kern_table(P, P->K, a, i, b, j);
  if (!P->K2) return k1;
  const double k2 = kern_table(P, P->K2, a, i, b, j);
  return k1 + P->w * (k2 - k1);
}

/* Bott's flux of the combined mass dM from bin k into bin k+1 of the product species.
 * [reading of Bott 1998] Inside bin k the mass is taken to follow an exponential profile
 * whose logarithmic slope x1 = ln(rho + eps) comes from the ratio rho of the upper
 * neighbour's content to bin k's content after the gain; the part of dM beyond the
 * fraction (1 - c) of the bin width moves up:
 *     F = dM * e^{x1/2} * (1 - e^{-c x1}) / x1,   F -> c dM as x1 -> 0,
 * clipped to [0, dM]. g_k and M_{k+1} are start-of-step values plus this pair's dM. */
static double bott_flux(double dM, double g_k, double M_k1, double c) {
  const double rho = M_k1 / g_k;
  const double x1 = log(rho + BOTT_EPS);
  double F;
  if (x1 == 0.0)
    F = dM * c;
  else if (isinf(x1))
    /* [reading] rho overflowed (g_k far below M_k1): the flux takes its limit as x1 grows,
     * all of dM for c > 0 and nothing for c = 0 */
    F = c > 0.0 ? dM : 0.0;
  else
    F = dM * exp(0.5 * x1) * (-expm1(-c * x1)) / x1;
  if (F < 0.0) F = 0.0;
  if (F > dM) F = dM;
  return F;
}

/* Deposit dM into product species slot cs at bin k (k may exceed the top bin) and split
 * it with the flux above. mk, mk1: the values the flux reads. */
static void deposit(const point_ctx* P, double* gain, int cs, int k, double c, double dM,
                    double Mk, double Mk1) {
  const int n = P->n;
  if (k >= n - 1) {
    /* [reading] The top bin keeps everything that reaches or passes it: no flux out of
     * bin n-1, and a pair whose sum lies beyond the grid is placed in bin n-1. */
    gain[cs * n + (n - 1)] += dM;
    return;
  }
  const double g_k = Mk + dM;
  const double F = bott_flux(dM, g_k, Mk1, c);
  gain[cs * n + k] += dM - F;
  gain[cs * n + k + 1] += F;
}

/* Active bin range of every stored species: the first and last bin whose content is
 * positive and at least tau times the species' largest bin. lo > hi means empty.
 * [reading] Bins inside [lo, hi] all take part; bins outside neither lose mass nor
 * collect others, but can still gain. */
static void active_ranges(const point_ctx* P, const double* M, int* lo, int* hi) {
  const int n = P->n;
  for (int s = 0; s < P->ns; ++s) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k)
      if (M[s * n + k] > mx) mx = M[s * n + k];
    lo[s] = n;
    hi[s] = -1;
    for (int k = 0; k < n; ++k) {
      const double v = M[s * n + k];
      if (v > 0.0 && v >= P->tau * mx) {
        if (k < lo[s]) lo[s] = k;
        hi[s] = k;
      }
    }
  }
}

/* Slot (position among the stored species) of species id c, or -1. */
static int slot_of(const point_ctx* P, int c) {
  for (int s = 0; s < P->ns; ++s)
    if (P->sp[s] == c) return s;
  return -1;
}

static double total_mass(const point_ctx* P, const double* M) {
  double sum = 0.0;
  for (int s = 0; s < P->ns; ++s)
    for (int k = 0; k < P->n; ++k) sum += M[s * P->n + k];
  return sum;
}

/* One PAIRWISE step (Jacobi form: every pair reads start-of-step values).
 * Returns 1 if the limiter fired. *min_rel receives min(M')/B before clamping. */
static int step_pairwise(const point_ctx* P, double* M, double dt, double B, double* err,
                         double* min_rel) {
  const int n = P->n, ns = P->ns;
  double N[MAX_SPECIES * MAX_BINS], R[MAX_SPECIES * MAX_BINS], lam[MAX_SPECIES * MAX_BINS];
  double loss[MAX_SPECIES * MAX_BINS], gain[MAX_SPECIES * MAX_BINS];
  int lo[MAX_SPECIES], hi[MAX_SPECIES];
  int limited = 0;

  /* number concentration N = M / x */
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < n; ++k) N[s * n + k] = M[s * n + k] / P->x[k];
  active_ranges(P, M, lo, hi);

  /* requested loss R^a_i = dt x_i N^a_i sum_b sum_j K(a,i;b,j) N^b_j over active (b,j),
   * j = i included with weight 1 (the diagonal pair removes two particles of bin i). */
  for (int s = 0; s < ns; ++s) {
    for (int i = 0; i < n; ++i) {
      R[s * n + i] = 0.0;
      lam[s * n + i] = 1.0;
      if (i < lo[s] || i > hi[s]) continue;
      double acc = 0.0;
      for (int t = 0; t < ns; ++t)
        for (int j = lo[t]; j <= hi[t]; ++j) acc += kern(P, P->sp[s], i, P->sp[t], j) * N[t * n + j];
      R[s * n + i] = dt * P->x[i] * N[s * n + i] * acc;
      /* limiter ratio lambda = min(1, M / R) */
      if (R[s * n + i] > 0.0 && M[s * n + i] / R[s * n + i] < 1.0) {
        lam[s * n + i] = M[s * n + i] / R[s * n + i];
        limited = 1;
      }
    }
  }

  memset(loss, 0, sizeof(double) * (size_t)ns * n);
  memset(gain, 0, sizeof(double) * (size_t)ns * n);

  /* every unordered pair of active particles (a,i), (b,j): same species i <= j */
  for (int sa = 0; sa < ns; ++sa) {
    for (int sb = sa; sb < ns; ++sb) {
      const int a = P->sp[sa], b = P->sp[sb];
      /* [reading] product species of an (a,b) collision: the table entry, default
       * max(a,b) in the order drops < ice < snow < graupel < hail */
      const int cs = slot_of(P, P->product[a * P->S + b]);
      for (int i = lo[sa]; i <= hi[sa]; ++i) {
        const int jstart = (sa == sb) ? i : lo[sb];
        for (int j = jstart; j <= hi[sb]; ++j) {
          const double h = (sa == sb && i == j) ? 0.5 : 1.0;
          const double phi = lam[sa * n + i] < lam[sb * n + j] ? lam[sa * n + i] : lam[sb * n + j];
          /* number of collisions per unit volume in dt */
          const double C = kern(P, a, i, b, j) * N[sa * n + i] * N[sb * n + j] * dt * h * phi;
          const double dM = C * (P->x[i] + P->x[j]);
          /* a pair whose transferred mass rounds to zero (deep spectral tails) does nothing */
          if (!(dM > 0.0)) continue;
          loss[sa * n + i] += C * P->x[i];
          loss[sb * n + j] += C * P->x[j];
          const int k = P->kidx[i * n + j];
          const double c = P->cfrac[i * n + j];
          const double Mk = (k < n) ? M[cs * n + k] : 0.0;
          const double Mk1 = (k + 1 < n) ? M[cs * n + k + 1] : 0.0;
          deposit(P, gain, cs, k, c, dM, Mk, Mk1);
        }
      }
    }
  }

  /* M' = M - loss + gain, its mass error against the budget, then renormalisation */
  double mn = 0.0;
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < n; ++k) {
      const double v = M[s * n + k] - loss[s * n + k] + gain[s * n + k];
      if (v / B < mn) mn = v / B;
      M[s * n + k] = v;
    }
  const double sum = total_mass(P, M);
  *err = fabs(sum - B) / B;
  *min_rel = mn;
  /* [reading] round-off can leave a bin the limiter emptied a few ulps below zero; such
   * bins are set to zero before the spectrum is rescaled to the budget */
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < n; ++k)
      if (M[s * n + k] < 0.0) M[s * n + k] = 0.0;
  const double sum2 = total_mass(P, M);
  const double scale = B / sum2;
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < n; ++k) M[s * n + k] = M[s * n + k] * scale;
  return limited;
}

/* One SWEEP step: Bott's sequential in-place order. Pairs are visited in a fixed order
 * (species pair (a <= b) lexicographic, i ascending, j ascending, j >= i on the same
 * species), each reading the current spectrum, with per-pair limits instead of lambda:
 * C x_i <= M^a_i, and C x_j <= M^b_j unless the pair's mass lands in that same bin
 * (product species b, bin k = j); on the diagonal 2 C x_i <= M^a_i. Cross-check only. */
static int step_sweep(const point_ctx* P, double* M, double dt, double B, double* err,
                      double* min_rel) {
  const int n = P->n, ns = P->ns;
  int lo[MAX_SPECIES], hi[MAX_SPECIES];
  int limited = 0;
  active_ranges(P, M, lo, hi);
  for (int sa = 0; sa < ns; ++sa) {
    for (int sb = sa; sb < ns; ++sb) {
      const int a = P->sp[sa], b = P->sp[sb];
      const int cs = slot_of(P, P->product[a * P->S + b]);
      for (int i = lo[sa]; i <= hi[sa]; ++i) {
        const int jstart = (sa == sb) ? i : lo[sb];
        for (int j = jstart; j <= hi[sb]; ++j) {
          const double xi = P->x[i], xj = P->x[j];
          const double Ni = M[sa * n + i] / xi, Nj = M[sb * n + j] / xj;
          const int k = P->kidx[i * n + j];
          const double c = P->cfrac[i * n + j];
          double C;
          /* [reading] the bin whose cap decides C gives up all its mass: it becomes exactly 0,
           * the exact value of M - (M / x) x, rather than that difference's rounding residue
           * (a residue in an emptied bin would later steer the logarithm of Bott's flux) */
          int emptied = 0; /* 1: bin i, 2: bin j */
          if (sa == sb && i == j) {
            C = 0.5 * kern(P, a, i, b, j) * Ni * Nj * dt;
            const double cap = M[sa * n + i] / (2.0 * xi);
            if (C > cap) { C = cap; limited = 1; emptied = 1; }
          } else {
            C = kern(P, a, i, b, j) * Ni * Nj * dt;
            const double capi = M[sa * n + i] / xi;
            if (C > capi) { C = capi; limited = 1; emptied = 1; }
            if (!(cs == sb && k == j)) {
              const double capj = M[sb * n + j] / xj;
              if (C > capj) { C = capj; limited = 1; emptied = 2; }
            }
          }
          if (!(C * (xi + xj) > 0.0)) continue;
          const double dM = C * (xi + xj);
          /* [reading] the product bin may be bin j itself (product species b, k = j): that bin
           * loses C x_j and receives dM = C (x_i + x_j) before the flux, so its content is
           * M_j + C x_i, formed as that sum (not as a difference of two large terms), and it
           * is filled before any clamping */
          const int into_j = (cs == sb && k == j);
          if (sa == sb && i == j) {
            M[sa * n + i] = emptied ? 0.0 : M[sa * n + i] - 2.0 * C * xi;
          } else {
            M[sa * n + i] = emptied == 1 ? 0.0 : M[sa * n + i] - C * xi;
            if (!into_j) M[sb * n + j] = emptied == 2 ? 0.0 : M[sb * n + j] - C * xj;
          }
          if (k >= n - 1) {
            M[cs * n + (n - 1)] = into_j ? M[sb * n + j] + C * xi : M[cs * n + (n - 1)] + dM;
          } else {
            const double g_k = into_j ? M[sb * n + j] + C * xi : M[cs * n + k] + dM;
            const double F = bott_flux(dM, g_k, M[cs * n + k + 1], c);
            M[cs * n + k] = g_k - F;
            M[cs * n + k + 1] += F;
          }
          /* round-off below zero in a bin its own limit emptied */
          if (M[sa * n + i] < 0.0) M[sa * n + i] = 0.0;
          if (M[sb * n + j] < 0.0) M[sb * n + j] = 0.0;
        }
      }
    }
  }
  double mn = 0.0;
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < n; ++k)
      if (M[s * n + k] / B < mn) mn = M[s * n + k] / B;
  const double sum = total_mass(P, M);
  *err = fabs(sum - B) / B;
  *min_rel = mn;
  const double scale = B / sum;
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < n; ++k) M[s * n + k] = M[s * n + k] * scale;
  return limited;
}

static int popcount8(unsigned v) {
  int c = 0;
  for (; v; v >>= 1) c += (int)(v & 1u);
  return c;
}

int oracle_coal_step(const oracle_config* cfg, const oracle_state* st, int64_t n_points,
                     double dt, int32_t n_steps, int32_t mode, int32_t n_threads) {
  if (!cfg || !st || n_points < 0 || !(dt >= 0.0) || !isfinite(dt) || n_steps < 0) return -1;
  if (mode != ORACLE_PAIRWISE && mode != ORACLE_SWEEP) return -1;
  if (cfg->n_species < 1 || cfg->n_species > MAX_SPECIES) return -1;
  if (cfg->n_grids < 1 || cfg->n_grids > MAX_GRIDS) return -1;
  if (!cfg->bins_per_grid || !cfg->x0_g || !cfg->alpha || !cfg->kernels || !cfg->product) return -1;
  if (n_points > 0 && (!st->spectra || !st->offset || !st->grid_id || !st->species_mask ||
                       !st->mass_budget || !st->mass_error || !st->status))
    return -1;
  const int S = cfg->n_species, G = cfg->n_grids;
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b) {
      const int p = cfg->product[a * S + b];
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      if (p != lo && p != hi) return -1;
      if (p != cfg->product[b * S + a]) return -1;
    }

  /* per-grid bin masses and pair tables */
  double* xg[MAX_GRIDS] = {0};
  int32_t* kg[MAX_GRIDS] = {0};
  double* cg[MAX_GRIDS] = {0};
  const double* Kg[MAX_GRIDS] = {0};
  const double* K2g[MAX_GRIDS] = {0};
  if (cfg->kernels_p2 &&
      (!isfinite(cfg->p1_hpa) || !isfinite(cfg->p2_hpa) || cfg->p1_hpa == cfg->p2_hpa))
    return -1;
  size_t koff = 0;
  int rc = 0;
  const int npairs = S * (S + 1) / 2;
  for (int g = 0; g < G; ++g) {
    const int n = cfg->bins_per_grid[g];
    if (n < 1 || n > MAX_BINS) { rc = -1; break; }
    xg[g] = (double*)malloc(sizeof(double) * n);
    kg[g] = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * n);
    cg[g] = (double*)malloc(sizeof(double) * (size_t)n * n);
    if (!xg[g] || !kg[g] || !cg[g]) { rc = -1; break; }
    for (int k = 0; k < n; ++k) xg[g][k] = bin_mass(cfg->x0_g[g], cfg->alpha[g], k);
    if (oracle_grid_tables(n, cfg->x0_g[g], cfg->alpha[g], kg[g], cg[g]) != 0) { rc = -1; break; }
    Kg[g] = cfg->kernels + koff;
    K2g[g] = cfg->kernels_p2 ? cfg->kernels_p2 + koff : NULL;
    koff += (size_t)npairs * n * n;
  }

  if (rc == 0) {
    int nt = n_threads > 0 ? n_threads : oracle_max_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t p = 0; p < n_points; ++p) {
      st->mass_budget[p] = 0.0;
      st->mass_error[p] = 0.0;
      if (st->min_rel_preclamp) st->min_rel_preclamp[p] = 0.0;
      /* C7: the point takes part only if cloudy and warmer than t_min (Listing 1) */
      if ((st->cloudy && st->cloudy[p] == 0) ||
          (st->temperature && !((double)st->temperature[p] > cfg->t_min_K))) {
        st->status[p] = ORACLE_ST_INACTIVE;
        continue;
      }
      const int g = st->grid_id[p];
      const unsigned mask = st->species_mask[p];
      if (g >= G || (mask >> S) != 0u) {
        st->status[p] = ORACLE_ST_BADINPUT;
        continue;
      }
      point_ctx P;
      P.n = cfg->bins_per_grid[g];
      P.S = S;
      P.ns = 0;
      for (int a = 0; a < S; ++a)
        if (mask & (1u << a)) P.sp[P.ns++] = a;
      P.x = xg[g];
      P.kidx = kg[g];
      P.cfrac = cg[g];
      P.K = Kg[g];
      P.K2 = K2g[g];
      P.w = 0.0;
      if (P.K2 && st->pressure) {
        const double pr = (double)st->pressure[p];
        if (!isfinite(pr)) {
          st->status[p] = ORACLE_ST_BADINPUT;
          continue;
        }
        double w = (cfg->p1_hpa - pr) / (cfg->p1_hpa - cfg->p2_hpa);
        if (w < 0.0) w = 0.0;
        if (w > 1.0) w = 1.0;
        P.w = w;
      }
      P.product = cfg->product;
      P.tau = cfg->active_rel_threshold;
      const int64_t len = st->offset[p + 1] - st->offset[p];
      if (len != (int64_t)popcount8(mask) * P.n) {
        st->status[p] = ORACLE_ST_BADINPUT;
        continue;
      }
      double* M = st->spectra + st->offset[p];
      int bad = 0;
      for (int64_t e = 0; e < len; ++e)
        if (!isfinite(M[e]) || M[e] < 0.0) bad = 1;
      if (bad) {
        st->status[p] = ORACLE_ST_BADINPUT;
        continue;
      }
      const double B = total_mass(&P, M);
      if (!(B > 0.0)) {
        st->status[p] = ORACLE_ST_INACTIVE;
        continue;
      }
      st->mass_budget[p] = B;
      int status = 0;
      double emax = 0.0, mnmin = 0.0;
      for (int s = 0; s < n_steps; ++s) {
        /* C1: the budget of every step is the start-of-step total mass */
        const double Bs = total_mass(&P, M);
        double e = 0.0, mn = 0.0;
        const int lim = (mode == ORACLE_PAIRWISE) ? step_pairwise(&P, M, dt, Bs, &e, &mn)
                                                  : step_sweep(&P, M, dt, Bs, &e, &mn);
        if (lim) status |= ORACLE_ST_LIMITED;
        if (e > emax) emax = e;
        if (mn < mnmin) mnmin = mn;
      }
      st->mass_error[p] = emax;
      st->status[p] = status;
      if (st->min_rel_preclamp) st->min_rel_preclamp[p] = mnmin;
    }
  }
  for (int g = 0; g < G; ++g) {
    free(xg[g]);
    free(kg[g]);
    free(cg[g]);
  }
  return rc;
}
