/*
 * fsbm_coal.h -- C ABI of the GB300 (sm_103a) FSBM collision-coalescence library.
 *
 * The operation: one call advances, on the GPU, the bin spectra of a ragged batch of
 * independent grid points by n_steps steps of the stochastic collection (collision-
 * coalescence) update that WRF's Fast Spectral Bin Microphysics performs per grid point in
 * coal_bott_new (arXiv 2409.07232, Sec. III, Listing 1). Collisions run only at points
 * warmer than t_min_K (Listing 1: TT > 223.15 K), with pair collection kernels tabulated
 * per species pair (Sec. VI-A, Listing 3) and read per entry (Listing 5), over mass bins
 * whose count the paper puts at 33, extendable to a few hundred (Sec. I); the cost is
 * quadratic in the bin count (Sec. VI-A). Grid points are independent (Sec. VI-A).
 *
 * The arithmetic is Bott's flux method in the pairwise form: per step, with every pair of
 * active bins reading start-of-step values,
 *   N = M / x;  R^a_i = dt x_i N^a_i sum_{b,j} K_ab(i,j) N^b_j;  lambda = min(1, M / R);
 *   C = K N^a_i N^b_j dt h min(lambda^a_i, lambda^b_j)   (h = 1/2 for a = b, i = j);
 *   both partners lose C x; dM = C (x_i + x_j) goes to species P(a,b), bin
 *   k = floor(log_alpha((x_i + x_j) / x_0)), and Bott's flux
 *   F = dM e^{x1/2} (1 - e^{-c x1}) / x1, x1 = ln(M_{k+1} / (M_k + dM) + 1e-60),
 *   c = (x_i + x_j - x_k) / (x_{k+1} - x_k), clipped to [0, dM], moves to bin k+1;
 *   M' = M - loss + gain, round-off negatives set to 0, then M' scaled so that the
 *   point's total mass equals its start-of-step total (FP64).
 * Bins outside a species' active range [lo, hi] (first/last bin with M > 0 and
 * M >= tau * max M) do not collect; a pair whose sum passes the top bin stays there.
 *
 * Units: CGS. M in g cm^-3, x in g, K in cm^3 s^-1, dt in s, T in K.
 *
 * Conventions for every entry point:
 *  - Ownership: the context owns its device copies of the tables and its scratch memory;
 *    the caller owns every state buffer. Spectra are updated in place; no output may alias
 *    the spectra.
 *  - Device pointers in fsbm_coal_state must be device memory of the context's device;
 *    fsbm_coal_step_host takes host pointers instead.
 *  - fsbm_coal_step is asynchronous on the context's stream. It allocates device memory
 *    only when n_points exceeds every earlier call's; later calls allocate nothing and do
 *    not synchronise the host.
 *  - Errors: invalid arguments return FSBM_E_ARG before anything is launched; CUDA errors
 *    return FSBM_E_CUDA; a message is kept for fsbm_coal_last_error. Bad data inside a
 *    point (NaN, Inf, negative bins, an unknown grid id, a species mask or spectrum length
 *    that does not match) never traps: the point is left unchanged and flagged in status.
 *  - Thread safety: a context (or a replica, fsbm_coal_clone) is used by one host thread at a
 *    time; different contexts and replicas may be used from different threads concurrently.
 */
#ifndef FSBM_COAL_H
#define FSBM_COAL_H

#include <stdint.h>

#if defined(__GNUC__)
#define FSBM_API __attribute__((visibility("default")))
#else
#define FSBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsbm_coal_ctx fsbm_coal_ctx; /* opaque, library-owned */

typedef enum {
  FSBM_OK = 0,
  FSBM_E_ARG = -1,         /* invalid argument; nothing launched                  */
  FSBM_E_CUDA = -2,        /* a CUDA call failed; see fsbm_coal_last_error         */
  FSBM_E_OOM = -3,         /* device allocation failed                            */
  FSBM_E_TIMEOUT = -4,     /* reserved: a bounded device wait gave up             */
  FSBM_E_UNSUPPORTED = -5  /* valid request the library does not implement         */
} fsbm_status;

typedef enum {
  FSBM_FP64 = 0,        /* FP64 spectra and FP64 arithmetic throughout              */
  FSBM_FP32_SPLIT = 1   /* FP32 spectra, FP32 pair fluxes and sums; FP64 budget,
                           limiter ratios, update and renormalisation             */
} fsbm_precision;

/* The order in which a step applies its pair transfers. Both use Bott's flux (Bott 1998), the
 * method of the routine the paper ports (coal_bott_new, Sec. III, Listing 1). */
typedef enum {
  FSBM_PAIRWISE = 0,    /* every pair reads the start-of-step spectrum (Jacobi form) with
                           one limiter ratio per bin; order-independent, parallel in a point */
  FSBM_SWEEP = 1        /* Bott's in-place order: species pairs (a <= b), i ascending, j
                           ascending (j >= i for a = b), each pair reading the spectrum its
                           predecessors left, with per-pair caps C x_i <= M_i and
                           C x_j <= M_j (none on bin j when the product lands there; 2 C x_i
                           <= M_i on the diagonal). One thread per point, the paper's own
                           mapping (Sec. VI-B). FP64 only.                                  */
} fsbm_mode;

/* Per-point status bits written by fsbm_coal_step. */
enum {
  FSBM_ST_LIMITED = 1,   /* the loss limiter fired (lambda < 1) in some bin and step   */
  FSBM_ST_BADINPUT = 2,  /* NaN/Inf/negative bin, unknown grid, mask/length mismatch:
                            point left unchanged                                       */
  FSBM_ST_INACTIVE = 4   /* not cloudy, T <= t_min_K, or zero mass: left unchanged     */
};

typedef struct {
  int32_t n_species;            /* species index space S, 1..5 (0 drops, 1 ice, 2 snow,
                                   3 graupel, 4 hail by convention)                      */
  int32_t n_grids;              /* 1..4 bin grids                                        */
  const int32_t* bins_per_grid; /* host [n_grids], each 2..512 (33 s for s bins/doubling) */
  const double* x0_g;           /* host [n_grids] smallest bin mass in g, > 0             */
  const double* alpha;          /* host [n_grids] mass ratio of adjacent bins, 1 < a <= 2 */
  const double* kernels;        /* host FP64 [grid][pair a<=b][n][n], finite, >= 0;
                                   pair index a*S - a(a-1)/2 + (b-a); entry [i][j] is the
                                   kernel of species a bin i with species b bin j; for a = b
                                   only the upper triangle i <= j is read               */
  const int8_t* product;        /* host [S][S] product species, P(a,b) = P(b,a) in {a,b};
                                   NULL = max(a,b)                                         */
  double t_min_K;               /* collisions only where T > t_min_K (223.15 in WRF)      */
  double active_rel_threshold;  /* tau in [0, 1): active range cut-off relative to the
                                   species' largest bin                                    */
  int32_t precision;            /* fsbm_precision                                         */
  int32_t mode;                 /* fsbm_mode: FSBM_PAIRWISE or FSBM_SWEEP (FP64 only;
                                   FSBM_SWEEP with FSBM_FP32_SPLIT: FSBM_E_UNSUPPORTED;
                                   any other value: FSBM_E_ARG)                            */
  /* Kernels at two pressure levels (Sec. VI-A, Listing 3: FSBM forms each collision table
   * from a 750 mb and a 500 mb table). NULL: `kernels` is used as is and pressures are
   * ignored. Otherwise `kernels` holds the tables at p1_hpa and kernels_p2 (host FP64, same
   * layout, finite, >= 0) those at p2_hpa, and a point at pressure p collides with
   *   K = K1 + w (K2 - K1),  w = (p1 - p) / (p1 - p2) clamped to [0, 1]
   * (linear between the levels, constant outside; the paper elides the formula). The tables
   * are read on demand per pair (Listing 5), one extra load and multiply-add each.         */
  const double* kernels_p2;
  double p1_hpa;                /* finite; p1_hpa != p2_hpa when kernels_p2 is set         */
  double p2_hpa;
} fsbm_coal_config;

typedef struct {                /* device pointers, caller-owned                          */
  void* spectra;                /* double (FSBM_FP64) or float (FSBM_FP32_SPLIT), packed:
                                   point p holds [stored species ascending][n_bins] at
                                   element offset[p]; updated in place. Must not be NULL
                                   when n_points > 0, even if no point stores a species
                                   (any valid device address then)                         */
  const int64_t* offset;        /* [n_points + 1] element offsets into spectra            */
  const uint8_t* grid_id;       /* [n_points]                                             */
  const uint8_t* species_mask;  /* [n_points] bit a set: species a stored                 */
  const uint8_t* cloudy;        /* [n_points], 0 = skip; NULL = every point cloudy         */
  const float* temperature;     /* [n_points] in K; NULL = every point warm enough         */
  double* mass_budget;          /* [n_points] out: total mass B at the start of the call  */
  double* mass_error;           /* [n_points] out: max over steps of |sum M' - B_s| / B_s
                                   before renormalisation                                  */
  int32_t* status;              /* [n_points] out: FSBM_ST_* bits                          */
  const float* pressure;        /* [n_points] in hPa, read when the context has
                                   kernels_p2; NULL = every point at p1_hpa; a non-finite
                                   value marks the point FSBM_ST_BADINPUT                  */
} fsbm_coal_state;

/* Counters of the most recent step (read back with a stream synchronisation). */
typedef struct {
  int64_t n_points;             /* points passed                                          */
  int64_t n_active;             /* points that passed the cloud/temperature/shape checks   */
  int32_t block_dim;            /* threads per CTA of the collision kernel                */
  int32_t grid_dim;             /* persistent CTAs                                        */
  int32_t graph_replayed;       /* 1 if the last step was a CUDA-graph replay             */
  int32_t tune_cache_hit;       /* 1 if the last autotune call took a remembered choice    */
  /* with timing on (fsbm_coal_set_timing), totals since the previous fsbm_coal_get_stats
   * call, measured with CUDA events on the context's stream:                            */
  double coal_ms;               /* collision-kernel time (steps launched without a graph) */
  int64_t coal_launches;        /* collision-kernel launches timed                        */
  double step_ms;               /* whole-step time (compaction + collision, any mode)     */
  int64_t steps_timed;          /* steps timed                                            */
  int64_t shard_begin;          /* the part [shard_begin, shard_end) of the ordered list of
                                   active points (fsbm_coal_get_active_list) the last step
                                   ran; [0, n_active) unless it was fsbm_coal_step_shard    */
  int64_t shard_end;
} fsbm_coal_stats;

/* Build a context: validates the configuration, derives every grid's pair tables (target
 * bin offset and Courant number per bin distance), lays out the kernels for the device and
 * copies them to the current CUDA device on `stream` (a cudaStream_t, NULL = default
 * stream). Synchronises the stream before returning. *out receives the context. */
FSBM_API fsbm_status fsbm_coal_init(const fsbm_coal_config* config, void* stream, fsbm_coal_ctx** out);

/* A replica of a context for another stream (NULL = the default stream). The paper runs
 * several MPI ranks per GPU, each with its own share of the domain (Sec. VII-A); replicas are
 * that mapping inside one process: they share the context's device tables (nothing is copied or
 * allocated by this call) and each has its own stream, scratch, launch plan, CUDA graph and
 * timing, so replicas step their own batches concurrently on their own streams, from one host
 * thread or several (each replica used by one thread at a time). The tables are freed when the
 * context and all its replicas are destroyed, in any order. fsbm_coal_step_noalloc uses one
 * library-wide array: replicas calling it must not overlap on the GPU. The context's device must
 * be current when a replica steps. */
FSBM_API fsbm_status fsbm_coal_clone(const fsbm_coal_ctx* ctx, void* stream, fsbm_coal_ctx** out);

/* Advance n_points points by n_steps steps of length dt (>= 0, finite) on the context's
 * stream. Inputs and outputs are device pointers (see fsbm_coal_state). */
FSBM_API fsbm_status fsbm_coal_step(fsbm_coal_ctx* ctx, const fsbm_coal_state* state, int64_t n_points,
                           double dt, int32_t n_steps);

/* One shard of a batch split across several GPUs (one process and one context per GPU, each
 * holding the whole batch's inputs). Grid points are independent (Sec. VI-A: no dependence
 * between the grid points of the collision loop), so the batch splits with no exchange between
 * the shards. Every shard classifies and orders all n_points exactly as fsbm_coal_step does (the
 * compaction pass, costliest class first), cuts the ordered list of active points into n_shards
 * contiguous parts of near-equal cost (bin pairs per collision step; every part lies within one
 * point's cost of the total over n_shards, the bounds fsbm_coal_shard_bounds returns), and
 * steps part `shard` only. Points of the other parts are left unchanged and their outputs are
 * not written; skipped points (inactive, bad input) get their outputs in every shard. The
 * union of the n_shards calls' results equals one fsbm_coal_step call's, bit for bit.
 * 0 <= shard < n_shards <= 1024, else FSBM_E_ARG. fsbm_coal_get_stats reports the part's list
 * positions (shard_begin, shard_end). */
FSBM_API fsbm_status fsbm_coal_step_shard(fsbm_coal_ctx* ctx, const fsbm_coal_state* state, int64_t n_points,
                                          double dt, int32_t n_steps, int32_t shard, int32_t n_shards);

/* The shard bounds fsbm_coal_step_shard uses, on the host (no context, no GPU): a cost-ordered
 * list of n_runs runs, run r holding run_count[r] entries of cost run_cost[r] each (both >= 0),
 * is cut into n_shards contiguous parts; bounds[q] (q = 0..n_shards, caller-owned) is the first
 * position whose cost prefix reaches ceil(q T / n_shards), T the total cost. Part q is
 * [bounds[q], bounds[q+1]); its cost differs from T / n_shards by less than the largest entry
 * cost plus one. FSBM_E_ARG for negative sizes, n_shards outside [1, 1024], or a total cost at
 * or above 2^62 / n_shards. */
FSBM_API fsbm_status fsbm_coal_shard_bounds(const int64_t* run_count, const int64_t* run_cost, int32_t n_runs,
                                            int32_t n_shards, int64_t* bounds);

/* Same as fsbm_coal_step with every fsbm_coal_state pointer in HOST memory: the arrays are
 * copied to context-owned device buffers, stepped, and the spectra and outputs copied back.
 * Synchronous (returns after the results are in host memory). Pinned host memory makes the
 * copies faster. */
FSBM_API fsbm_status fsbm_coal_step_host(fsbm_coal_ctx* ctx, const fsbm_coal_state* host_state,
                                int64_t n_points, double dt, int32_t n_steps);

/* fsbm_coal_step without any device allocation. The paper has no counterpart: this is for
 * callers that cannot let a library call cudaMalloc -- a host model that reserves all device
 * memory in its own pool (for example several model processes sharing one GPU), or one that
 * cannot take the device-wide synchronisation an allocation implies inside its time loop.
 * Same arguments, same results and same stream semantics as fsbm_coal_step, but the
 * compaction scratch lives in a fixed array inside the library (about 1.1 MB on every GPU
 * that loads it, held until the process exits), so n_points is limited to 262144; larger
 * batches return FSBM_E_ARG. The context's device must be current. The first call on a
 * device looks the array up (cudaGetSymbolAddress): make it before any stream capture. All
 * calls share the array, so calls that overlap on the GPU (different streams or threads) race
 * and must be serialised by the caller. It is never captured in a CUDA graph by the library
 * or timed (fsbm_coal_set_graph and fsbm_coal_set_timing do not apply to it), and
 * fsbm_coal_get_stats and fsbm_coal_get_active_list report fsbm_coal_step's own scratch, not
 * this array. The array's device address is looked up once per device and kept: after a
 * cudaDeviceReset the library must be reloaded before this entry point is used again. Errors
 * name this entry point in fsbm_coal_last_error. */
FSBM_API fsbm_status fsbm_coal_step_noalloc(fsbm_coal_ctx* ctx, const fsbm_coal_state* state, int64_t n_points,
                                            double dt, int32_t n_steps);

/* Bin fields in WRF's own memory layout (Sec. I: a patch's arrays span the memory ranges
 * ims:ime, kms:kme, jms:jme, and a thread works on a tile its:ite, kts:kte, jts:jte inside
 * them; Sec. III, Listing 1: the collision step runs at every tile point (i, k, j) warmer than
 * t_min_K; Sec. VI-B, Listing 6: a predicate array kept from the loop fission says where the
 * collision step is called). Ranges are inclusive, in the caller's index space (Fortran's
 * 1-based indices work as they are). All pointers are device pointers, caller-owned.        */
typedef struct {
  void* ff[5];                  /* per species id a: its bins, element (i, k, j, bin b) at
                                   ((b * jm + (j - jms)) * km + (k - kms)) * im + (i - ims),
                                   im = ime - ims + 1 and so on (i fastest: Fortran's
                                   ff(i, k, j, b)); double or float as the context's
                                   precision; NULL = species not carried. Updated in place at
                                   the points the step runs on, untouched elsewhere.           */
  const float* temperature;     /* [j][k][i] over the memory ranges, K; NULL = all warm       */
  const uint8_t* predicate;     /* [j][k][i], nonzero = run the collision step here;
                                   NULL = everywhere (still subject to temperature)           */
  const float* pressure;        /* [j][k][i] hPa for kernels at two pressure levels, or NULL */
  int32_t* status;              /* [j][k][i] out (FSBM_ST_* bits) at tile points, or NULL   */
  double* mass_budget;          /* [j][k][i] out at tile points, or NULL                    */
  double* mass_error;           /* [j][k][i] out at tile points, or NULL                    */
  int32_t ims, ime, kms, kme, jms, jme;  /* memory ranges                                   */
  int32_t its, ite, kts, kte, jts, jte;  /* tile ranges, inside the memory ranges; an empty
                                            tile (its > ite, ...) is a no-op                 */
  int32_t grid;                 /* bin grid (index into bins_per_grid) of every point         */
} fsbm_wrf_state;

/* Advance every tile point of a WRF-layout state n_steps collision steps of dt seconds: the
 * tile's points are packed into a context-owned buffer of the packed layout, stepped exactly
 * as by fsbm_coal_step, and the points it ran on are written back. Asynchronous on the
 * context's stream. The buffer holds (tile points) x (species carried) x bins values of the
 * context's precision and grows on demand (about 8.4 GB for a 425 x 300 x 50 tile with 5
 * species, 33 bins in FP64). Errors: FSBM_E_ARG for ranges outside the memory ranges, an
 * unknown grid or no species; FSBM_E_OOM if the buffer cannot be allocated. */
FSBM_API fsbm_status fsbm_coal_step_wrf(fsbm_coal_ctx* ctx, const fsbm_wrf_state* state, double dt,
                                        int32_t n_steps);

/* Time the collision kernel for each candidate CTA size (32, 64, 128, 256, 512 threads) and
 * keep the fastest for later steps. The whole batch is classified and ordered as a step would
 * order it; the timed sample is an even stride through that ordered list of active points,
 * holding a fixed amount of work (every class in its share, wherever in the batch its points
 * lie), stepped up to 4 collision steps of dt seconds (the caller's own step length: the
 * limiter's firing, and so the cost, depends on dt). The choice is remembered for the process
 * under a key of the device, precision, mode, kernel levels, bin grids, species count, range
 * threshold, dt, n_steps, gain split and the batch's mix of active point classes (grid and
 * stored-species count, in eighths): a later call with the same key, from this or another
 * context, takes it without timing (fsbm_coal_get_stats: tune_cache_hit). A batch with no
 * active point keeps the current CTA size. The caller's arrays are not modified: the tuner
 * works on a temporary copy of the spectra and its own outputs. Synchronous; allocates that
 * copy. The paper has no counterpart. */
FSBM_API fsbm_status fsbm_coal_autotune_steps(fsbm_coal_ctx* ctx, const fsbm_coal_state* state, int64_t n_points,
                                              double dt, int32_t n_steps);

/* fsbm_coal_autotune_steps with dt = 5 s and 3 steps. */
FSBM_API fsbm_status fsbm_coal_autotune(fsbm_coal_ctx* ctx, const fsbm_coal_state* state, int64_t n_points);

/* Enable (1) or disable (0, the default) CUDA-graph capture of fsbm_coal_step: the first
 * call with a given argument set records the launch sequence, later identical calls replay
 * it. */
FSBM_API fsbm_status fsbm_coal_set_graph(fsbm_coal_ctx* ctx, int32_t enable);

/* Force the collision kernel's CTA size (0 = library default); for benchmarks and the
 * autotuner's tests. Valid sizes: 32, 64, 128, 256, 512. */
FSBM_API fsbm_status fsbm_coal_set_block(fsbm_coal_ctx* ctx, int32_t block_dim);

/* Lanes that share one gain item's bin pairs in the pairwise kernels: 1, 2, 4 or 8, or 0
 * (the default) for the library's rule, which gives a point whose gain items would fill fewer
 * than four warps (one or two species on a short grid) up to 8 lanes per item and every other
 * point one. The lanes take every P-th bin distance and their partial sums are added in a
 * fixed order, so results depend on this setting (to rounding) but never on the CTA size.
 * Ignored by SWEEP. Returns FSBM_E_ARG for any other value. */
FSBM_API fsbm_status fsbm_coal_set_gain_split(fsbm_coal_ctx* ctx, int32_t lanes);

/* Enable (1) or disable (0, the default) CUDA-event timing of the collision kernel and of
 * whole steps; fsbm_coal_get_stats returns the totals. Costs two event records per step. */
FSBM_API fsbm_status fsbm_coal_set_timing(fsbm_coal_ctx* ctx, int32_t enable);

/* Synchronise the context's stream and fill *out with the last step's counters (and the
 * timing totals, which it then resets). */
FSBM_API fsbm_status fsbm_coal_get_stats(fsbm_coal_ctx* ctx, fsbm_coal_stats* out);

/* Synchronise and copy the last step's compacted list of active point indices (in the
 * order the collision kernel takes them: costliest class first, ascending point index
 * within a class) to host memory `out` of capacity `cap` entries. *n_out receives the
 * count (which may exceed cap; then only cap entries are written). */
FSBM_API fsbm_status fsbm_coal_get_active_list(fsbm_coal_ctx* ctx, int32_t* out, int64_t cap, int64_t* n_out);

/* Self-check of the library's FP64 helpers of the FP64 pair flux over a fixed sweep of
 * arguments, against CUDA's own functions: out5[0..4] receive the largest errors of the
 * logarithm (absolute; relative where |ln x| > 1), the exponential and e^y - 1 (relative),
 * and the reciprocal square root and reciprocal (relative). Synchronous; allocates 40 bytes. */
FSBM_API fsbm_status fsbm_coal_math_check(fsbm_coal_ctx* ctx, double* out5);

/* The bounds-checked build of this library (libfsbm_coal_checked.so, the same entry points
 * compiled with -DFSBM_CHECKED) checks, before every kernel walks a range of indices, the
 * range's ends against its arrays, skips a range that fails and counts the failure instead of
 * trapping. out4[0] receives the failures counted since the previous call (then reset), out4[1]
 * the source line of the first one, out4[2] and out4[3] its index and bound (low 32 bits).
 * Synchronises the context's stream. The normal build returns FSBM_E_UNSUPPORTED with zeros.
 * The paper has no counterpart; it stands in for a memory checker on small cases. */
FSBM_API fsbm_status fsbm_coal_check_record(fsbm_coal_ctx* ctx, uint32_t* out4);

/* Free the context and everything it owns. NULL is accepted. */
FSBM_API fsbm_status fsbm_coal_destroy(fsbm_coal_ctx* ctx);

/* Message of the context's last error ("" if none); a static message for NULL. */
FSBM_API const char* fsbm_coal_last_error(const fsbm_coal_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FSBM_COAL_H */
