// fsbm_internal.cuh -- device-side data shared by the library's translation units.
//
// Layout of everything the kernels read, per grid (all device memory, context-owned):
//   kappa[d], cd[d]   target-bin offset and Courant number of a bin pair at distance
//                     d = |i - j|: on a geometric grid x_k = x0 alpha^k the pair's mass
//                     x_i + x_j = x_max (1 + alpha^-d) lands in bin max(i,j) + kappa[d]
//                     with c = ((1 + alpha^-d) alpha^-kappa - 1) / (alpha - 1), so both
//                     depend on d only (the pair tables of Sec. VI-A shrink to length n).
//   x[k]              bin masses.
//   Kd[d][m][s*S+l]   kernel of species s bin m-d with species l bin m times
//                     1 + alpha^-d = (x_{m-d} + x_m) / x_m (halved for the same-species
//                     diagonal d = 0, s = l, which counts once), the S*S ordered species pairs
//                     innermost: the gain pass puts one lane per species orientation on the
//                     same (d, m), so a warp's loads are contiguous.
//   Kr[a][b][j][i]    kernel of species a bin i with species b bin j (i fastest): the
//                     layout of the loss mat-vec, one lane per row i.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "fsbm_math.cuh"

namespace fsbm {

// Bounds-checked build (compiled with -DFSBM_CHECKED into libfsbm_coal_checked.so): before a
// kernel walks a range of indices it checks the range's ends (a point's list slot, grid, bin
// count and element count; a gain group's bins, distances and table entries; a loss row's
// columns; a compaction slot; a WRF-layout element) against the arrays' sizes. A failed check
// adds one to the context's check record, keeps the first failing source line, index and bound,
// and the kernel skips that range: nothing traps and no access leaves its array. The normal
// build compiles the checks out.
#ifdef FSBM_CHECKED
__device__ __forceinline__ bool fsbm_in_range(unsigned* chk, long long i, long long bound, int line) {
  if (i >= 0 && i < bound) return true;
  if (chk) {
    atomicAdd(chk, 1u);
    if (atomicCAS(chk + 1, 0u, (unsigned)line) == 0u) {
      chk[2] = (unsigned)i;
      chk[3] = (unsigned)bound;
    }
  }
  return false;
}
#define FSBM_OK(chk, i, bound) fsbm_in_range((chk), (long long)(i), (long long)(bound), __LINE__)
#define FSBM_CHECKED_BUILD 1
#else
#define FSBM_OK(chk, i, bound) true
#define FSBM_CHECKED_BUILD 0
#endif

constexpr int kMaxSpecies = 5;
constexpr int kMaxGrids = 4;
constexpr int kMaxBins = 512;
constexpr int kMaxKappa = 15;      // kappa[0] = floor(log_alpha 2) <= 15 -> alpha >= 2^(1/15)
constexpr int kMaxOrient = kMaxSpecies * kMaxSpecies;
constexpr int kNumBuckets = kMaxGrids * kMaxSpecies;

// Bott's constant added to the bin ratio before its logarithm (FP64 form).
constexpr double kBottEps = 1e-60;
// ln(1e-60): the FP32 form clamps the logarithm here instead of adding 1e-60.
constexpr float kLnBottEps = -138.15510557964274f;

struct GridDev {
  unsigned* chk;                  // check record of the bounds-checked build (else NULL)
  int n;
  unsigned inv_n;                 // floor(2^32 / n) + 1: e / n = umulhi(e, inv_n) for e < 5 n
  int kappa_max;                  // kappa[0]
  int d_lo[kMaxKappa + 1];        // D_kappa = {d : kappa[d] = kappa} = [d_lo, d_hi]
  int d_hi[kMaxKappa + 1];
  const int* kapd;                // kappa[d], d = 0..n-1 (the per-pair lookup of the SWEEP form)
  const double* x64;
  const float* x32;
  const double* invx64;
  const float* invx32;
  const double* cd64;
  const float* cd32;
  const double* Kd64;
  const float* Kd32;
  const double* Kr64;
  const float* Kr32;
  // second pressure level: D = K2 - K1 in both layouts (NULL without a second level);
  // a point with weight w reads K1 + w D
  const double* Kd64_d;
  const float* Kd32_d;
  const double* Kr64_d;
  const float* Kr32_d;
};

struct Tables {
  unsigned* chk;                  // check record of the bounds-checked build (else NULL)
  int S;
  int G;
  int64_t rank_cost[kMaxGrids * kMaxSpecies];  // bin pairs per step of a point of each LPT rank
  int mode;                       // 0 pairwise (Jacobi), 1 SWEEP (Bott's in-place order, FP64)
  int levels;                     // 1: kernels at two pressure levels (per-point weight)
  int gain_split;                 // lanes per gain item (1, 2, 4, 8); 0: chosen per point
  double p1, p2;                  // their pressures, hPa
  double t_min;
  double tau;
  int8_t product[kMaxSpecies * kMaxSpecies];
  int8_t bucket_rank[kMaxGrids * (kMaxSpecies + 1)];  // [g][n stored species] -> LPT rank
  GridDev g[kMaxGrids];
  MathTabs math;
};

// Caller-owned per-point arrays (device pointers).
struct PointsDev {
  int64_t n_points;
  void* spectra;
  const int64_t* offset;
  const uint8_t* grid_id;
  const uint8_t* species_mask;
  const uint8_t* cloudy;
  const float* temperature;
  double* mass_budget;
  double* mass_error;
  int32_t* status;
  const float* pressure;
};

// Weight of the second pressure level at pressure p: (p1 - p) / (p1 - p2) clamped to [0, 1];
// 0 without levels or pressures. Callers have rejected non-finite pressures.
__device__ __forceinline__ double level_weight(const Tables& t, const PointsDev& pd, int p) {
  if (!t.levels || !pd.pressure) return 0.0;
  const double w = (t.p1 - (double)pd.pressure[p]) / (t.p1 - t.p2);
  return fmin(fmax(w, 0.0), 1.0);
}

// Context-owned scratch of one step.
struct Scratch {
  int32_t* block_counts;   // [kNumBuckets][n_blocks]
  int32_t* active_list;    // [n_points]
  int32_t* counters;       // [0] active count, [1] queue head, [2] end of the list part this
                           // call steps, [3] its start
  int64_t n_blocks;
};

// zero entries after every Kr table: a loss item's second row reads one entry past the
// last column's first row
constexpr int kKrPad = 8;
constexpr int kMaxShards = 1024;

// Equal-cost contiguous shards of a cost-ordered list. Grid points are independent (Sec. VI-A),
// so a list split into contiguous parts needs no exchange between the parts. The list is n_runs
// runs; run r holds cnt[r] entries of cost cost[r] >= 0 each. With T the total cost, bound q of
// W (q = 0..W) is the first position whose cost prefix reaches ceil(q T / W) (bound 0 is 0,
// bound W the entry count), so every shard's cost lies within one entry's cost (plus one) of
// T / W. Integer arithmetic only: the same bounds on the host and on the device. Callers keep
// W <= kMaxShards and T below 2^62 / W.
__host__ __device__ inline int64_t shard_bound(const int64_t* cnt, const int64_t* cost, int n_runs, int W, int q) {
  int64_t T = 0, N = 0;
  for (int r = 0; r < n_runs; ++r) {
    T += cnt[r] * cost[r];
    N += cnt[r];
  }
  if (q <= 0) return 0;
  if (q >= W) return N;
  const int64_t target = ((int64_t)q * T + W - 1) / W;
  int64_t pos = 0, pre = 0;
  for (int r = 0; r < n_runs; ++r) {
    const int64_t run = cnt[r] * cost[r];
    if (pre + run >= target) {
      const int64_t need = target - pre;
      return pos + (need > 0 ? (need + cost[r] - 1) / cost[r] : 0);  // need > 0 implies cost[r] > 0
    }
    pre += run;
    pos += cnt[r];
  }
  return N;
}

constexpr int kCompactThreads = 256;

// compact.cu: classify, order, and (n_shards > 1) keep shard `shard` of the ordered list
cudaError_t launch_compact(const Tables& t, const PointsDev& p, int64_t n_points, const Scratch& s,
                           cudaStream_t stream, int shard = 0, int n_shards = 1);

// coal_kernel.cu
struct CoalLaunch {
  int block_dim;
  int grid_dim;
  size_t smem;
};
size_t coal_smem_bytes(const Tables& t, int precision);  // dynamic shared memory of one CTA
cudaError_t coal_plan(const Tables& t, int precision, int block_dim, int n_sms, CoalLaunch* out);
cudaError_t launch_coal(const Tables& t, int precision, const PointsDev& p, const Scratch& s, double dt,
                        int n_steps, const CoalLaunch& plan, cudaStream_t stream);
// WRF-layout fields (the public fsbm_wrf_state, resolved): memory extents, tile extents and the
// carried species in slot order.
struct WrfDev {
  unsigned* chk;                // check record of the bounds-checked build (else NULL)
  const void* ff[kMaxSpecies];  // by slot (species id sp[s])
  int ns;
  int n;                        // bins of the grid
  int grid;
  unsigned mask;                // species mask of every point
  const float* temperature;
  const uint8_t* predicate;
  const float* pressure;
  int32_t* status;
  double* mass_budget;
  double* mass_error;
  int ims, kms, jms, im, km, jm;  // memory origin and extents
  int its, kts, jts, ti, tk, tj;  // tile origin and extents
};
// wrf_frontend.cu: tile -> packed points (metadata and spectra), and back
cudaError_t launch_wrf_pack(const WrfDev& w, int precision, const PointsDev& pk, int64_t n_tile, double t_min,
                            cudaStream_t stream);
cudaError_t launch_wrf_unpack(const WrfDev& w, int precision, const PointsDev& pk, int64_t n_tile,
                              cudaStream_t stream);

// sweep_kernel.cu: the SWEEP form, one thread per point (launched by launch_coal when mode = 1)
cudaError_t sweep_plan(int block_dim, int n_sms, CoalLaunch* out);
cudaError_t launch_sweep(const Tables& t, const PointsDev& p, const Scratch& s, double dt, int n_steps,
                         const CoalLaunch& plan, cudaStream_t stream);
// Largest errors of the FP64 helpers over a fixed sweep of arguments (written to out[0..4] on
// device): fsbm_log (absolute, relative where |ln x| > 1), fsbm_exp, the e^y - 1 of
// fsbm_exp_em1 (relative, against CUDA's log, exp, expm1), fsbm_rsqrt and fsbm_rcp (relative).
cudaError_t launch_math_check(const Tables& t, double* out, cudaStream_t stream);

}  // namespace fsbm
