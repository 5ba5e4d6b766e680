// sweep_kernel.cu -- Bott's sequential in-place order (SWEEP) on the GPU, FP64.
//
// Bott's flux method as published updates a point's bins pair by pair, each pair reading the
// spectrum its predecessors left (Bott 1998; the routine the paper ports is coal_bott_new,
// Sec. III, Listing 1). The result depends on the visiting order, so there is no parallelism
// inside a point: this kernel gives each grid point one thread, which is the paper's own
// mapping of the collision loop (one OpenMP-offload thread per point, Sec. VI-B, Listing 6).
// It is the cross-check form next to the pairwise kernel; it runs in FP64 only.
//
// Per point and step, in this order:
//   1. budget B = sum M (species then bins, sequential), active ranges [lo, hi] per species;
//   2. pairs: species pairs (a <= b) by slot, i ascending, j ascending (j >= i for a = b), over
//      the active ranges fixed at step start. Each pair reads the current M:
//        N_i = M_i / x_i, N_j = M_j / x_j, C = K N_i N_j dt (times 1/2 on the same-species
//        diagonal), capped so that C x_i <= M_i and C x_j <= M_j (2 C x_i <= M_i on the
//        diagonal; no cap on bin j when the product lands in bin j itself), the bin whose
//        cap decided C ending at exactly 0 (the exact value of M - (M / x) x);
//        the partners lose C x_i and C x_j, bin k = max(i,j) + kappa(|i-j|) of the product
//        species gains dM = C (x_i + x_j) split by Bott's flux with g_k = M_k + dM read now
//        (M_j + C x_i when bin k is partner bin j itself);
//        bins i and j are set to 0 if round-off left them below;
//   3. mass error |sum M - B| / B, then M *= B / sum M.
// The spectrum is updated where it lies (the caller's buffer, through L1/L2): one thread walks
// a few KB, and the FP64 pipe, not memory, bounds the pair loop.
//
// This file is compiled with -fmad=false: every product and sum rounds on its own, as in the
// C oracle, so that the two sides differ only through the math library (log, exp, expm1).
// Where a pair's product lands in its own partner bin j (k = j), bin j's content before the
// flux is M_j - C x_j + C (x_i + x_j) = M_j + C x_i, formed as that sum: the difference of
// the two large terms would cancel when C x_j is far above M_j.
#include <cfloat>
#include <cmath>

#include "fsbm_internal.cuh"

namespace fsbm {
namespace {

// Bott's flux of dM from bin k (content g_k after the deposit) toward bin k+1.
__device__ __forceinline__ double sweep_flux(double dM, double g_k, double M_k1, double c) {
  const double x1 = log(M_k1 / g_k + kBottEps);
  double F;
  if (x1 == 0.0)
    F = dM * c;
  else if (isinf(x1))  // the ratio overflowed: the limit is all of dM (c > 0) or nothing
    F = c > 0.0 ? dM : 0.0;
  else
    F = dM * exp(0.5 * x1) * (-expm1(-c * x1)) / x1;
  return fmin(fmax(F, 0.0), dM);
}

__global__ void k_sweep(Tables t, PointsDev pd, const int32_t* __restrict__ list, const int32_t* counters,
                        double dt, int n_steps) {
  const int q0 = counters[1], q1 = counters[2];  // the list part this call steps
  const int S = t.S;
  for (int q = q0 + blockIdx.x * blockDim.x + threadIdx.x; q < q1; q += gridDim.x * blockDim.x) {
    if (FSBM_CHECKED_BUILD && !FSBM_OK(t.chk, q, counters[0])) break;
    const int p = list[q];
    if (FSBM_CHECKED_BUILD && !(FSBM_OK(t.chk, p, pd.n_points) && FSBM_OK(t.chk, pd.grid_id[p], t.G))) continue;
    const GridDev& G = t.g[pd.grid_id[p]];
    const int n = G.n;
    const unsigned mask = pd.species_mask[p];
    int sp[kMaxSpecies];
    int ns = 0;
    for (int a = 0; a < S; ++a)
      if (mask >> a & 1u) sp[ns++] = a;
    if (FSBM_CHECKED_BUILD && !FSBM_OK(t.chk, pd.offset[p + 1] - pd.offset[p] - (int64_t)ns * n, 1)) continue;
    double* M = reinterpret_cast<double*>(pd.spectra) + pd.offset[p];
    const int E = ns * n;
    bool bad = false;
    double B0 = 0.0;
    for (int e = 0; e < E; ++e) {
      const double v = M[e];
      bad |= !(v >= 0.0) || !(v <= DBL_MAX);
      B0 += v;
    }
    if (bad) {
      pd.status[p] = 2;
      pd.mass_budget[p] = 0.0;
      pd.mass_error[p] = 0.0;
      continue;
    }
    if (!(B0 > 0.0)) {
      pd.status[p] = 4;
      pd.mass_budget[p] = 0.0;
      pd.mass_error[p] = 0.0;
      continue;
    }
    // product slot of every slot pair
    int cs_of[kMaxSpecies * kMaxSpecies];
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) {
        const int prod = t.product[sp[a] * S + sp[b]];
        cs_of[a * kMaxSpecies + b] = prod == sp[a] ? a : b;
      }
    const double* __restrict__ x = G.x64;
    const double* __restrict__ Kr = G.Kr64;
    const double* __restrict__ cd = G.cd64;
    const int* __restrict__ kapd = G.kapd;
    // kernels at two pressure levels: K1 + w (K2 - K1) (w = 0: the first table alone)
    const double wlev = level_weight(t, pd, p);
    const double* __restrict__ Krd = wlev != 0.0 ? G.Kr64_d : nullptr;
    int status = 0;
    double emax = 0.0;
    for (int step = 0; step < n_steps; ++step) {
      double B = 0.0;
      for (int e = 0; e < E; ++e) B += M[e];
      int lo[kMaxSpecies], hi[kMaxSpecies];
      for (int a = 0; a < ns; ++a) {
        double mx = 0.0;
        for (int k = 0; k < n; ++k) mx = fmax(mx, M[a * n + k]);
        const double thr = t.tau * mx;
        lo[a] = n;
        hi[a] = -1;
        for (int k = 0; k < n; ++k) {
          const double v = M[a * n + k];
          if (v > 0.0 && v >= thr) {
            lo[a] = min(lo[a], k);
            hi[a] = k;
          }
        }
      }
      for (int sa = 0; sa < ns; ++sa) {
        for (int sb = sa; sb < ns; ++sb) {
          const int cs = cs_of[sa * kMaxSpecies + sb];
          const double* __restrict__ Kab = Kr + (size_t)(sp[sa] * S + sp[sb]) * n * n;  // [j][i]
          double* Ma = M + sa * n;
          double* Mb = M + sb * n;
          double* Mc = M + cs * n;
          for (int i = lo[sa]; i <= hi[sa]; ++i) {
            const double xi = x[i];
            for (int j = (sa == sb) ? i : lo[sb]; j <= hi[sb]; ++j) {
              const double xj = x[j];
              const double Ni = Ma[i] / xi, Nj = Mb[j] / xj;
              const int dd = i < j ? j - i : i - j;
              if (FSBM_CHECKED_BUILD && !(FSBM_OK(t.chk, i, n) && FSBM_OK(t.chk, j, n) && FSBM_OK(t.chk, cs, ns)))
                continue;
              const int k = (i > j ? i : j) + kapd[dd];
              double K = __ldg(Kab + (size_t)j * n + i);
              if (Krd) K = K + wlev * __ldg(Krd + (size_t)(sp[sa] * S + sp[sb]) * n * n + (size_t)j * n + i);
              double C;
              int emptied = 0;  // the bin whose cap decided C (1: i, 2: j) ends at exactly 0
              const bool diag = sa == sb && i == j;
              if (diag) {
                C = 0.5 * K * Ni * Nj * dt;
                const double cap = Ma[i] / (2.0 * xi);
                if (C > cap) {
                  C = cap;
                  status |= 1;
                  emptied = 1;
                }
              } else {
                C = K * Ni * Nj * dt;
                const double capi = Ma[i] / xi;
                if (C > capi) {
                  C = capi;
                  status |= 1;
                  emptied = 1;
                }
                if (!(cs == sb && k == j)) {
                  const double capj = Mb[j] / xj;
                  if (C > capj) {
                    C = capj;
                    status |= 1;
                    emptied = 2;
                  }
                }
              }
              const double dM = C * (xi + xj);
              if (!(dM > 0.0)) continue;
              // the product lands in partner bin j itself: that bin's content before the flux
              // is M_j - C x_j + dM = M_j + C x_i, formed as that sum
              const bool into_j = cs == sb && k == j;
              if (diag) {
                Ma[i] = emptied ? 0.0 : Ma[i] - 2.0 * C * xi;
              } else {
                Ma[i] = emptied == 1 ? 0.0 : Ma[i] - C * xi;
                if (!into_j) Mb[j] = emptied == 2 ? 0.0 : Mb[j] - C * xj;
              }
              if (k >= n - 1) {
                // the top bin keeps what reaches or passes it
                Mc[n - 1] = into_j ? Mb[j] + C * xi : Mc[n - 1] + dM;
              } else {
                // Courant number from its definition, (x_i + x_j - x_k) / (x_{k+1} - x_k); an
                // exact landing (c(d) = 0 in the table) stays 0
                const double c = cd[dd] == 0.0 ? 0.0 : (xi + xj - x[k]) / (x[k + 1] - x[k]);
                const double g_k = into_j ? Mb[j] + C * xi : Mc[k] + dM;
                const double F = sweep_flux(dM, g_k, Mc[k + 1], c);
                Mc[k] = g_k - F;
                Mc[k + 1] += F;
              }
              if (Ma[i] < 0.0) Ma[i] = 0.0;
              if (Mb[j] < 0.0) Mb[j] = 0.0;
            }
          }
        }
      }
      double sum = 0.0;
      for (int e = 0; e < E; ++e) sum += M[e];
      emax = fmax(emax, fabs(sum - B) / B);
      const double scale = B / sum;
      for (int e = 0; e < E; ++e) M[e] *= scale;
    }
    pd.status[p] = status;
    pd.mass_budget[p] = B0;
    pd.mass_error[p] = emax;
  }
}

}  // namespace

cudaError_t sweep_plan(int block_dim, int n_sms, CoalLaunch* out) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep, block_dim, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  out->block_dim = block_dim;
  out->grid_dim = per_sm * n_sms;
  out->smem = 0;
  return cudaSuccess;
}

cudaError_t launch_sweep(const Tables& t, const PointsDev& p, const Scratch& s, double dt, int n_steps,
                         const CoalLaunch& plan, cudaStream_t stream) {
  k_sweep<<<plan.grid_dim, plan.block_dim, 0, stream>>>(t, p, s.active_list, s.counters, dt, n_steps);
  return cudaGetLastError();
}

}  // namespace fsbm
