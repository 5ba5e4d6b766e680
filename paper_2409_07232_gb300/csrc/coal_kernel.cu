// coal_kernel.cu -- the persistent collision-coalescence kernel (both precision forms).
//
// One CTA owns one grid point at a time (the unit coal_bott_new is called on, Sec. III,
// Listing 1) and takes the next point from the compacted, cost-ordered list through an
// atomic queue head until the list is exhausted. The point's spectra live in shared memory
// for all n_steps steps; only the first load and the final store touch the caller's buffer.
// The pair collection kernels are read straight from the L2-resident tables (one FP64 and
// one FP32 copy per layout), one entry per bin pair (the on-demand lookup of Listing 4).
//
// Per step (Bott's flux method, pairwise form):
//   1. budget B = sum M (FP64, fixed reduction tree), active bin range of every species;
//   2. N = M / x;  R^a_i = dt x_i N^a_i sum_{b,j} K N^b_j      (row mat-vec, lane per row);
//      lambda = min(1, M / R) in FP64;
//   3. loss^a_i = dt x_i N^a_i sum_{b,j} K N^b_j min(lambda^a_i, lambda^b_j)
//      (equal to R when no ratio fired anywhere in the point: the pass is skipped);
//   4. gain pass: for every ordered orientation (small-index species s, large-index
//      species l) one lane per target bin k walks the bin distances d of the pairs
//      (m - d, m) whose mass lands in k (m = k - kappa[d]), computes dM and Bott's flux F,
//      and keeps (sum of dM - F) for bin k and (sum of F) for bin k + 1 in registers;
//      all lanes of a warp walk the same d, so the kernel and spectrum loads are
//      contiguous across the warp. Partial sums land in per-orientation shared arrays and
//      are added in a fixed order: the result does not depend on scheduling;
//   5. M' = M - loss + gain (FP64), mass error, round-off negatives to 0, rescale to B.
// FP32_SPLIT runs 2-4 with float values and float sums; 1 and 5 stay FP64.
#include <cfloat>
#include <cstdio>

#include "fsbm_internal.cuh"

namespace fsbm {
namespace {

struct Orient {
  int8_t s, l;      // slots of the small-index and the large-index partner
  int8_t dmin;      // 0, or 1 when the two species' roles are swapped (d = 0 belongs to the
                    // other orientation of the same species pair)
  int8_t half;      // same species: the diagonal pair counts once, h = 1/2
  int8_t c;         // slot of the product species
  int table;        // element offset of Kd[s][l] in the grid's table
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Deterministic block sum of one value per thread (fixed butterfly + fixed warp order).
__device__ double block_sum(double v, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double u = lane < nw ? red[lane] : 0.0;
    u = warp_sum(u);
    if (lane == 0) red[32] = u;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// Bott's flux of mass dM deposited in bin k toward bin k + 1 (see fsbm_coal.h).
__device__ __forceinline__ double bott_flux(double dM, double Mk, double Mk1, double c) {
  const double g = Mk + dM;
  const double x1 = log(Mk1 / g + kBottEps);
  double F;
  if (x1 == 0.0)
    F = dM * c;
  else if (isinf(x1))  // the ratio overflowed: the flux's limit is all of dM (c > 0) or 0
    F = c > 0.0 ? dM : 0.0;
  else
    F = dM * exp(0.5 * x1) * (-expm1(-c * x1)) / x1;
  return fmin(fmax(F, 0.0), dM);
}

// FP32 form. 1e-60 is below FP32's range, so ln(rho + 1e-60) becomes ln(rho) clamped at
// ln(1e-60); the two differ only for rho within a few orders of 1e-60. ln(rho) is capped at
// 80, above which F >= dM for every c > 0 (and F = 0 for c = 0) in either form.
__device__ __forceinline__ float bott_flux(float dM, float Mk, float Mk1, float c) {
  const float g = Mk + dM;
  float x1 = logf(Mk1 / g);
  x1 = fminf(fmaxf(x1, kLnBottEps), 80.f);
  float F;
  if (x1 == 0.f) {
    F = dM * c;
  } else {
    const float z = -c * x1;
    F = (z > 80.f) ? dM : dM * expf(0.5f * x1) * (-expm1f(z)) / x1;
  }
  return fminf(fmaxf(F, 0.f), dM);
}

template <typename T> struct Sel;
template <> struct Sel<double> {
  static __device__ const double* x(const GridDev& g) { return g.x64; }
  static __device__ const double* cd(const GridDev& g) { return g.cd64; }
  static __device__ const double* Kd(const GridDev& g) { return g.Kd64; }
  static __device__ const double* Kr(const GridDev& g) { return g.Kr64; }
};
template <> struct Sel<float> {
  static __device__ const float* x(const GridDev& g) { return g.x32; }
  static __device__ const float* cd(const GridDev& g) { return g.cd32; }
  static __device__ const float* Kd(const GridDev& g) { return g.Kd32; }
  static __device__ const float* Kr(const GridDev& g) { return g.Kr32; }
};

// Shared-memory carve-up for nmax bins and S species (T = pair-arithmetic type).
// Sums are held in FP64 in both forms: the FP32 form adds short runs of pair terms in FP32
// and folds each run into an FP64 total (see Acc).
template <typename T>
struct Smem {
  double* M;      // [S][nmax] FP64 state
  double* loss;   // [S][nmax] R, then loss
  double* stay;   // [S*S][nmax]
  double* up;     // [S*S][nmax]
  T* Mt;          // [S][nmax] state in T (aliases M when T = double)
  T* N;           // [S][nmax]
  T* lam;         // [S][nmax]
  T* xs;          // [nmax]
  static __host__ __device__ size_t bytes(int nmax, int S) {
    size_t b = sizeof(double) * (2 * S * nmax + 2 * S * S * nmax);
    if (sizeof(T) != sizeof(double)) b += sizeof(T) * S * nmax;
    b += sizeof(T) * (2 * S * nmax + nmax);
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(unsigned char* base, int nmax, int S) {
    unsigned char* p = base;
    M = reinterpret_cast<double*>(p);
    p += sizeof(double) * S * nmax;
    loss = reinterpret_cast<double*>(p);
    p += sizeof(double) * S * nmax;
    stay = reinterpret_cast<double*>(p);
    p += sizeof(double) * S * S * nmax;
    up = reinterpret_cast<double*>(p);
    p += sizeof(double) * S * S * nmax;
    if (sizeof(T) != sizeof(double)) {
      Mt = reinterpret_cast<T*>(p);
      p += sizeof(T) * S * nmax;
    } else {
      Mt = reinterpret_cast<T*>(M);
    }
    N = reinterpret_cast<T*>(p);
    p += sizeof(T) * S * nmax;
    lam = reinterpret_cast<T*>(p);
    p += sizeof(T) * S * nmax;
    xs = reinterpret_cast<T*>(p);
  }
};

// Running sum of pair terms: FP64 adds each term; FP32 adds a run of terms in FP32 and
// folds the run into an FP64 total at flush(), so rounding grows with the run length (16 or
// 32 terms), not with the full sum over a few hundred bins.
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double total() const { return s; }
};
template <> struct Acc<float> {
  float r = 0.f;
  double s = 0.0;
  __device__ __forceinline__ void add(float v) { r += v; }
  __device__ __forceinline__ void flush() {
    s += (double)r;
    r = 0.f;
  }
  __device__ __forceinline__ double total() const { return s + (double)r; }
};
constexpr int kGainRun = 16;
constexpr int kLossRun = 32;

// Gain pass for one (orientation, block of 32 target bins) warp task.
template <typename T, bool LIMITED>
__device__ __forceinline__ void gain_task(const GridDev& G, const Smem<T>& sm, const Orient& o, const int* lo,
                                          const int* hi, int k, T dt, double* out_stay, double* out_up) {
  const int n = G.n;
  Acc<T> stay, up;
  if (k >= 1 && k < n) {
    const T* __restrict__ Kd = Sel<T>::Kd(G) + o.table;
    const T* __restrict__ cd = Sel<T>::cd(G);
    const T* Ns = sm.N + o.s * n;
    const T* Nl = sm.N + o.l * n;
    const T* Ls = sm.lam + o.s * n;
    const T* Ll = sm.lam + o.l * n;
    const int lo_s = lo[o.s], hi_s = hi[o.s], lo_l = lo[o.l], hi_l = hi[o.l];
    const bool top = (k == n - 1);
    // regular target: pairs with m + kappa[d] == k; top bin: every pair with m + kappa[d] >= n-1
    // stays there without a flux
    const T Mk = top ? T(0) : sm.Mt[o.c * n + k];
    const T Mk1 = top ? T(0) : sm.Mt[o.c * n + k + 1];
    for (int kap = 0; kap <= G.kappa_max; ++kap) {
      const int mlo = top ? max(n - 1 - kap, lo_l) : max(k - kap, lo_l);
      const int mhi = top ? min(n - 1, hi_l) : min(k - kap, hi_l);
      for (int m = mlo; m <= mhi; ++m) {
        const int d0 = max(max(G.d_lo[kap], (int)o.dmin), m - hi_s);
        const int d1 = min(G.d_hi[kap], m - lo_s);
        const T nl = Nl[m] * dt;
        const T xl = sm.xs[m];
        const T ll = LIMITED ? Ll[m] : T(1);
        for (int r0 = d0; r0 <= d1; r0 += kGainRun) {
          const int r1 = min(d1, r0 + kGainRun - 1);
          for (int d = r0; d <= r1; ++d) {
            const int i = m - d;
            T C = __ldg(Kd + (size_t)d * n + m) * Ns[i] * nl;
            if (LIMITED) C *= (Ls[i] < ll ? Ls[i] : ll);
            if (o.half && d == 0) C *= T(0.5);
            const T dM = C * (sm.xs[i] + xl);
            if (dM > T(0)) {
              if (top) {
                stay.add(dM);
              } else {
                const T F = bott_flux(dM, Mk, Mk1, __ldg(cd + d));
                stay.add(dM - F);
                up.add(F);
              }
            }
          }
          stay.flush();
          up.flush();
        }
      }
    }
  }
  *out_stay = stay.total();
  *out_up = up.total();
}

template <typename T>
struct StoreOf { using type = T; };

template <typename T>
__global__ void k_coal(Tables t, PointsDev pd, const int32_t* __restrict__ list, int32_t* counters, double dt,
                       int n_steps, int nmax) {
  using Store = typename StoreOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ Orient ori[kMaxOrient];
  __shared__ int s_lo[kMaxSpecies], s_hi[kMaxSpecies], s_sp[kMaxSpecies];
  __shared__ int s_next;

  const int S = t.S;
  Smem<T> sm;
  sm.carve(smem_raw, nmax, S);
  const int tid = threadIdx.x, NT = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = NT >> 5;
  const int n_active = counters[0];
  const T dtT = (T)dt;

  for (;;) {
    if (tid == 0) s_next = atomicAdd(&counters[1], 1);
    __syncthreads();
    const int idx = s_next;
    __syncthreads();
    if (idx >= n_active) break;
    const int p = list[idx];
    const int g = pd.grid_id[p];
    const GridDev& G = t.g[g];
    const int n = G.n;
    const unsigned mask = pd.species_mask[p];
    const int ns = __popc(mask);
    const int64_t off = pd.offset[p];
    Store* spec = reinterpret_cast<Store*>(pd.spectra) + off;
    const int E = ns * n;

    if (tid == 0) {
      int q = 0;
      for (int a = 0; a < S; ++a)
        if (mask >> a & 1u) s_sp[q++] = a;
    }
    // load the spectrum (FP64 on chip) and the bin masses
    bool bad = false;
    double part = 0.0;
    for (int e = tid; e < E; e += NT) {
      const double v = (double)spec[e];
      bad |= !(v >= 0.0) || !(v <= DBL_MAX);
      sm.M[e] = v;
      part += v;
    }
    for (int k = tid; k < n; k += NT) sm.xs[k] = Sel<T>::x(G)[k];
    if (__syncthreads_or(bad)) {
      if (tid == 0) {
        pd.status[p] = 2;
        pd.mass_budget[p] = 0.0;
        pd.mass_error[p] = 0.0;
      }
      continue;
    }
    const double B0 = block_sum(part, red);
    if (!(B0 > 0.0)) {
      if (tid == 0) {
        pd.status[p] = 4;
        pd.mass_budget[p] = 0.0;
        pd.mass_error[p] = 0.0;
      }
      continue;
    }
    // orientation list: same species once; each cross pair in both index orders
    if (tid == 0) {
      int q = 0;
      const size_t nn = (size_t)n * n;
      for (int a = 0; a < ns; ++a)
        for (int b = a; b < ns; ++b) {
          const int ia = s_sp[a], ib = s_sp[b];
          const int prod = t.product[ia * S + ib];
          const int cs = (prod == ia) ? a : b;
          ori[q++] = Orient{(int8_t)a, (int8_t)b, 0, (int8_t)(a == b), (int8_t)cs, (int)((ia * S + ib) * nn)};
          if (a != b) ori[q++] = Orient{(int8_t)b, (int8_t)a, 1, 0, (int8_t)cs, (int)((ib * S + ia) * nn)};
        }
    }
    __syncthreads();
    const int O = ns * ns;
    const int nkb = (n + 31) >> 5;

    int status = 0;
    double emax = 0.0;
    for (int step = 0; step < n_steps; ++step) {
      // 1. budget and active ranges
      double ps = 0.0;
      for (int e = tid; e < E; e += NT) ps += sm.M[e];
      const double Bs = block_sum(ps, red);
      for (int a = warp; a < ns; a += nw) {
        const double* Ma = sm.M + a * n;
        double mx = 0.0;
        for (int k = lane; k < n; k += 32) mx = fmax(mx, Ma[k]);
        mx = warp_max(mx);
        const double thr = t.tau * mx;
        int lo = n, hi = -1;
        for (int k = lane; k < n; k += 32) {
          const double v = Ma[k];
          if (v > 0.0 && v >= thr) {
            lo = min(lo, k);
            hi = max(hi, k);
          }
        }
        lo = warp_min_i(lo);
        hi = warp_max_i(hi);
        if (lane == 0) {
          s_lo[a] = lo;
          s_hi[a] = hi;
        }
      }
      for (int e = tid; e < E; e += NT) {
        const int k = e % n;
        const double m = sm.M[e];
        sm.N[e] = (T)(m / Sel<double>::x(G)[k]);
        if (sizeof(T) != sizeof(double)) sm.Mt[e] = (T)m;
      }
      __syncthreads();

      // 2. requested loss and limiter ratios
      const T* __restrict__ Kr = Sel<T>::Kr(G);
      bool fired = false;
      for (int r = tid; r < E; r += NT) {
        const int a = r / n, i = r - a * n;
        double R = 0.0;
        double lamd = 1.0;
        if (i >= s_lo[a] && i <= s_hi[a]) {
          Acc<T> acc;
          for (int b = 0; b < ns; ++b) {
            const T* Kab = Kr + (size_t)(s_sp[a] * S + s_sp[b]) * n * n + i;
            const T* Nb = sm.N + b * n;
            for (int j0 = s_lo[b]; j0 <= s_hi[b]; j0 += kLossRun) {
              const int j1 = min(s_hi[b], j0 + kLossRun - 1);
              for (int j = j0; j <= j1; ++j) acc.add(__ldg(Kab + (size_t)j * n) * Nb[j]);
              acc.flush();
            }
          }
          R = dt * sm.M[r] * acc.total();
          if (R > 0.0 && sm.M[r] / R < 1.0) {
            lamd = sm.M[r] / R;
            fired = true;
          }
        }
        sm.loss[r] = R;
        sm.lam[r] = (T)lamd;
      }
      const bool limited = __syncthreads_or(fired);
      if (limited) status |= 1;

      // 3. limited losses
      if (limited) {
        for (int r = tid; r < E; r += NT) {
          const int a = r / n, i = r - a * n;
          if (i < s_lo[a] || i > s_hi[a]) continue;
          const T li = sm.lam[r];
          Acc<T> acc;
          for (int b = 0; b < ns; ++b) {
            const T* Kab = Kr + (size_t)(s_sp[a] * S + s_sp[b]) * n * n + i;
            const T* Nb = sm.N + b * n;
            const T* Lb = sm.lam + b * n;
            for (int j0 = s_lo[b]; j0 <= s_hi[b]; j0 += kLossRun) {
              const int j1 = min(s_hi[b], j0 + kLossRun - 1);
              for (int j = j0; j <= j1; ++j) {
                const T phi = Lb[j] < li ? Lb[j] : li;
                acc.add(__ldg(Kab + (size_t)j * n) * Nb[j] * phi);
              }
              acc.flush();
            }
          }
          sm.loss[r] = dt * sm.M[r] * acc.total();
        }
      }

      // 4. gains
      for (int task = warp; task < O * nkb; task += nw) {
        const int oi = task / nkb, kb = task - oi * nkb;
        const int k = kb * 32 + lane;
        double st_, up_;
        if (limited)
          gain_task<T, true>(G, sm, ori[oi], s_lo, s_hi, k, dtT, &st_, &up_);
        else
          gain_task<T, false>(G, sm, ori[oi], s_lo, s_hi, k, dtT, &st_, &up_);
        if (k < n) {
          sm.stay[oi * n + k] = st_;
          sm.up[oi * n + k] = up_;
        }
      }
      __syncthreads();

      // 5. update, mass error, clamp, renormalise
      double pre = 0.0, post = 0.0;
      for (int e = tid; e < E; e += NT) {
        const int c = e / n, k = e - c * n;
        double gsum = 0.0;
        for (int q = 0; q < O; ++q) {
          if (ori[q].c != c) continue;
          gsum += sm.stay[q * n + k];
          if (k > 0) gsum += sm.up[q * n + k - 1];
        }
        double v = sm.M[e] - sm.loss[e] + gsum;
        pre += v;
        if (v < 0.0) v = 0.0;
        post += v;
        sm.M[e] = v;
      }
      const double spre = block_sum(pre, red);
      const double spost = block_sum(post, red);
      const double err = fabs(spre - Bs) / Bs;
      emax = fmax(emax, err);
      const double scale = Bs / spost;
      for (int e = tid; e < E; e += NT) sm.M[e] = sm.M[e] * scale;
      __syncthreads();
    }

    for (int e = tid; e < E; e += NT) spec[e] = (Store)sm.M[e];
    if (tid == 0) {
      pd.status[p] = status;
      pd.mass_budget[p] = B0;
      pd.mass_error[p] = emax;
    }
    (void)lane;
  }
}

template <typename T>
cudaError_t plan_t(const Tables& t, int block_dim, int n_sms, CoalLaunch* out) {
  int nmax = 0;
  for (int g = 0; g < t.G; ++g) nmax = t.g[g].n > nmax ? t.g[g].n : nmax;
  const size_t smem = Smem<T>::bytes(nmax, t.S);
  cudaError_t e = cudaFuncSetAttribute(k_coal<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coal<T>, block_dim, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  out->block_dim = block_dim;
  out->grid_dim = per_sm * n_sms;
  out->smem = smem;
  return cudaSuccess;
}

}  // namespace

cudaError_t coal_plan(const Tables& t, int precision, int block_dim, int n_sms, CoalLaunch* out) {
  return precision == 0 ? plan_t<double>(t, block_dim, n_sms, out) : plan_t<float>(t, block_dim, n_sms, out);
}

cudaError_t launch_coal(const Tables& t, int precision, const PointsDev& p, const Scratch& s, double dt,
                        int n_steps, const CoalLaunch& plan, cudaStream_t stream) {
  int nmax = 0;
  for (int g = 0; g < t.G; ++g) nmax = t.g[g].n > nmax ? t.g[g].n : nmax;
  if (precision == 0)
    k_coal<double><<<plan.grid_dim, plan.block_dim, plan.smem, stream>>>(t, p, s.active_list, s.counters, dt,
                                                                         n_steps, nmax);
  else
    k_coal<float><<<plan.grid_dim, plan.block_dim, plan.smem, stream>>>(t, p, s.active_list, s.counters, dt,
                                                                        n_steps, nmax);
  return cudaGetLastError();
}

}  // namespace fsbm
