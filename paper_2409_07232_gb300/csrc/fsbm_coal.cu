// fsbm_coal.cu -- host side of the C ABI declared in include/fsbm_coal.h.
//
// fsbm_coal_init derives every grid's pair tables and lays the tabulated pair kernels out
// for the device once, replacing the per-call kernel filling the paper profiled in
// kernals_ks (Sec. VI-A, Listing 3) with a lookup of one entry per bin pair (Listing 5).
// fsbm_coal_step runs the compaction pass (the predicate array of Sec. VI-B, Listing 6) and
// the persistent collision kernel on the caller's stream, optionally as a CUDA-graph replay.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fsbm_coal.h"
#include "fsbm_internal.cuh"

using namespace fsbm;

// Device tables of a context (kernel layouts, bin grids, math tables), shared by the context
// and its replicas (fsbm_coal_clone) and freed with the last of them.
struct TableStore {
  std::vector<void*> allocs;
  ~TableStore() {
    for (void* p : allocs) cudaFree(p);
  }
};

struct fsbm_coal_ctx {
  int S = 0, G = 0, precision = 0, device = 0, n_sms = 0;
  cudaStream_t stream = nullptr;
  Tables t{};
  std::shared_ptr<TableStore> tables = std::make_shared<TableStore>();
  // step scratch
  Scratch scratch{};
  int64_t cap_points = -1;
  // host-pointer mirrors for fsbm_coal_step_host
  void* h_spectra = nullptr;
  size_t h_spectra_bytes = 0;
  void* h_meta = nullptr;
  size_t h_meta_bytes = 0;
  // packed copy of a WRF-layout tile for fsbm_coal_step_wrf
  void* wrf_spec = nullptr;
  size_t wrf_spec_bytes = 0;
  void* wrf_meta = nullptr;
  size_t wrf_meta_bytes = 0;
  // launch plan
  int block_dim = 256;
  CoalLaunch plan{};
  bool plan_valid = false;
  // CUDA graph of the last argument set
  bool graph_enabled = false;
  cudaStream_t cap_stream = nullptr;  // private stream the launch sequence is captured on
  cudaGraphExec_t gexec = nullptr;
  PointsDev g_points{};
  int64_t g_n = -1;
  double g_dt = 0.0;
  int g_steps = -1;
  CoalLaunch g_plan{};
  int g_shard = 0, g_nshards = 1;
  bool last_replayed = false;
  int64_t last_n = 0;
  int tune_cache_hit = 0;
  // CUDA-event timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_coal, ev_step;
  std::string err;
};

namespace {

const char* kNullCtxMsg = "fsbm_coal: null context";

// NVTX range around an entry point (and its compaction / collision enqueues), so that a timeline
// from a profiler shows the library's calls by name. Costs nothing measurable without a tool.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

fsbm_status fail(fsbm_coal_ctx* c, fsbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

fsbm_status cuda_fail(fsbm_coal_ctx* c, cudaError_t e, const char* what) {
  const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? FSBM_E_OOM : FSBM_E_CUDA, m);
}

#define CU(ctx, call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int pair_index(int S, int a, int b) { return a * S - a * (a - 1) / 2 + (b - a); }

// Kernel of species a bin i with species b bin j from the caller's [pair a<=b][n][n] block.
double kern_entry(const double* Kg, int S, int n, int a, int i, int b, int j) {
  const size_t nn = (size_t)n * n;
  if (a < b) return Kg[(size_t)pair_index(S, a, b) * nn + (size_t)i * n + j];
  if (a > b) return Kg[(size_t)pair_index(S, b, a) * nn + (size_t)j * n + i];
  const int lo = std::min(i, j), hi = std::max(i, j);
  return Kg[(size_t)pair_index(S, a, a) * nn + (size_t)lo * n + hi];
}

template <typename V>
fsbm_status upload(fsbm_coal_ctx* c, const std::vector<V>& h, const V** out) {
  void* d = nullptr;
  CU(c, cudaMalloc(&d, sizeof(V) * std::max<size_t>(h.size(), 1)));
  c->tables->allocs.push_back(d);
  if (!h.empty()) CU(c, cudaMemcpyAsync(d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, c->stream));
  *out = static_cast<const V*>(d);
  return FSBM_OK;
}

// Target-bin offset kappa(d) and Courant number c(d) of a bin pair at distance d on the grid
// x_k = x0 alpha^k: x_i + x_j = x_max (1 + alpha^-d); its position above bin max(i,j) is
// u = log_alpha(1 + alpha^-d). A position within 1e-9 of an integer is taken as exact
// (c = 0): the i = j pair of the mass-doubling grid lands exactly one bin up.
void pair_offsets(int n, double alpha, std::vector<int>& kap, std::vector<double>& cd) {
  kap.assign(n, 0);
  cd.assign(n, 0.0);
  const double la = std::log(alpha);
  for (int d = 0; d < n; ++d) {
    const double r = std::pow(alpha, -(double)d);
    const double u = std::log1p(r) / la;
    const double m = std::floor(u + 0.5);
    if (std::fabs(u - m) < 1e-9) {
      kap[d] = (int)m;
      cd[d] = 0.0;
    } else {
      const int k = (int)std::floor(u);
      kap[d] = k;
      cd[d] = k == 0 ? r / (alpha - 1.0) : ((1.0 + r) * std::pow(alpha, -(double)k) - 1.0) / (alpha - 1.0);
    }
  }
}

fsbm_status ensure_scratch(fsbm_coal_ctx* c, int64_t n_points) {
  const int64_t nblk = (n_points + kCompactThreads - 1) / kCompactThreads;
  if (n_points > c->cap_points) {
    if (c->gexec) {  // a captured graph refers to the old scratch buffers
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    if (c->scratch.block_counts) cudaFree(c->scratch.block_counts);
    if (c->scratch.active_list) cudaFree(c->scratch.active_list);
    if (c->scratch.counters) cudaFree(c->scratch.counters);
    c->scratch = Scratch{};
    c->cap_points = -1;
    CU(c, cudaMalloc(&c->scratch.block_counts, sizeof(int32_t) * std::max<int64_t>(1, nblk * kNumBuckets)));
    CU(c, cudaMalloc(&c->scratch.active_list, sizeof(int32_t) * std::max<int64_t>(1, n_points)));
    CU(c, cudaMalloc(&c->scratch.counters, sizeof(int32_t) * 4));
    CU(c, cudaMemsetAsync(c->scratch.counters, 0, sizeof(int32_t) * 4, c->stream));
    c->cap_points = n_points;
  }
  c->scratch.n_blocks = nblk;
  return FSBM_OK;
}

fsbm_status ensure_plan(fsbm_coal_ctx* c) {
  if (c->plan_valid) return FSBM_OK;
  CU(c, coal_plan(c->t, c->precision, c->block_dim, c->n_sms, &c->plan));
  c->plan_valid = true;
  return FSBM_OK;
}

fsbm_status check_state(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points, double dt, int32_t n_steps,
                        const char* who = "fsbm_coal_step") {
  const std::string w(who);
  if (!s) return fail(c, FSBM_E_ARG, w + ": state is NULL");
  if (n_points < 0 || n_points > INT32_MAX - 1) return fail(c, FSBM_E_ARG, w + ": n_points must be in [0, 2^31 - 2]");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(c, FSBM_E_ARG, w + ": dt must be finite and >= 0");
  if (n_steps < 0) return fail(c, FSBM_E_ARG, w + ": n_steps must be >= 0");
  if (n_points > 0 && (!s->spectra || !s->offset || !s->grid_id || !s->species_mask || !s->mass_budget ||
                       !s->mass_error || !s->status))
    return fail(c, FSBM_E_ARG, w + ": a required state pointer is NULL");
  return FSBM_OK;
}

PointsDev to_dev(const fsbm_coal_state* s, int64_t n_points) {
  PointsDev p;
  p.n_points = n_points;
  p.spectra = s->spectra;
  p.offset = s->offset;
  p.grid_id = s->grid_id;
  p.species_mask = s->species_mask;
  p.cloudy = s->cloudy;
  p.temperature = s->temperature;
  p.mass_budget = s->mass_budget;
  p.mass_error = s->mass_error;
  p.status = s->status;
  p.pressure = s->pressure;
  return p;
}

bool same_points(const PointsDev& a, const PointsDev& b) { return std::memcmp(&a, &b, sizeof(PointsDev)) == 0; }

fsbm_status take_events(fsbm_coal_ctx* c, std::pair<cudaEvent_t, cudaEvent_t>* out) {
  cudaEvent_t e[2];
  for (int q = 0; q < 2; ++q) {
    if (!c->ev_pool.empty()) {
      e[q] = c->ev_pool.back();
      c->ev_pool.pop_back();
    } else {
      CU(c, cudaEventCreate(&e[q]));
    }
  }
  *out = {e[0], e[1]};
  return FSBM_OK;
}

fsbm_status enqueue(fsbm_coal_ctx* c, const PointsDev& p, int64_t n_points, double dt, int n_steps,
                    const CoalLaunch& plan, bool capturing, int shard, int n_shards) {
  cudaStream_t stream = capturing ? c->cap_stream : c->stream;
  {
    NvtxRange r("fsbm_coal compact");
    CU(c, launch_compact(c->t, p, n_points, c->scratch, stream, shard, n_shards));
  }
  NvtxRange r("fsbm_coal collide");
  const bool timed = c->timing && !capturing;
  std::pair<cudaEvent_t, cudaEvent_t> ev{};
  if (timed) {
    fsbm_status st = take_events(c, &ev);
    if (st != FSBM_OK) return st;
    CU(c, cudaEventRecord(ev.first, c->stream));
  }
  CU(c, launch_coal(c->t, c->precision, p, c->scratch, dt, n_steps, plan, stream));
  if (timed) {
    CU(c, cudaEventRecord(ev.second, c->stream));
    c->ev_coal.push_back(ev);
  }
  return FSBM_OK;
}

fsbm_status launch_step(fsbm_coal_ctx* c, const PointsDev& p, int64_t n_points, double dt, int n_steps, int shard,
                        int n_shards);

fsbm_status run_step(fsbm_coal_ctx* c, const PointsDev& p, int64_t n_points, double dt, int n_steps,
                     int shard = 0, int n_shards = 1) {
  fsbm_status st = ensure_scratch(c, n_points);
  if (st != FSBM_OK) return st;
  st = ensure_plan(c);
  if (st != FSBM_OK) return st;
  c->last_n = n_points;
  std::pair<cudaEvent_t, cudaEvent_t> ev{};
  if (c->timing) {
    st = take_events(c, &ev);
    if (st != FSBM_OK) return st;
    CU(c, cudaEventRecord(ev.first, c->stream));
  }
  st = launch_step(c, p, n_points, dt, n_steps, shard, n_shards);
  if (st != FSBM_OK) return st;
  if (c->timing) {
    CU(c, cudaEventRecord(ev.second, c->stream));
    c->ev_step.push_back(ev);
  }
  return FSBM_OK;
}

fsbm_status launch_step(fsbm_coal_ctx* c, const PointsDev& p, int64_t n_points, double dt, int n_steps, int shard,
                        int n_shards) {
  if (!c->graph_enabled) {
    c->last_replayed = false;
    return enqueue(c, p, n_points, dt, n_steps, c->plan, false, shard, n_shards);
  }
  const bool hit = c->gexec && same_points(p, c->g_points) && n_points == c->g_n && dt == c->g_dt &&
                   n_steps == c->g_steps && std::memcmp(&c->plan, &c->g_plan, sizeof(CoalLaunch)) == 0 &&
                   shard == c->g_shard && n_shards == c->g_nshards;
  if (!hit) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    // capture on the context's own stream (the caller's may be the legacy default stream,
    // which cannot be captured); the graph then runs on the caller's stream
    if (!c->cap_stream) CU(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CU(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    fsbm_status est = enqueue(c, p, n_points, dt, n_steps, c->plan, true, shard, n_shards);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
    if (est != FSBM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return est;
    }
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      c->gexec = nullptr;
      return cuda_fail(c, ce, "cudaGraphInstantiate");
    }
    c->g_points = p;
    c->g_n = n_points;
    c->g_dt = dt;
    c->g_steps = n_steps;
    c->g_plan = c->plan;
    c->g_shard = shard;
    c->g_nshards = n_shards;
  }
  CU(c, cudaGraphLaunch(c->gexec, c->stream));
  c->last_replayed = hit;
  return FSBM_OK;
}

}  // namespace

extern "C" {

fsbm_status fsbm_coal_init(const fsbm_coal_config* cfg, void* stream, fsbm_coal_ctx** out) {
  NvtxRange nvtx_("fsbm_coal_init");
  if (!out) return FSBM_E_ARG;
  *out = nullptr;
  if (!cfg) return FSBM_E_ARG;
  fsbm_coal_ctx* c = new fsbm_coal_ctx();
  auto bail = [&](fsbm_status s) {
    // keep the context only to report the message? no: the caller gets NULL; free everything
    delete c;  // frees the tables allocated so far
    return s;
  };
  const int S = cfg->n_species, G = cfg->n_grids;
  if (S < 1 || S > kMaxSpecies || G < 1 || G > kMaxGrids || !cfg->bins_per_grid || !cfg->x0_g || !cfg->alpha ||
      !cfg->kernels)
    return bail(FSBM_E_ARG);
  if (cfg->precision != FSBM_FP64 && cfg->precision != FSBM_FP32_SPLIT) return bail(FSBM_E_ARG);
  // mode 1 (SWEEP) is Bott's in-place order, FP64 only
  if (cfg->mode != 0 && cfg->mode != 1) return bail(FSBM_E_ARG);
  if (cfg->mode == 1 && cfg->precision != FSBM_FP64) return bail(FSBM_E_UNSUPPORTED);
  if (!std::isfinite(cfg->t_min_K) || !(cfg->active_rel_threshold >= 0.0) || !(cfg->active_rel_threshold < 1.0))
    return bail(FSBM_E_ARG);
  if (cfg->kernels_p2 &&
      (!std::isfinite(cfg->p1_hpa) || !std::isfinite(cfg->p2_hpa) || cfg->p1_hpa == cfg->p2_hpa))
    return bail(FSBM_E_ARG);
  c->t.levels = cfg->kernels_p2 ? 1 : 0;
  c->t.p1 = cfg->p1_hpa;
  c->t.p2 = cfg->p2_hpa;
  c->S = S;
  c->G = G;
  c->precision = cfg->precision;
  c->stream = static_cast<cudaStream_t>(stream);
#ifdef FSBM_CHECKED
  {
    const unsigned* chk = nullptr;
    const std::vector<unsigned> zero(4, 0u);
    if (upload(c, zero, &chk) != FSBM_OK) return bail(FSBM_E_CUDA);
    c->t.chk = const_cast<unsigned*>(chk);
  }
#endif
  c->t.S = S;
  c->t.mode = cfg->mode;
  c->t.G = G;
  c->t.t_min = cfg->t_min_K;
  c->t.tau = cfg->active_rel_threshold;
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b) {
      const int p = cfg->product ? cfg->product[a * S + b] : std::max(a, b);
      const int q = cfg->product ? cfg->product[b * S + a] : std::max(a, b);
      if (p != q || (p != a && p != b)) return bail(FSBM_E_ARG);
      c->t.product[a * S + b] = (int8_t)p;
    }
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return bail(FSBM_E_CUDA);

  // LPT class ranks: costliest (grid, stored-species count) first
  struct Cls { double cost; int g, ns; };
  std::vector<Cls> cls;
  size_t koff = 0;
  const int npairs = S * (S + 1) / 2;
  for (int g = 0; g < G; ++g) {
    const int n = cfg->bins_per_grid[g];
    const double x0 = cfg->x0_g[g], al = cfg->alpha[g];
    if (n < 2 || n > kMaxBins || !(x0 > 0.0) || !std::isfinite(x0) || !(al > 1.0) || !(al <= 2.0))
      return bail(FSBM_E_ARG);
    const double* Kg = cfg->kernels + koff;
    const double* K2g = cfg->kernels_p2 ? cfg->kernels_p2 + koff : nullptr;
    const size_t nn = (size_t)n * n;
    for (size_t e = 0; e < (size_t)npairs * nn; ++e) {
      if (!(Kg[e] >= 0.0) || !std::isfinite(Kg[e])) return bail(FSBM_E_ARG);
      if (K2g && (!(K2g[e] >= 0.0) || !std::isfinite(K2g[e]))) return bail(FSBM_E_ARG);
    }
    koff += (size_t)npairs * nn;
    for (int ns = 1; ns <= S; ++ns)
      cls.push_back(Cls{(double)ns * n * (n + 1) / 2.0 + (double)ns * (ns - 1) / 2.0 * (double)n * n, g, ns});

    GridDev& gd = c->t.g[g];
    gd.chk = c->t.chk;
    gd.n = n;
    gd.inv_n = (unsigned)((uint64_t(1) << 32) / (uint64_t)n + 1);
    std::vector<int> kap;
    std::vector<double> cd;
    pair_offsets(n, al, kap, cd);
    gd.kappa_max = kap[0];
    if (gd.kappa_max > kMaxKappa) return bail(FSBM_E_ARG);
    for (int q = 0; q <= kMaxKappa; ++q) {
      gd.d_lo[q] = n;
      gd.d_hi[q] = -1;
    }
    for (int d = 0; d < n; ++d) {
      if (d > 0 && kap[d] > kap[d - 1]) return bail(FSBM_E_ARG);  // not monotone: not a geometric grid
      gd.d_lo[kap[d]] = std::min(gd.d_lo[kap[d]], d);
      gd.d_hi[kap[d]] = std::max(gd.d_hi[kap[d]], d);
    }
    std::vector<double> x(n), invx(n);
    for (int k = 0; k < n; ++k) {
      x[k] = x0 * std::pow(al, (double)k);
      invx[k] = 1.0 / x[k];
    }
    const int S2 = S * S;
    // the two layouts of one grid's kernel tables
    auto layouts = [&](const double* Kt, std::vector<double>& Kd, std::vector<double>& Kr) {
      Kd.assign((size_t)S2 * nn, 0.0);
      Kr.assign((size_t)S2 * nn + kKrPad, 0.0);
      for (int s = 0; s < S; ++s)
        for (int l = 0; l < S; ++l) {
          double* kr = Kr.data() + (size_t)(s * S + l) * nn;
          // Kd[d][m][s*S+l]: the orientations of one (d, m) sit side by side. Each entry is
          // scaled by 1 + alpha^-d = (x_{m-d} + x_m) / x_m, so that the gain pass forms the
          // pair's mass C (x_i + x_m) as entry * N_i * (M_m dt). The same-species diagonal pair
          // (d = 0, s = l) is counted once with weight 1/2 (a bin collecting itself), so its
          // entry holds K (1 + 1) / 2 and the gain pass needs no weight.
          for (int d = 0; d < n; ++d) {
            const double sd = 1.0 + std::pow(al, -(double)d);
            for (int m = d; m < n; ++m)
              Kd[((size_t)d * n + m) * S2 + (s * S + l)] =
                  kern_entry(Kt, S, n, s, m - d, l, m) * sd * ((d == 0 && s == l) ? 0.5 : 1.0);
          }
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) kr[(size_t)j * n + i] = kern_entry(Kt, S, n, s, i, l, j);
        }
    };
    std::vector<double> Kd, Kr;
    layouts(Kg, Kd, Kr);
    std::vector<float> x32(x.begin(), x.end()), invx32(invx.begin(), invx.end()), cd32(cd.begin(), cd.end()),
        Kd32(Kd.begin(), Kd.end()), Kr32(Kr.begin(), Kr.end());
    fsbm_status st;
    if (K2g) {
      // second pressure level: the differences D = K2 - K1 in both layouts and precisions
      std::vector<double> Kd2, Kr2;
      layouts(K2g, Kd2, Kr2);
      for (size_t e = 0; e < Kd2.size(); ++e) Kd2[e] -= Kd[e];
      for (size_t e = 0; e < Kr2.size(); ++e) Kr2[e] -= Kr[e];
      std::vector<float> Kd2f(Kd2.begin(), Kd2.end()), Kr2f(Kr2.begin(), Kr2.end());
      if ((st = upload(c, Kd2, &gd.Kd64_d)) != FSBM_OK || (st = upload(c, Kd2f, &gd.Kd32_d)) != FSBM_OK ||
          (st = upload(c, Kr2, &gd.Kr64_d)) != FSBM_OK || (st = upload(c, Kr2f, &gd.Kr32_d)) != FSBM_OK ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(st != FSBM_OK ? st : FSBM_E_CUDA);
    }
    if ((st = upload(c, x, &gd.x64)) != FSBM_OK || (st = upload(c, x32, &gd.x32)) != FSBM_OK ||
        (st = upload(c, invx, &gd.invx64)) != FSBM_OK || (st = upload(c, invx32, &gd.invx32)) != FSBM_OK ||
        (st = upload(c, cd, &gd.cd64)) != FSBM_OK || (st = upload(c, cd32, &gd.cd32)) != FSBM_OK ||
        (st = upload(c, kap, &gd.kapd)) != FSBM_OK ||
        (st = upload(c, Kd, &gd.Kd64)) != FSBM_OK || (st = upload(c, Kd32, &gd.Kd32)) != FSBM_OK ||
        (st = upload(c, Kr, &gd.Kr64)) != FSBM_OK || (st = upload(c, Kr32, &gd.Kr32)) != FSBM_OK)
      return bail(st);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(FSBM_E_CUDA);
  }
  {
    // one point's spectra, sums and partial gains live in shared memory: refuse grids whose
    // working set (about 8 (2 S + 2 S^2) n bytes plus 6 to 9 values of the form's width per
    // species and bin) exceeds the device's per-CTA limit (on GB300: 297 bins with 5 species
    // in FP64, 368 in FP32)
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess)
      return bail(FSBM_E_CUDA);
    if (c->t.mode == 0 && coal_smem_bytes(c->t, c->precision) + 1024 > (size_t)optin) return bail(FSBM_E_UNSUPPORTED);
  }
  {
    // tables of the FP64 logarithm and exponential (Tang's table-driven methods), in long double
    std::vector<double> lt(2 * kLogTab), et(2 * kExpTab);
    for (int j = 0; j < kLogTab; ++j) {
      const long double F = 1.0L + (long double)j / 512.0L;
      lt[2 * j] = (double)(1.0L / F);
      lt[2 * j + 1] = (double)logl(F);
    }
    for (int j = 0; j < kExpTab; ++j) {
      const long double v = exp2l((long double)j / 256.0L);
      et[2 * j] = (double)v;
      et[2 * j + 1] = (double)(v - (long double)et[2 * j]);
    }
    fsbm_status st;
    const double* ltd = nullptr;
    const double* etd = nullptr;
    if ((st = upload(c, lt, &ltd)) != FSBM_OK || (st = upload(c, et, &etd)) != FSBM_OK) return bail(st);
    c->t.math.logtab = reinterpret_cast<const double2*>(ltd);  // cudaMalloc: 256-byte aligned
    c->t.math.exptab = reinterpret_cast<const double2*>(etd);
    const long double ln2 = logl(2.0L);
    uint64_t bits;
    const double ln2d = (double)ln2;
    std::memcpy(&bits, &ln2d, sizeof bits);
    bits &= ~uint64_t(0xffffffffu);  // clear 32 low mantissa bits: e * hi exact for |e| < 2^11
    double hi;
    std::memcpy(&hi, &bits, sizeof hi);
    c->t.math.ln2_hi = hi;
    c->t.math.ln2_lo = (double)(ln2 - (long double)hi);
    std::vector<double> ebt(2 * 2048);
    for (int b = 0; b < 2048; ++b) {
      const double e = (double)(b - 1023);
      ebt[2 * b] = e * c->t.math.ln2_hi;  // exact: 21 significant bits times 11
      ebt[2 * b + 1] = e * c->t.math.ln2_lo;
    }
    const double* ebd = nullptr;
    if ((st = upload(c, ebt, &ebd)) != FSBM_OK) return bail(st);
    c->t.math.etab = reinterpret_cast<const double2*>(ebd);
    c->t.math.l256_hi = hi / 256.0;
    c->t.math.l256_lo = c->t.math.ln2_lo / 256.0;
    c->t.math.inv_l256 = (double)(256.0L / ln2);
    c->t.math.ln_eps = std::log(kBottEps);
    c->t.math.sqrt_eps = std::exp(0.5 * c->t.math.ln_eps);
  }
  std::stable_sort(cls.begin(), cls.end(), [](const Cls& a, const Cls& b) { return a.cost > b.cost; });
  std::memset(c->t.bucket_rank, -1, sizeof(c->t.bucket_rank));
  std::memset(c->t.rank_cost, 0, sizeof(c->t.rank_cost));
  for (size_t r = 0; r < cls.size(); ++r) {
    c->t.bucket_rank[cls[r].g * (kMaxSpecies + 1) + cls[r].ns] = (int8_t)r;
    c->t.rank_cost[r] = (int64_t)cls[r].cost;  // an integer below 2^53: exact
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(FSBM_E_CUDA);
  *out = c;
  return FSBM_OK;
}

fsbm_status fsbm_coal_clone(const fsbm_coal_ctx* src, void* stream, fsbm_coal_ctx** out) {
  NvtxRange nvtx_("fsbm_coal_clone");
  if (!out) return FSBM_E_ARG;
  *out = nullptr;
  if (!src) return FSBM_E_ARG;
  fsbm_coal_ctx* c = new fsbm_coal_ctx();
  c->S = src->S;
  c->G = src->G;
  c->precision = src->precision;
  c->device = src->device;
  c->n_sms = src->n_sms;
  c->stream = static_cast<cudaStream_t>(stream);
  c->t = src->t;            // device pointers into the shared tables
  c->tables = src->tables;  // one more holder
  c->block_dim = src->block_dim;
  c->plan_valid = false;    // planned again on the replica's first step (no allocation)
  *out = c;
  return FSBM_OK;
}

fsbm_status fsbm_coal_step(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points, double dt,
                           int32_t n_steps) {
  NvtxRange nvtx_("fsbm_coal_step");
  if (!c) return FSBM_E_ARG;
  fsbm_status st = check_state(c, s, n_points, dt, n_steps);
  if (st != FSBM_OK) return st;
  return run_step(c, to_dev(s, n_points), n_points, dt, n_steps);
}

fsbm_status fsbm_coal_step_shard(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points, double dt,
                                 int32_t n_steps, int32_t shard, int32_t n_shards) {
  NvtxRange nvtx_("fsbm_coal_step_shard");
  if (!c) return FSBM_E_ARG;
  fsbm_status st = check_state(c, s, n_points, dt, n_steps, "fsbm_coal_step_shard");
  if (st != FSBM_OK) return st;
  if (n_shards < 1 || n_shards > kMaxShards || shard < 0 || shard >= n_shards)
    return fail(c, FSBM_E_ARG, "fsbm_coal_step_shard: need 0 <= shard < n_shards <= 1024");
  return run_step(c, to_dev(s, n_points), n_points, dt, n_steps, shard, n_shards);
}

fsbm_status fsbm_coal_shard_bounds(const int64_t* run_count, const int64_t* run_cost, int32_t n_runs,
                                   int32_t n_shards, int64_t* bounds) {
  if (n_runs < 0 || (n_runs > 0 && (!run_count || !run_cost)) || n_shards < 1 || n_shards > kMaxShards || !bounds)
    return FSBM_E_ARG;
  int64_t T = 0;
  for (int r = 0; r < n_runs; ++r) {
    if (run_count[r] < 0 || run_cost[r] < 0) return FSBM_E_ARG;
    if (run_cost[r] > 0 && run_count[r] > ((int64_t)1 << 62) / n_shards / run_cost[r]) return FSBM_E_ARG;
    T += run_count[r] * run_cost[r];
    if (T > ((int64_t)1 << 62) / n_shards) return FSBM_E_ARG;
  }
  for (int q = 0; q <= n_shards; ++q) bounds[q] = shard_bound(run_count, run_cost, n_runs, n_shards, q);
  return FSBM_OK;
}

fsbm_status fsbm_coal_step_host(fsbm_coal_ctx* c, const fsbm_coal_state* h, int64_t n_points, double dt,
                                int32_t n_steps) {
  NvtxRange nvtx_("fsbm_coal_step_host");
  if (!c) return FSBM_E_ARG;
  fsbm_status st = check_state(c, h, n_points, dt, n_steps, "fsbm_coal_step_host");
  if (st != FSBM_OK) return st;
  if (n_points == 0) return FSBM_OK;
  const size_t esz = c->precision == FSBM_FP64 ? sizeof(double) : sizeof(float);
  const int64_t base = h->offset[0], total = h->offset[n_points] - base;
  if (base < 0 || total < 0) return fail(c, FSBM_E_ARG, "fsbm_coal_step_host: offsets must be non-decreasing");
  const size_t spec_bytes = (size_t)total * esz;
  // device mirror of the metadata and outputs: offsets, outputs, then byte arrays
  const size_t n = (size_t)n_points;
  const size_t meta = sizeof(int64_t) * (n + 1) + sizeof(double) * 2 * n + sizeof(int32_t) * n +
                      2 * sizeof(float) * n + 3 * n + 64;
  if (spec_bytes > c->h_spectra_bytes) {
    if (c->h_spectra) cudaFree(c->h_spectra);
    c->h_spectra = nullptr;
    c->h_spectra_bytes = 0;
    CU(c, cudaMalloc(&c->h_spectra, std::max<size_t>(spec_bytes, 16)));
    c->h_spectra_bytes = spec_bytes;
  }
  if (meta > c->h_meta_bytes) {
    if (c->h_meta) cudaFree(c->h_meta);
    c->h_meta = nullptr;
    c->h_meta_bytes = 0;
    CU(c, cudaMalloc(&c->h_meta, meta));
    c->h_meta_bytes = meta;
  }
  char* m = static_cast<char*>(c->h_meta);
  int64_t* d_off = reinterpret_cast<int64_t*>(m);
  m += sizeof(int64_t) * (n + 1);
  double* d_bud = reinterpret_cast<double*>(m);
  m += sizeof(double) * n;
  double* d_err = reinterpret_cast<double*>(m);
  m += sizeof(double) * n;
  int32_t* d_st = reinterpret_cast<int32_t*>(m);
  m += sizeof(int32_t) * n;
  float* d_T = reinterpret_cast<float*>(m);
  m += sizeof(float) * n;
  float* d_P = reinterpret_cast<float*>(m);
  m += sizeof(float) * n;
  uint8_t* d_gid = reinterpret_cast<uint8_t*>(m);
  uint8_t* d_mask = d_gid + n;
  uint8_t* d_cl = d_mask + n;
  char* d_spec = static_cast<char*>(c->h_spectra);
  cudaStream_t sm = c->stream;
  CU(c, cudaMemcpyAsync(d_spec, static_cast<const char*>(h->spectra) + (size_t)base * esz, spec_bytes,
                        cudaMemcpyHostToDevice, sm));
  CU(c, cudaMemcpyAsync(d_off, h->offset, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, sm));
  CU(c, cudaMemcpyAsync(d_gid, h->grid_id, n, cudaMemcpyHostToDevice, sm));
  CU(c, cudaMemcpyAsync(d_mask, h->species_mask, n, cudaMemcpyHostToDevice, sm));
  if (h->cloudy) CU(c, cudaMemcpyAsync(d_cl, h->cloudy, n, cudaMemcpyHostToDevice, sm));
  if (h->temperature) CU(c, cudaMemcpyAsync(d_T, h->temperature, sizeof(float) * n, cudaMemcpyHostToDevice, sm));
  const bool has_p = h->pressure && c->t.levels;
  if (has_p) CU(c, cudaMemcpyAsync(d_P, h->pressure, sizeof(float) * n, cudaMemcpyHostToDevice, sm));
  PointsDev p;
  p.n_points = n_points;
  p.spectra = d_spec - (size_t)base * esz;  // the offsets index from the caller's base
  p.offset = d_off;
  p.grid_id = d_gid;
  p.species_mask = d_mask;
  p.cloudy = h->cloudy ? d_cl : nullptr;
  p.temperature = h->temperature ? d_T : nullptr;
  p.mass_budget = d_bud;
  p.mass_error = d_err;
  p.status = d_st;
  p.pressure = has_p ? d_P : nullptr;
  st = run_step(c, p, n_points, dt, n_steps);
  if (st != FSBM_OK) return st;
  CU(c, cudaMemcpyAsync(static_cast<char*>(h->spectra) + (size_t)base * esz, d_spec, spec_bytes,
                        cudaMemcpyDeviceToHost, sm));
  CU(c, cudaMemcpyAsync(h->mass_budget, d_bud, sizeof(double) * n, cudaMemcpyDeviceToHost, sm));
  CU(c, cudaMemcpyAsync(h->mass_error, d_err, sizeof(double) * n, cudaMemcpyDeviceToHost, sm));
  CU(c, cudaMemcpyAsync(h->status, d_st, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, sm));
  CU(c, cudaStreamSynchronize(sm));
  return FSBM_OK;
}

fsbm_status fsbm_coal_step_wrf(fsbm_coal_ctx* c, const fsbm_wrf_state* w, double dt, int32_t n_steps) {
  NvtxRange nvtx_("fsbm_coal_step_wrf");
  if (!c) return FSBM_E_ARG;
  if (!w) return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: state is NULL");
  if (!(dt >= 0.0) || !std::isfinite(dt) || n_steps < 0)
    return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: dt must be finite and >= 0, n_steps >= 0");
  if (w->grid < 0 || w->grid >= c->G) return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: unknown grid");
  if (w->ime < w->ims || w->kme < w->kms || w->jme < w->jms)
    return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: empty memory ranges");
  const int64_t ti = (int64_t)w->ite - w->its + 1, tk = (int64_t)w->kte - w->kts + 1, tj = (int64_t)w->jte - w->jts + 1;
  if (ti <= 0 || tk <= 0 || tj <= 0) return FSBM_OK;  // empty tile
  if (w->its < w->ims || w->ite > w->ime || w->kts < w->kms || w->kte > w->kme || w->jts < w->jms || w->jte > w->jme)
    return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: tile ranges outside the memory ranges");
  WrfDev d{};
  d.chk = c->t.chk;
  d.ns = 0;
  d.mask = 0;
  for (int a = 0; a < c->S; ++a)
    if (w->ff[a]) {
      d.ff[d.ns++] = w->ff[a];
      d.mask |= 1u << a;
    }
  for (int a = c->S; a < kMaxSpecies; ++a)
    if (w->ff[a]) return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: a field for a species beyond n_species");
  if (d.ns == 0) return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: no species field");
  d.n = c->t.g[w->grid].n;
  d.grid = w->grid;
  d.temperature = w->temperature;
  d.predicate = w->predicate;
  d.pressure = w->pressure;
  d.status = w->status;
  d.mass_budget = w->mass_budget;
  d.mass_error = w->mass_error;
  d.ims = w->ims;
  d.kms = w->kms;
  d.jms = w->jms;
  d.im = w->ime - w->ims + 1;
  d.km = w->kme - w->kms + 1;
  d.jm = w->jme - w->jms + 1;
  d.its = w->its;
  d.kts = w->kts;
  d.jts = w->jts;
  d.ti = (int)ti;
  d.tk = (int)tk;
  d.tj = (int)tj;
  const int64_t n_tile = ti * tk * tj;
  if (n_tile > INT32_MAX - 1) return fail(c, FSBM_E_ARG, "fsbm_coal_step_wrf: more than 2^31 - 2 tile points");
  const size_t esz = c->precision == FSBM_FP64 ? sizeof(double) : sizeof(float);
  const size_t n = (size_t)n_tile;
  const size_t spec_bytes = n * (size_t)d.ns * d.n * esz;
  const size_t meta = sizeof(int64_t) * (n + 1) + sizeof(double) * 2 * n + sizeof(int32_t) * n +
                      2 * sizeof(float) * n + 3 * n + 64;
  if (spec_bytes > c->wrf_spec_bytes) {
    if (c->wrf_spec) cudaFree(c->wrf_spec);
    c->wrf_spec = nullptr;
    c->wrf_spec_bytes = 0;
    if (cudaMalloc(&c->wrf_spec, spec_bytes) != cudaSuccess) {
      cudaGetLastError();
      c->wrf_spec = nullptr;
      return fail(c, FSBM_E_OOM, "fsbm_coal_step_wrf: packed tile buffer");
    }
    c->wrf_spec_bytes = spec_bytes;
  }
  if (meta > c->wrf_meta_bytes) {
    if (c->wrf_meta) cudaFree(c->wrf_meta);
    c->wrf_meta = nullptr;
    c->wrf_meta_bytes = 0;
    if (cudaMalloc(&c->wrf_meta, meta) != cudaSuccess) {
      cudaGetLastError();
      c->wrf_meta = nullptr;
      return fail(c, FSBM_E_OOM, "fsbm_coal_step_wrf: packed tile metadata");
    }
    c->wrf_meta_bytes = meta;
  }
  char* m = static_cast<char*>(c->wrf_meta);
  PointsDev p{};
  p.n_points = n_tile;
  p.offset = reinterpret_cast<int64_t*>(m);
  m += sizeof(int64_t) * (n + 1);
  p.mass_budget = reinterpret_cast<double*>(m);
  m += sizeof(double) * n;
  p.mass_error = reinterpret_cast<double*>(m);
  m += sizeof(double) * n;
  p.status = reinterpret_cast<int32_t*>(m);
  m += sizeof(int32_t) * n;
  float* tbuf = reinterpret_cast<float*>(m);
  m += sizeof(float) * n;
  float* pbuf = reinterpret_cast<float*>(m);
  m += sizeof(float) * n;
  p.grid_id = reinterpret_cast<uint8_t*>(m);
  p.species_mask = reinterpret_cast<uint8_t*>(m) + n;
  p.cloudy = reinterpret_cast<uint8_t*>(m) + 2 * n;
  p.temperature = w->temperature ? tbuf : nullptr;
  p.pressure = (w->pressure && c->t.levels) ? pbuf : nullptr;
  p.spectra = c->wrf_spec;
  d.pressure = p.pressure ? w->pressure : nullptr;
  CU(c, launch_wrf_pack(d, c->precision, p, n_tile, c->t.t_min, c->stream));
  fsbm_status st = run_step(c, p, n_tile, dt, n_steps);
  if (st != FSBM_OK) return st;
  CU(c, launch_wrf_unpack(d, c->precision, p, n_tile, c->stream));
  return FSBM_OK;
}

}  // extern "C"

namespace {

// Launch shapes the autotuner remembers for the process, keyed by everything that changes the
// kernel's cost: the device, precision, mode, kernel levels, bin grids, species count, range
// threshold, step length, steps per call, and the sample's mix of point classes (grid and
// stored-species count, in eighths of the sample).
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;

std::string tune_key(const fsbm_coal_ctx* c, double dt, int n_steps, const int32_t* cls_count, int n_cls, int64_t P) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, c->device);
  std::string k = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount) + "|p" +
                  std::to_string(c->precision) + "|m" + std::to_string(c->t.mode) + "|l" + std::to_string(c->t.levels) +
                  "|S" + std::to_string(c->S);
  char buf[64];
  for (int g = 0; g < c->G; ++g) {
    std::snprintf(buf, sizeof buf, "|g%d:%d", c->t.g[g].n, c->t.g[g].kappa_max);
    k += buf;
  }
  std::snprintf(buf, sizeof buf, "|tau%.17g|dt%.17g|n%d|P%d|", c->t.tau, dt, n_steps, c->t.gain_split);
  k += buf;
  for (int r = 0; r < n_cls; ++r) k += std::to_string(P > 0 ? (8 * (int64_t)cls_count[r] + P / 2) / P : 0) + ",";
  return k;
}

fsbm_status autotune_at(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points, double dt, int n_steps,
                        const char* who) {
  fsbm_status st = check_state(c, s, n_points, dt, n_steps, who);
  if (st != FSBM_OK) return st;
  c->tune_cache_hit = 0;
  if (n_points == 0) return FSBM_OK;
  // The whole batch is classified and ordered, as a step would (on a copy of the spectra and
  // scratch outputs, so the caller's arrays are left alone), which gives its class mix. The
  // timed sample is an even stride through the ordered active list holding about kTuneWork
  // pair updates at the caller's dt and up to 4 of its steps (at least 2432 points, several per
  // resident CTA, so that the last points' tail weighs about as much as in a real call): every
  // class in its share and order, wherever in the batch its points lie, and about 0.1 s per
  // candidate for any grid.
  int64_t off[2];
  CU(c, cudaMemcpyAsync(&off[0], s->offset, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaMemcpyAsync(&off[1], s->offset + n_points, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  const size_t esz = c->precision == FSBM_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)(off[1] - off[0]) * esz;
  const size_t spec_b = (bytes + 15) & ~size_t(15);
  const size_t outb = ((sizeof(double) * 2 + sizeof(int32_t)) * (size_t)n_points + 15) & ~size_t(15);
  char* tmp = nullptr;
  CU(c, cudaMalloc(&tmp, spec_b + outb + sizeof(int32_t) * (size_t)n_points + 64));
  const char* src = static_cast<const char*>(s->spectra) + (size_t)off[0] * esz;
  PointsDev p = to_dev(s, n_points);
  p.spectra = tmp - (size_t)off[0] * esz;
  p.mass_budget = reinterpret_cast<double*>(tmp + spec_b);
  p.mass_error = p.mass_budget + n_points;
  p.status = reinterpret_cast<int32_t*>(p.mass_error + n_points);
  int32_t* sample_list = reinterpret_cast<int32_t*>(tmp + spec_b + outb);
  st = ensure_scratch(c, n_points);
  if (st != FSBM_OK) {
    cudaFree(tmp);
    return st;
  }
  const int64_t nblk = c->scratch.n_blocks;
  // the class mix: first positions of the classes in the ordered list (the scanned counts'
  // first block of every class) and the active count
  const int n_cls = c->G * c->S;
  int32_t first[kNumBuckets + 1] = {};
  cudaError_t ce = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (ce == cudaSuccess) ce = launch_compact(c->t, p, n_points, c->scratch, c->stream);
  for (int r = 0; r < n_cls && ce == cudaSuccess; ++r)
    ce = cudaMemcpyAsync(&first[r], c->scratch.block_counts + (int64_t)r * nblk, sizeof(int32_t),
                         cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(&first[n_cls], c->scratch.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) {
    cudaFree(tmp);
    return cuda_fail(c, ce, who);
  }
  const int64_t n_act = first[n_cls];
  int32_t cls_count[kNumBuckets] = {};
  double work = 0.0;
  for (int r = 0; r < n_cls; ++r) {
    cls_count[r] = first[r + 1] - first[r];
    work += (double)cls_count[r] * (double)c->t.rank_cost[r];
  }
  if (n_act == 0) {  // nothing would be stepped: no candidate to time
    cudaFree(tmp);
    return FSBM_OK;
  }
  const std::string key = tune_key(c, dt, n_steps, cls_count, n_cls, n_act);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      cudaFree(tmp);
      c->block_dim = it->second;
      c->plan_valid = false;
      c->tune_cache_hit = 1;
      return ensure_plan(c);
    }
  }
  const int tune_steps = std::min(n_steps, 4);
  const double kTuneWork = c->precision == FSBM_FP64 ? 1.5e9 : 3e10;  // pair updates per run
  const double per_point = work / (double)n_act;                      // pair updates per step
  const int64_t Pt = std::max<int64_t>(std::min<int64_t>(n_act, 2432),
                                       std::min<int64_t>(n_act, (int64_t)(kTuneWork / std::max(per_point * tune_steps, 1.0))));
  {
    std::vector<int32_t> full((size_t)n_act), samp((size_t)Pt);
    ce = cudaMemcpyAsync(full.data(), c->scratch.active_list, sizeof(int32_t) * (size_t)n_act,
                         cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    for (int64_t q = 0; q < Pt && ce == cudaSuccess; ++q) samp[(size_t)q] = full[(size_t)(q * n_act / Pt)];
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(sample_list, samp.data(), sizeof(int32_t) * (size_t)Pt, cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(c, ce, who);
    }
  }
  Scratch ts = c->scratch;  // the sample's list; the queue counters are reset before every run
  ts.active_list = sample_list;
  const int32_t cnt[4] = {(int32_t)Pt, 0, (int32_t)Pt, 0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // small CTAs suit points with few species (one or two warp tasks per step): more of them
  // fit on an SM
  const int cands[5] = {32, 64, 128, 256, 512};
  float best = 1e30f;
  int best_b = c->block_dim;
  for (int b : cands) {
    CoalLaunch plan;
    if (coal_plan(c->t, c->precision, b, c->n_sms, &plan) != cudaSuccess) continue;
    float ms_tot = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
      cudaMemcpyAsync(c->scratch.counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice, c->stream);
      cudaEventRecord(e0, c->stream);
      launch_coal(c->t, c->precision, p, ts, dt, tune_steps, plan, c->stream);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep) ms_tot += ms;
    }
    if (ms_tot < best) {
      best = ms_tot;
      best_b = b;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t le = cudaGetLastError();
  cudaFree(tmp);
  if (le != cudaSuccess) return cuda_fail(c, le, who);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_b;
  }
  c->block_dim = best_b;
  c->plan_valid = false;
  return ensure_plan(c);
}

}  // namespace

extern "C" {

fsbm_status fsbm_coal_autotune(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points) {
  NvtxRange nvtx_("fsbm_coal_autotune");
  if (!c) return FSBM_E_ARG;
  return autotune_at(c, s, n_points, 5.0, 3, "fsbm_coal_autotune");
}

fsbm_status fsbm_coal_autotune_steps(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points, double dt,
                                     int32_t n_steps) {
  NvtxRange nvtx_("fsbm_coal_autotune_steps");
  if (!c) return FSBM_E_ARG;
  if (n_steps < 1) return fail(c, FSBM_E_ARG, "fsbm_coal_autotune_steps: n_steps must be >= 1");
  return autotune_at(c, s, n_points, dt, n_steps, "fsbm_coal_autotune_steps");
}

fsbm_status fsbm_coal_set_graph(fsbm_coal_ctx* c, int32_t enable) {
  if (!c) return FSBM_E_ARG;
  c->graph_enabled = enable != 0;
  if (!c->graph_enabled && c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return FSBM_OK;
}

fsbm_status fsbm_coal_set_block(fsbm_coal_ctx* c, int32_t block_dim) {
  if (!c) return FSBM_E_ARG;
  if (block_dim == 0) block_dim = 256;
  if (block_dim != 32 && block_dim != 64 && block_dim != 128 && block_dim != 256 && block_dim != 512)
    return fail(c, FSBM_E_ARG, "fsbm_coal_set_block: block_dim must be 32, 64, 128, 256 or 512");
  c->block_dim = block_dim;
  c->plan_valid = false;
  return ensure_plan(c);
}

fsbm_status fsbm_coal_set_gain_split(fsbm_coal_ctx* c, int32_t lanes) {
  if (!c) return FSBM_E_ARG;
  if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
    return fail(c, FSBM_E_ARG, "fsbm_coal_set_gain_split: lanes must be 0, 1, 2, 4 or 8");
  c->t.gain_split = lanes;
  if (c->gexec) {  // a captured graph holds the old tables by value
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return FSBM_OK;
}

fsbm_status fsbm_coal_set_timing(fsbm_coal_ctx* c, int32_t enable) {
  if (!c) return FSBM_E_ARG;
  c->timing = enable != 0;
  return FSBM_OK;
}

fsbm_status fsbm_coal_get_stats(fsbm_coal_ctx* c, fsbm_coal_stats* out) {
  if (!c || !out) return FSBM_E_ARG;
  std::memset(out, 0, sizeof(*out));
  CU(c, cudaStreamSynchronize(c->stream));
  for (auto* lst : {&c->ev_coal, &c->ev_step}) {
    double tot = 0.0;
    for (auto& ev : *lst) {
      float ms = 0.f;
      CU(c, cudaEventElapsedTime(&ms, ev.first, ev.second));
      tot += ms;
      c->ev_pool.push_back(ev.first);
      c->ev_pool.push_back(ev.second);
    }
    if (lst == &c->ev_coal) {
      out->coal_ms = tot;
      out->coal_launches = (int64_t)lst->size();
    } else {
      out->step_ms = tot;
      out->steps_timed = (int64_t)lst->size();
    }
    lst->clear();
  }
  int32_t cnt[4] = {0, 0, 0, 0};
  if (c->scratch.counters) CU(c, cudaMemcpy(cnt, c->scratch.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  out->n_points = c->last_n;
  out->n_active = cnt[0];
  out->shard_begin = cnt[3];
  out->shard_end = cnt[2];
  out->block_dim = c->plan.block_dim;
  out->grid_dim = c->plan.grid_dim;
  out->graph_replayed = c->last_replayed ? 1 : 0;
  out->tune_cache_hit = c->tune_cache_hit;
  return FSBM_OK;
}

fsbm_status fsbm_coal_get_active_list(fsbm_coal_ctx* c, int32_t* out, int64_t cap, int64_t* n_out) {
  if (!c || !n_out || cap < 0 || (cap > 0 && !out)) return FSBM_E_ARG;
  *n_out = 0;
  CU(c, cudaStreamSynchronize(c->stream));
  if (!c->scratch.counters) return FSBM_OK;
  int32_t cnt = 0;
  CU(c, cudaMemcpy(&cnt, c->scratch.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  *n_out = cnt;
  const int64_t m = std::min<int64_t>(cap, cnt);
  if (m > 0) CU(c, cudaMemcpy(out, c->scratch.active_list, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
  return FSBM_OK;
}

fsbm_status fsbm_coal_destroy(fsbm_coal_ctx* c) {
  if (!c) return FSBM_OK;
  cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->tables.reset();  // freed here unless a replica still holds them
  if (c->scratch.block_counts) cudaFree(c->scratch.block_counts);
  if (c->scratch.active_list) cudaFree(c->scratch.active_list);
  if (c->scratch.counters) cudaFree(c->scratch.counters);
  if (c->h_spectra) cudaFree(c->h_spectra);
  if (c->h_meta) cudaFree(c->h_meta);
  if (c->wrf_spec) cudaFree(c->wrf_spec);
  if (c->wrf_meta) cudaFree(c->wrf_meta);
  for (auto& ev : c->ev_coal) c->ev_pool.insert(c->ev_pool.end(), {ev.first, ev.second});
  for (auto& ev : c->ev_step) c->ev_pool.insert(c->ev_pool.end(), {ev.first, ev.second});
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return FSBM_OK;
}

fsbm_status fsbm_coal_math_check(fsbm_coal_ctx* c, double* out5) {
  if (!c || !out5) return FSBM_E_ARG;
  double* d = nullptr;
  CU(c, cudaMalloc(&d, 5 * sizeof(double)));
  cudaError_t e = launch_math_check(c->t, d, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out5, d, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(c, e, "fsbm_coal_math_check");
  return FSBM_OK;
}

fsbm_status fsbm_coal_check_record(fsbm_coal_ctx* c, uint32_t* out4) {
  if (!c || !out4) return FSBM_E_ARG;
#ifdef FSBM_CHECKED
  CU(c, cudaStreamSynchronize(c->stream));
  CU(c, cudaMemcpy(out4, c->t.chk, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  CU(c, cudaMemset(c->t.chk, 0, 4 * sizeof(uint32_t)));
  return FSBM_OK;
#else
  out4[0] = out4[1] = out4[2] = out4[3] = 0;
  return fail(c, FSBM_E_UNSUPPORTED, "fsbm_coal_check_record: this library is built without bounds checks "
                                     "(libfsbm_coal_checked.so has them)");
#endif
}

const char* fsbm_coal_last_error(const fsbm_coal_ctx* c) { return c ? c->err.c_str() : kNullCtxMsg; }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// fsbm_coal_step_noalloc: fsbm_coal_step for callers that must not allocate device memory.
//
// fsbm_coal_step sizes its scratch (the compaction pass's class counts, the list of active
// points and two counters) with cudaMalloc the first time it sees a batch that large. Some
// callers cannot let a library do that: a host model that reserves all device memory up
// front in its own pool (several model processes sharing one GPU leave no headroom for a
// library allocation), or one that cannot accept the device-wide synchronisation that
// cudaMalloc and cudaFree imply in the middle of its time loop. This entry point runs the
// same compaction pass and collision kernel with its scratch in a fixed array compiled into
// the library, and calls no allocating routine.
//
// The array is sized for kNoAllocMaxPoints points (about 1.1 MB) and exists on every GPU that
// loads the library until the process exits. The first call on a device looks up the array's
// device address (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture. All calls share the one array: two calls whose work overlaps on
// the GPU (two streams or two host threads) race on it and must be ordered by the caller.
// Every call rewrites all of the array it uses (the class counts, the list, and both
// counters, which the scan kernel resets), so nothing left by a previous call is read.
namespace {
constexpr int64_t kNoAllocMaxPoints = 262144;
constexpr int64_t kNoAllocMaxBlocks = (kNoAllocMaxPoints + kCompactThreads - 1) / kCompactThreads;
constexpr int64_t kNoAllocWords = (int64_t)kNumBuckets * kNoAllocMaxBlocks + kNoAllocMaxPoints + 4;
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int32_t* g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

extern "C" fsbm_status fsbm_coal_step_noalloc(fsbm_coal_ctx* c, const fsbm_coal_state* s, int64_t n_points,
                                              double dt, int32_t n_steps) {
  NvtxRange nvtx_("fsbm_coal_step_noalloc");
  if (!c) return FSBM_E_ARG;
  fsbm_status st = check_state(c, s, n_points, dt, n_steps, "fsbm_coal_step_noalloc");
  if (st != FSBM_OK) return st;
  if (n_points > kNoAllocMaxPoints)
    return fail(c, FSBM_E_ARG,
                "fsbm_coal_step_noalloc: n_points exceeds the fixed scratch capacity of 262144 points "
                "(use fsbm_coal_step, or split the batch)");
  int dev = -1;
  CU(c, cudaGetDevice(&dev));
  if (dev != c->device)
    return fail(c, FSBM_E_ARG, "fsbm_coal_step_noalloc: the context's device must be the current device");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(c, FSBM_E_UNSUPPORTED, "fsbm_coal_step_noalloc: device ordinal");
  int32_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(c, e, "fsbm_coal_step_noalloc: cudaGetSymbolAddress");
      g_noalloc_addr[dev] = static_cast<int32_t*>(p);
    }
    base = g_noalloc_addr[dev];
  }
  st = ensure_plan(c);  // launch shape only (function attributes, occupancy): no allocation
  if (st != FSBM_OK) return st;
  Scratch sc{};
  sc.n_blocks = (n_points + kCompactThreads - 1) / kCompactThreads;
  sc.block_counts = base;
  sc.active_list = base + (int64_t)kNumBuckets * kNoAllocMaxBlocks;
  sc.counters = sc.active_list + kNoAllocMaxPoints;
  const PointsDev p = to_dev(s, n_points);
  CU(c, launch_compact(c->t, p, n_points, sc, c->stream));
  CU(c, launch_coal(c->t, c->precision, p, sc, dt, n_steps, c->plan, c->stream));
  return FSBM_OK;
}
