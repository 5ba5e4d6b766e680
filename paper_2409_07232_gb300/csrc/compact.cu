// compact.cu -- the compaction pass: which points collide this call, and in what order.
//
// WRF calls coal_bott_new only for grid points that pass two temperature tests inside the
// grid loop (Listing 1); the paper's loop fission records that branch outcome in a
// predicate array and runs the collision loop over the predicate (Sec. VI-B, Listing 6),
// and notes that cloud-free points make the per-point work uneven (Sec. VIII). Here the
// predicate is evaluated for every point, the passing points are packed into a list, and
// the list is ordered costliest class first (longest-processing-time order for the
// persistent collision kernel): a stable counting sort over (grid, stored-species count)
// classes whose rank the host derived from the pair count n(n+1)/2 * ns + ns(ns-1)/2 * n^2.
//
// Three launches, no host synchronisation, no atomics (the order is deterministic):
//   classify  -- per point: status for skipped points, class counts per CTA;
//   scan      -- one CTA: exclusive scan of the [class][CTA] counts, the active count,
//                and the persistent queue's head and end reset to the whole list;
//   scatter   -- per point: its slot = class base + CTA base + rank within the CTA.
// A sharded call (several GPUs splitting one batch) adds one single-thread launch after the
// scan that narrows the queue to its shard of the ordered list (shard_bound).
#include "fsbm_internal.cuh"

namespace fsbm {
namespace {

constexpr int kWarps = kCompactThreads / 32;

// Class rank of point p, or -1 with *st set to the status of a skipped point.
__device__ __forceinline__ int classify_point(const Tables& t, const PointsDev& pd, int64_t p, int* st) {
  *st = 0;
  if ((pd.cloudy && pd.cloudy[p] == 0) ||
      (pd.temperature && !((double)pd.temperature[p] > t.t_min))) {
    *st = 4;
    return -1;
  }
  const int g = pd.grid_id[p];
  const unsigned mask = pd.species_mask[p];
  if (g >= t.G || (mask >> t.S) != 0u) {
    *st = 2;
    return -1;
  }
  if (t.levels && pd.pressure && !isfinite(pd.pressure[p])) {  // the kernels need a pressure
    *st = 2;
    return -1;
  }
  const int ns = __popc(mask);
  const int64_t len = pd.offset[p + 1] - pd.offset[p];
  if (len != (int64_t)ns * t.g[g].n) {
    *st = 2;
    return -1;
  }
  if (ns == 0) {  // nothing stored: no mass
    *st = 4;
    return -1;
  }
  return t.bucket_rank[g * (kMaxSpecies + 1) + ns];
}

__global__ void __launch_bounds__(kCompactThreads) k_classify(Tables t, PointsDev pd, int64_t n_points,
                                                              int32_t* block_counts, int64_t n_blocks) {
  __shared__ int wc[kNumBuckets][kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
  int r = -1;
  if (p < n_points) {
    int st;
    r = classify_point(t, pd, p, &st);
    if (r < 0) {
      pd.status[p] = st;
      pd.mass_budget[p] = 0.0;
      pd.mass_error[p] = 0.0;
    }
  }
  const int nb = t.G * t.S;
  for (int b = 0; b < nb; ++b) {
    const unsigned m = __ballot_sync(0xffffffffu, r == b);
    if (lane == 0) wc[b][warp] = __popc(m);
  }
  __syncthreads();
  if (threadIdx.x < nb && FSBM_OK(t.chk, (int64_t)threadIdx.x * n_blocks + blockIdx.x, (int64_t)kNumBuckets * n_blocks)) {
    int s = 0;
    for (int w = 0; w < kWarps; ++w) s += wc[threadIdx.x][w];
    block_counts[(int64_t)threadIdx.x * n_blocks + blockIdx.x] = s;
  }
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan(int32_t* counts, int64_t total, int32_t* counters) {
  __shared__ int64_t part[kScanThreads];
  const int tid = threadIdx.x;
  const int64_t chunk = (total + kScanThreads - 1) / kScanThreads;
  const int64_t b0 = tid * chunk;
  const int64_t b1 = b0 + chunk < total ? b0 + chunk : total;
  int64_t s = 0;
  for (int64_t e = b0; e < b1; ++e) s += counts[e];
  part[tid] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread sums
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const int64_t v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int64_t run = part[tid] - s;  // exclusive prefix of this thread's chunk
  for (int64_t e = b0; e < b1; ++e) {
    const int32_t c = counts[e];
    counts[e] = (int32_t)run;
    run += c;
  }
  if (tid == kScanThreads - 1) {
    counters[0] = (int32_t)part[kScanThreads - 1];
    counters[1] = 0;
    counters[2] = (int32_t)part[kScanThreads - 1];
    counters[3] = 0;
  }
}

// Shard `shard` of n_shards: its bounds in the ordered list from the class sizes (the scanned
// counts hold each class's first position in their first block's entry) and the class costs.
// The collision kernels then take points from [counters[1], counters[2]).
__global__ void k_shard(Tables t, const int32_t* counts, int64_t n_blocks, int32_t* counters, int shard,
                        int n_shards) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nb = t.G * t.S;
  int64_t cnt[kNumBuckets], cost[kNumBuckets];
  const int64_t n_active = counters[0];
  for (int c = 0; c < nb; ++c) {
    const int64_t a = counts[(int64_t)c * n_blocks];
    const int64_t b = c + 1 < nb ? counts[(int64_t)(c + 1) * n_blocks] : n_active;
    cnt[c] = b - a;
    cost[c] = t.rank_cost[c];
  }
  const int64_t lo = shard_bound(cnt, cost, nb, n_shards, shard);
  const int64_t hi = shard_bound(cnt, cost, nb, n_shards, shard + 1);
  counters[1] = (int32_t)lo;
  counters[2] = (int32_t)hi;
  counters[3] = (int32_t)lo;
}

__global__ void __launch_bounds__(kCompactThreads) k_scatter(Tables t, PointsDev pd, int64_t n_points,
                                                             const int32_t* offsets, int64_t n_blocks,
                                                             int32_t* list) {
  __shared__ int wc[kNumBuckets][kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
  int r = -1;
  if (p < n_points) {
    int st;
    r = classify_point(t, pd, p, &st);
  }
  const int nb = t.G * t.S;
  for (int b = 0; b < nb; ++b) {
    const unsigned m = __ballot_sync(0xffffffffu, r == b);
    if (lane == 0) wc[b][warp] = __popc(m);
  }
  __syncthreads();
  if (r >= 0) {
    const unsigned same = __match_any_sync(__activemask(), r);
    int rank = __popc(same & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += wc[r][w];
    if (FSBM_OK(t.chk, offsets[(int64_t)r * n_blocks + blockIdx.x] + rank, n_points))
      list[offsets[(int64_t)r * n_blocks + blockIdx.x] + rank] = (int32_t)p;
  }
}

}  // namespace

cudaError_t launch_compact(const Tables& t, const PointsDev& p, int64_t n_points, const Scratch& s,
                           cudaStream_t stream, int shard, int n_shards) {
  const int64_t nblk = (n_points + kCompactThreads - 1) / kCompactThreads;
  if (nblk != s.n_blocks) return cudaErrorInvalidValue;
  if (nblk > 0) {
    k_classify<<<(unsigned)nblk, kCompactThreads, 0, stream>>>(t, p, n_points, s.block_counts, nblk);
  }
  k_scan<<<1, kScanThreads, 0, stream>>>(s.block_counts, (int64_t)t.G * t.S * nblk, s.counters);
  if (nblk > 0 && n_shards > 1) k_shard<<<1, 32, 0, stream>>>(t, s.block_counts, nblk, s.counters, shard, n_shards);
  if (nblk > 0) {
    k_scatter<<<(unsigned)nblk, kCompactThreads, 0, stream>>>(t, p, n_points, s.block_counts, nblk,
                                                            s.active_list);
  }
  return cudaGetLastError();
}

}  // namespace fsbm
