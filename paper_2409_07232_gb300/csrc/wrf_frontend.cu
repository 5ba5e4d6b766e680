// wrf_frontend.cu -- the collision step on fields in WRF's memory layout.
//
// WRF keeps a patch's fields over memory ranges (ims:ime, kms:kme, jms:jme), i fastest, and a
// thread works on a tile inside them (Sec. I); FSBM keeps one such array per species with the
// bin as the last index. The collision step runs at the tile points that pass the loop's tests
// (Sec. III, Listing 1) and the predicate kept from the loop fission (Sec. VI-B, Listing 6).
// These kernels move the tile into the packed point layout the collision kernels read (one
// fixed slot of ns x n values per tile point, so no prefix sum is needed; only the slots of
// points that will be stepped are filled) and write the stepped points back.
#include "fsbm_internal.cuh"

namespace fsbm {
namespace {

// element index over the memory ranges (one bin plane) of tile point q (i fastest, then k, j)
__device__ __forceinline__ int64_t mem_index(const WrfDev& w, int64_t q) {
  const int64_t tik = (int64_t)w.ti * w.tk;
  const int j = w.jts + (int)(q / tik);
  const int64_t r = q - (int64_t)(j - w.jts) * tik;
  const int k = w.kts + (int)(r / w.ti);
  const int i = w.its + (int)(r - (int64_t)(k - w.kts) * w.ti);
  return ((int64_t)(j - w.jms) * w.km + (k - w.kms)) * w.im + (i - w.ims);
}

// per tile point: the packed point's metadata (offset, grid, species, cloud flag, T, p)
__global__ void k_wrf_meta(WrfDev w, PointsDev pk, int64_t n_tile) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t slot = (int64_t)w.ns * w.n;
  if (q == 0) const_cast<int64_t*>(pk.offset)[n_tile] = n_tile * slot;
  if (q >= n_tile) return;
  const int64_t m = mem_index(w, q);
  if (FSBM_CHECKED_BUILD && !FSBM_OK(w.chk, m, (int64_t)w.im * w.km * w.jm)) return;
  const_cast<int64_t*>(pk.offset)[q] = q * slot;
  const_cast<uint8_t*>(pk.grid_id)[q] = (uint8_t)w.grid;
  const_cast<uint8_t*>(pk.species_mask)[q] = (uint8_t)w.mask;
  const_cast<uint8_t*>(pk.cloudy)[q] = w.predicate ? (w.predicate[m] != 0) : 1;
  if (pk.temperature) const_cast<float*>(pk.temperature)[q] = w.temperature[m];
  if (pk.pressure) const_cast<float*>(pk.pressure)[q] = w.pressure[m];
}

// spectra of the points the step will run on: blockIdx.y = species slot x bin
template <typename T>
__global__ void k_wrf_pack(WrfDev w, PointsDev pk, int64_t n_tile, double t_min) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_tile) return;
  if (!pk.cloudy[q] || (pk.temperature && !((double)pk.temperature[q] > t_min))) return;
  const int e = blockIdx.y, s = e / w.n, b = e - s * w.n;
  const int64_t plane = (int64_t)w.im * w.km * w.jm;
  const T* src = static_cast<const T*>(w.ff[s]);
  if (FSBM_CHECKED_BUILD && !(FSBM_OK(w.chk, mem_index(w, q), plane) && FSBM_OK(w.chk, s, w.ns))) return;
  static_cast<T*>(pk.spectra)[q * ((int64_t)w.ns * w.n) + e] = src[(int64_t)b * plane + mem_index(w, q)];
}

// stepped points back into the fields (status 0 or 1: the step ran there), outputs too
template <typename T>
__global__ void k_wrf_unpack(WrfDev w, PointsDev pk, int64_t n_tile) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_tile) return;
  const int st = pk.status[q];
  const int64_t m = mem_index(w, q);
  const int e = blockIdx.y;
  if (FSBM_CHECKED_BUILD && !FSBM_OK(w.chk, m, (int64_t)w.im * w.km * w.jm)) return;
  if (e == 0) {
    if (w.status) w.status[m] = st;
    if (w.mass_budget) w.mass_budget[m] = pk.mass_budget[q];
    if (w.mass_error) w.mass_error[m] = pk.mass_error[q];
  }
  if (st & ~1) return;  // skipped (bad input) or inactive: left as it was
  const int s = e / w.n, b = e - s * w.n;
  const int64_t plane = (int64_t)w.im * w.km * w.jm;
  T* dst = static_cast<T*>(const_cast<void*>(w.ff[s]));
  dst[(int64_t)b * plane + m] = static_cast<const T*>(pk.spectra)[q * ((int64_t)w.ns * w.n) + e];
}

constexpr int kWrfThreads = 256;

}  // namespace

cudaError_t launch_wrf_pack(const WrfDev& w, int precision, const PointsDev& pk, int64_t n_tile, double t_min,
                            cudaStream_t stream) {
  const unsigned nb = (unsigned)((n_tile + kWrfThreads - 1) / kWrfThreads);
  k_wrf_meta<<<nb, kWrfThreads, 0, stream>>>(w, pk, n_tile);
  const dim3 grid(nb, (unsigned)(w.ns * w.n));
  if (precision == 0)
    k_wrf_pack<double><<<grid, kWrfThreads, 0, stream>>>(w, pk, n_tile, t_min);
  else
    k_wrf_pack<float><<<grid, kWrfThreads, 0, stream>>>(w, pk, n_tile, t_min);
  return cudaGetLastError();
}

cudaError_t launch_wrf_unpack(const WrfDev& w, int precision, const PointsDev& pk, int64_t n_tile,
                              cudaStream_t stream) {
  const unsigned nb = (unsigned)((n_tile + kWrfThreads - 1) / kWrfThreads);
  const dim3 grid(nb, (unsigned)(w.ns * w.n));
  if (precision == 0)
    k_wrf_unpack<double><<<grid, kWrfThreads, 0, stream>>>(w, pk, n_tile);
  else
    k_wrf_unpack<float><<<grid, kWrfThreads, 0, stream>>>(w, pk, n_tile);
  return cudaGetLastError();
}

}  // namespace fsbm
