// Device-wide primitives: exclusive prefix sums and a stable LSD radix sort.
//
// Scan: reduce-then-scan over tiles of 4096 elements (per-tile sums, one CTA
// scans the tile sums, each tile rescans itself with its offset).
// Radix sort: 8-bit digits, per pass a per-tile digit histogram (digit-major
// layout), an exclusive scan of the histogram, and a stable scatter that ranks
// equal digits with __match_any_sync inside each warp and a per-digit prefix
// over the warps of the CTA.
#include "common.cuh"

namespace cd {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread across the CTA; returns the CTA total.
template <class T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T x, T* total) {
  __shared__ T warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = warp_inclusive_scan(x);
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T t = lane < NT / 32 ? warp_tot[lane] : T(0);
    T ti = warp_inclusive_scan(t);
    if (lane < NT / 32) warp_tot[lane] = ti - t;
    if (lane == NT / 32 - 1) *total = ti;
  }
  __syncthreads();
  T r = inc - x + warp_tot[wid];
  __syncthreads();
  return r;
}

struct InI64 {
  const int64_t* p;
  __device__ __forceinline__ int64_t operator()(int64_t i) const { return p[i]; }
};
struct InHead {  // 1 where a run of equal keys starts
  const uint64_t* k;
  __device__ __forceinline__ int64_t operator()(int64_t i) const {
    return (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
  }
};
struct InU8 {
  const uint8_t* p;
  __device__ __forceinline__ int32_t operator()(int64_t i) const { return (int32_t)p[i]; }
};

template <class T, class In>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(In in, int64_t n, T* sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  T s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j)
    if (base + j < n) s += in(base + j);
  __shared__ T tot;
  block_exclusive_scan<T, SCAN_THREADS>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(1024) k_scan_sums(T* sums, int64_t nb, int64_t* total) {
  __shared__ T tot;
  T run = 0;
  for (int64_t c = 0; c < nb; c += 1024) {
    int64_t i = c + threadIdx.x;
    T x = i < nb ? sums[i] : T(0);
    T ex = block_exclusive_scan<T, 1024>(x, &tot);
    if (i < nb) sums[i] = run + ex;
    run += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = (int64_t)run;
}

template <class T, class In>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(In in, int64_t n, const T* sums,
                                                            T* out) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    v[j] = base + j < n ? in(base + j) : T(0);
    s += v[j];
  }
  __shared__ T tot;
  T ex = block_exclusive_scan<T, SCAN_THREADS>(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    if (base + j < n) out[base + j] = ex;
    ex += v[j];
  }
}

template <class T, class In>
int scan_impl(In in, T* out, int64_t n, int64_t* total_dev, cudaStream_t s) {
  if (n <= 0) {
    if (total_dev) CD_CHECK(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
    return CD_OK;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  T* sums = nullptr;
  int rc = dev_alloc_t(&sums, nb, s);
  if (rc) return rc;
  CD_LAUNCH(k_scan_reduce<T, In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums));
  CD_LAUNCH(k_scan_sums<T><<<1, 1024, 0, s>>>(sums, nb, total_dev));
  CD_LAUNCH(k_scan_down<T, In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums, out));
  dev_free(sums, s);
  CD_CHECK(cudaGetLastError());
  return CD_OK;
}

// ---------------------------------------------------------------- radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                        int shift, int64_t ntiles,
                                                        int64_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int j = 0; j < RS_ITEMS; ++j) {
    int64_t i = base + (int64_t)j * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(
    const uint64_t* __restrict__ keys, const int64_t* __restrict__ vals, int64_t n, int shift,
    int64_t ntiles, const int64_t* __restrict__ offsets, uint64_t* __restrict__ keys_out,
    int64_t* __restrict__ vals_out) {
  __shared__ int64_t base_d[256];
  __shared__ uint32_t wcnt[RS_WARPS][256];
  __shared__ uint32_t total_d[256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  base_d[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  int64_t tile = (int64_t)blockIdx.x * RS_TILE;
  for (int j = 0; j < RS_ITEMS; ++j) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = tile + (int64_t)j * RS_THREADS + threadIdx.x;
    bool valid = i < n;
    uint64_t k = valid ? keys[i] : 0;
    int64_t v = valid ? vals[i] : 0;
    int d = valid ? (int)((k >> shift) & 0xFF) : 256 + lane;  // invalid lanes match nobody
    unsigned peers = __match_any_sync(FULL, d);
    unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) {
        uint32_t c = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = run;
        run += c;
      }
      total_d[threadIdx.x] = run;
    }
    __syncthreads();
    if (valid) {
      int64_t pos = base_d[d] + wcnt[wid][d] + rank;
      keys_out[pos] = k;
      vals_out[pos] = v;
    }
    __syncthreads();
    base_d[threadIdx.x] += total_d[threadIdx.x];
    __syncthreads();
  }
}

}  // namespace

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                       cudaStream_t s) {
  return scan_impl<int64_t>(InI64{in}, out, n, total_dev, s);
}

int exclusive_scan_u8_to_i32(const uint8_t* in, int32_t* out, int64_t n, int64_t* total_dev,
                             cudaStream_t s) {
  return scan_impl<int32_t>(InU8{in}, out, n, total_dev, s);
}

int exclusive_scan_head(const uint64_t* keys, int64_t* out, int64_t n, int64_t* total_dev,
                        cudaStream_t s) {
  return scan_impl<int64_t>(InHead{keys}, out, n, total_dev, s);
}

int radix_sort_pairs(uint64_t* keys, int64_t* vals, uint64_t* keys_tmp, int64_t* vals_tmp,
                     int64_t n, int bits, cudaStream_t s, uint64_t** keys_out,
                     int64_t** vals_out) {
  *keys_out = keys;
  *vals_out = vals;
  if (n <= 1 || bits <= 0) return CD_OK;
  int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  int64_t* counts = nullptr;
  int rc = dev_alloc_t(&counts, 256 * ntiles, s);
  if (rc) return rc;
  uint64_t *ka = keys, *kb = keys_tmp;
  int64_t *va = vals, *vb = vals_tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    CD_LAUNCH(k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, ntiles, counts));
    rc = exclusive_scan_i64(counts, counts, 256 * ntiles, nullptr, s);
    if (rc) break;
    CD_LAUNCH(k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, n, shift, ntiles, counts, kb, vb));
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  dev_free(counts, s);
  if (rc) return rc;
  CD_CHECK(cudaGetLastError());
  *keys_out = ka;
  *vals_out = va;
  return CD_OK;
}

}  // namespace cd
