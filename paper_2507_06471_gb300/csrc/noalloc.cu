// cd_modularity_noalloc: modularity of a partition computed without any
// device allocation, for callers that cannot call cudaMalloc (for example a
// host process whose device memory is entirely owned and budgeted by another
// allocator, where an extra driver allocation may fail or is not permitted).
//
// The per-community volume accumulators and the few control words live in one
// file-scope static __device__ array, g_noalloc_scratch, sized for at most
// kNoallocMaxN vertices: 16 MiB that every GPU which loads the library keeps
// until the process exits. Host code cannot use the array's name as a device
// address; on the first call on each device (with that device current) the
// entry point looks the address up once with cudaGetSymbolAddress and keeps
// it, and loads the entry point's kernels. That first call should therefore
// come before any stream capture on the device. The kept address belongs to
// the device's primary context: after cudaDeviceReset the library must not be
// used again in the process.
//
// All calls share the one array and it keeps the previous call's contents, so
// each call first clears the part it uses. Calls whose work overlaps on the
// GPU (different streams, or different host threads, without ordering between
// them) race on the array and must not be issued.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kNoallocMaxN = 1 << 21;  // vertices (and community ids) at most
constexpr int kCtlWords = 8;               // S low, S high, I, vol(V), status
constexpr int NT = 256;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocMaxN + kCtlWords];

constexpr int kMaxDevices = 64;
unsigned long long* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t load_kernels();

int scratch_on_current_device(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cd::set_cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices) return CD_EINVAL;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cd::set_cuda_error(e);
    // With lazy module loading a kernel's code is loaded, which can take
    // device memory, at its first launch; load all of this entry point's
    // kernels now so that no later call (weighted or not) loads anything.
    if ((e = load_kernels()) != cudaSuccess) return cd::set_cuda_error(e);
    g_scratch_dev[dev] = (unsigned long long*)p;
  }
  *out = g_scratch_dev[dev];
  return CD_OK;
}

__device__ __forceinline__ void na_fail(unsigned long long* ctl, int code) {
  atomicCAS(&ctl[4], 0ull, (unsigned long long)(unsigned)(-code));
}

// Warp per vertex: deg_w(v) (a loop counted twice) into the volume of v's
// community, the weight of arcs inside communities (a loop arc counts 2L) and
// vol(V). Every index is checked before use; a bad one sets the status word.
template <bool UNIT>
__global__ void __launch_bounds__(NT) k_noalloc_pass(const int64_t* __restrict__ off,
                                                     const int32_t* __restrict__ cols,
                                                     const int32_t* __restrict__ w,
                                                     const int32_t* __restrict__ labels, int64_t n,
                                                     int64_t nnz, unsigned long long* scratch) {
  unsigned long long* volc = scratch;
  unsigned long long* ctl = scratch + kNoallocMaxN;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  unsigned long long my_in = 0, my_vol = 0;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t a = labels[v];
    const int64_t beg = off[v], end = off[v + 1];
    if (a < 0 || a >= n) {
      if (lane == 0) na_fail(ctl, CD_EINVAL);
      continue;
    }
    if (beg < 0 || end < beg || end > nnz) {
      if (lane == 0) na_fail(ctl, CD_ENOTSYM);
      continue;
    }
    long long s = 0, in = 0;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t u = cols[e];
      const long long x = UNIT ? 1 : (long long)w[e];
      if (u < 0 || u >= n) {
        na_fail(ctl, CD_EBOUNDS);
        continue;
      }
      if (x < 1) na_fail(ctl, CD_EINVAL);
      s += u == v ? 2 * x : x;
      if (labels[u] == a) in += u == v ? 2 * x : x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(cd::FULL, s, o);
      in += __shfl_xor_sync(cd::FULL, in, o);
    }
    if (lane == 0) {
      atomicAdd(&volc[a], (unsigned long long)s);
      my_in += (unsigned long long)in;
      my_vol += (unsigned long long)s;
    }
  }
  if (lane == 0) {
    if (my_in) atomicAdd(&ctl[2], my_in);
    if (my_vol) atomicAdd(&ctl[3], my_vol);
  }
}

// Sum of squared community volumes, exact in 128 bits (ctl[0] low, ctl[1] high).
__global__ void __launch_bounds__(NT) k_noalloc_square(int64_t n, unsigned long long* scratch) {
  __shared__ unsigned __int128 part[NT];
  const unsigned long long* volc = scratch;
  unsigned long long* ctl = scratch + kNoallocMaxN;
  unsigned __int128 s = 0;
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t c = (int64_t)blockIdx.x * NT + threadIdx.x; c < n; c += stride)
    s += (unsigned __int128)volc[c] * volc[c];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && part[0]) {
    const unsigned long long lo = (unsigned long long)part[0], hi = (unsigned long long)(part[0] >> 64);
    const unsigned long long old = atomicAdd(&ctl[0], lo);
    const unsigned long long carry = old + lo < old ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&ctl[1], hi + carry);
  }
}

cudaError_t load_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k_noalloc_pass<true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_noalloc_pass<false>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_noalloc_square);
  return e;
}

}  // namespace

extern "C" int cd_modularity_noalloc(const int64_t* off, const int32_t* cols, const int32_t* w,
                                     const int32_t* labels, int64_t n, int64_t nnz, void* stream,
                                     double* q_out) {
  if (!q_out || n < 0 || nnz < 0 || (n > 0 && (!off || !labels)) || (nnz > 0 && !cols))
    return CD_EINVAL;
  if (n > kNoallocMaxN) return CD_EINVAL;  // larger than the static scratch
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  unsigned long long* ctl = scratch + kNoallocMaxN;
  CD_CHECK(cudaMemsetAsync(scratch, 0, (size_t)n * sizeof(unsigned long long), s));
  CD_CHECK(cudaMemsetAsync(ctl, 0, kCtlWords * sizeof(unsigned long long), s));
  if (n > 0) {
    int64_t blocks = (n * 32 + NT - 1) / NT;
    const unsigned grid = (unsigned)(blocks < 152 * 16 ? blocks : 152 * 16);
    if (w)
      CD_LAUNCH(k_noalloc_pass<false><<<grid, NT, 0, s>>>(off, cols, w, labels, n, nnz, scratch));
    else
      CD_LAUNCH(k_noalloc_pass<true><<<grid, NT, 0, s>>>(off, cols, w, labels, n, nnz, scratch));
    int64_t sb = (n + NT - 1) / NT;
    CD_LAUNCH(k_noalloc_square<<<(unsigned)(sb < 152 * 4 ? sb : 152 * 4), NT, 0, s>>>(n, scratch));
    CD_CHECK(cudaGetLastError());
  }
  unsigned long long h[kCtlWords] = {};
  CD_CHECK(cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
  CD_CHECK(cudaStreamSynchronize(s));
  if (h[4]) return -(int)h[4];
  const int64_t vol = (int64_t)h[3];
  if (vol == 0) {
    *q_out = 0.0;
    return CD_OK;
  }
  const unsigned __int128 S = ((unsigned __int128)h[1] << 64) | h[0];
  const cd::i128 num = (cd::i128)(int64_t)h[2] * vol - (cd::i128)S;
  const cd::i128 den = (cd::i128)vol * vol;
  *q_out = (double)num / (double)den;
  return CD_OK;
}
