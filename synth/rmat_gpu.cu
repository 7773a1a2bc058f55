// Device R-MAT edge generator for the synthetic inputs (not part of the
// community-detection path). Edge i descends `scale` levels of the R-MAT
// recursion; level l draws number (i * 64 + l) of the SplitMix64 stream with
// state `key` (Steele, Lea and Flood, OOPSLA 2014) and picks the quadrant from
// its top 32 bits. The host generator in synth/__init__.py implements the same
// definition, so both produce identical edges.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm64_draw(uint64_t key, uint64_t ctr) {
  return sm64_mix(key + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
}

__global__ void rmat_keys_kernel(uint64_t key, int scale, uint32_t tA, uint32_t tAB, uint32_t tABC,
                                 int64_t first, int64_t count, int64_t* __restrict__ out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
    uint64_t i = (uint64_t)(first + t);
    uint64_t src = 0, dst = 0;
    for (int l = 0; l < scale; ++l) {
      uint32_t x = (uint32_t)(sm64_draw(key, (i << 6) | (uint64_t)l) >> 32);
      uint64_t bs = x >= tAB;
      uint64_t bd = (x >= tA && x < tAB) || x >= tABC;
      src = (src << 1) | bs;
      dst = (dst << 1) | bd;
    }
    uint64_t lo = src < dst ? src : dst, hi = src < dst ? dst : src;
    out[t] = lo == hi ? -1 : (int64_t)((lo << 32) | hi);
  }
}

// Planted-partition pairs of many graphs: thread per row u of graph b; the
// pair {u, v} (u < v, ids local to b) is an edge iff draw number u * n_b + v
// of graph b's stream is below the threshold for "same block" (p_in) or
// "different blocks" (p_out); block(u) = min(u / (n_b / k_b), k_b - 1).
// Edges are appended as (b << 40 | u << 20 | v).
__global__ void sbm_rows_kernel(const int64_t* __restrict__ vstart, const int32_t* __restrict__ row_graph,
                                const int32_t* __restrict__ blocks, const uint64_t* __restrict__ keys,
                                uint64_t t_in, uint64_t t_out, int64_t rows, int64_t* __restrict__ out,
                                unsigned long long* __restrict__ out_n, int64_t cap) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    const int32_t b = row_graph[r];
    const int64_t n = vstart[b + 1] - vstart[b];
    const int64_t u = r - vstart[b];
    const int64_t k = blocks[b];
    int64_t bsz = n / k;
    if (bsz < 1) bsz = 1;
    const int64_t bu = u / bsz < k - 1 ? u / bsz : k - 1;
    for (int64_t v = u + 1; v < n; ++v) {
      const int64_t bv = v / bsz < k - 1 ? v / bsz : k - 1;
      const uint64_t x = sm64_draw(keys[b], (uint64_t)(u * n + v));
      if (x < (bu == bv ? t_in : t_out)) {
        const unsigned long long pos = atomicAdd(out_n, 1ull);
        if ((int64_t)pos < cap) out[pos] = ((int64_t)b << 40) | (u << 20) | v;
      }
    }
  }
}

// Edge-sampled planted partition (for sparse graphs too large for the
// pairwise definition): edge j takes draws 3j, 3j+1, 3j+2 of the stream. Its
// first endpoint u is uniform on [0, n); with block size s of u's block it
// stays inside that block with probability 100 (s-1) / (100 (s-1) + n - s)
// (p_out = p_in / 100) and then v is uniform in the block, else v is uniform
// over the other n - s vertices. Uniform picks are multiply-shift on the top
// 32 bits (spans stay below 2^32 for n <= 4e7). Loops give -1; keys are
// lo << 32 | hi.
__device__ __forceinline__ uint64_t pick32(uint64_t r, uint64_t span) { return ((r >> 32) * span) >> 32; }

__global__ void sbm_edges_kernel(uint64_t key, int64_t n, int64_t k, int64_t m, int64_t* __restrict__ out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t bsz = n / k;
  if (bsz < 1) bsz = 1;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const uint64_t c = 3ull * (uint64_t)j;
    const int64_t u = (int64_t)pick32(sm64_draw(key, c), (uint64_t)n);
    const int64_t bu = u / bsz < k - 1 ? u / bsz : k - 1;
    const int64_t b0 = bu * bsz;
    const int64_t s = bu == k - 1 ? n - b0 : bsz;
    const uint64_t in_w = 100ull * (uint64_t)(s - 1), out_w = (uint64_t)(n - s);
    int64_t v = u;
    if (in_w + out_w > 0) {
      if (pick32(sm64_draw(key, c + 1), in_w + out_w) < in_w) {
        v = b0 + (int64_t)pick32(sm64_draw(key, c + 2), (uint64_t)s);
      } else {
        const int64_t x = (int64_t)pick32(sm64_draw(key, c + 2), out_w);
        v = x < b0 ? x : x + s;
      }
    }
    const int64_t lo = u < v ? u : v, hi = u < v ? v : u;
    out[j] = lo == hi ? -1 : (lo << 32) | hi;
  }
}

}  // namespace

extern "C" int synth_sbm_edges(uint64_t key, int64_t n, int64_t k, int64_t m, void* out, void* stream) {
  if (n < 1 || n > 40000000 || k < 1 || m < 0 || (m > 0 && out == nullptr)) return -1;
  if (m == 0) return 0;
  int64_t blocks = (m + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  sbm_edges_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(key, n, k, m, (int64_t*)out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int synth_sbm_rows(const void* vstart, const void* row_graph, const void* blocks, const void* keys,
                              uint64_t t_in, uint64_t t_out, int64_t rows, void* out, void* out_n, int64_t cap,
                              void* stream) {
  if (rows <= 0) return 0;
  int64_t nb = (rows + 255) / 256;
  if (nb > 152 * 64) nb = 152 * 64;
  sbm_rows_kernel<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(
      (const int64_t*)vstart, (const int32_t*)row_graph, (const int32_t*)blocks, (const uint64_t*)keys, t_in,
      t_out, rows, (int64_t*)out, (unsigned long long*)out_n, cap);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int synth_rmat_keys(uint64_t key, int scale, uint32_t tA, uint32_t tAB, uint32_t tABC,
                               int64_t first, int64_t count, void* out, void* stream) {
  if (scale < 1 || scale > 31 || count < 0 || (count > 0 && out == nullptr)) return -1;
  if (count == 0) return 0;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  rmat_keys_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(key, scale, tA, tAB, tABC, first,
                                                                        count, (int64_t*)out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
