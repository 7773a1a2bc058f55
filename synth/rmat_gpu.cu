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

}  // namespace

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
