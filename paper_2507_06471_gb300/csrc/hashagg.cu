// Louvain aggregation by hashing (Algorithm 3, Aggregation): the coarse
// graph without a global sort of the arcs.
//
// 1. The n vertices are sorted by A = new(C[v]) (radix sort of n keys, not of
//    m arcs), which lists every community's members together.
// 2. An exclusive scan of the member degrees gives each community a contiguous
//    segment of the arc space; every arc u->x of a member u writes
//    (B = new(C[x]), w) into its community's segment (no atomics).
// 3. Each segment is combined by hashing B: one warp for a segment of at most
//    AG_WARP_MAX arcs, one CTA for at most AG_CTA_MAX, each with a
//    shared-memory table; a larger segment is cut into AG_CHUNK-arc chunks,
//    each combined in shared memory, whose distinct entries are then merged in
//    a global table sized for the segment. The distinct (B, sum w) of a
//    segment are written back at its start.
// 4. The segments are compacted into the coarse CSR (k rows, columns in no
//    particular order, int64 weights; (A, A) collects every arc inside A,
//    i.e. twice its internal weight, the internal convention for loops).
// The content of every row equals that of the sort-based aggregation; only the
// order of columns inside a row differs, and no later step depends on it.
#include <algorithm>

#include "common.cuh"

namespace cd {
namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int AG_WARP_MAX = 256;   // arcs of a segment combined by one warp (512-slot table)
constexpr int AG_CTA_MAX = 4096;   // by one CTA (8192-slot table)
constexpr int AG_CHUNK = 4096;     // arcs per chunk of a larger segment
constexpr int AG_WCAP = 2 * AG_WARP_MAX;
constexpr int AG_CCAP = 2 * AG_CTA_MAX;
constexpr int AG_SLICE = 1024;     // global-table slots per extraction item (tables are multiples)
constexpr int AG_CNT = 512;        // threads of the CTA-per-segment kernel
constexpr int32_t AG_EMPTY = -1;

unsigned gcap(int64_t blocks, int64_t cap = 152 * 16) {
  if (blocks < 1) blocks = 1;
  return (unsigned)(blocks < cap ? blocks : cap);
}

__device__ __forceinline__ unsigned lg_for(int64_t x) {  // smallest lg >= 1 with 2^lg >= x
  unsigned lg = 1;
  while (((int64_t)1 << lg) < x) ++lg;
  return lg;
}

// ------------------------------------------------------------------ steps 1-2

__global__ void k_ag_vkeys(const int32_t* __restrict__ labels, const int32_t* __restrict__ newid, int64_t n,
                           uint64_t* __restrict__ key, int64_t* __restrict__ val) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    key[v] = (uint64_t)newid[labels[v]];
    val[v] = v;
  }
}

__global__ void k_ag_mdeg(const int64_t* __restrict__ off, const int64_t* __restrict__ mem, int64_t n,
                          int64_t* __restrict__ md) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t v = mem[i];
    md[i] = off[v + 1] - off[v];
  }
}

// sstart[A] = arc-space start of community A (its first member's prefix).
__global__ void k_ag_heads(const uint64_t* __restrict__ skey, const int64_t* __restrict__ mpre, int64_t n,
                           int64_t* __restrict__ sstart) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (i == 0 || skey[i] != skey[i - 1]) sstart[skey[i]] = mpre[i];
}

// Warp per member: the member's arcs into its community's segment.
template <class W>
__global__ void __launch_bounds__(NT) k_ag_scatter(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                                   const void* w, const int32_t* __restrict__ labels,
                                                   const int32_t* __restrict__ newid, const int64_t* __restrict__ mem,
                                                   const int64_t* __restrict__ mpre, int64_t n,
                                                   int32_t* __restrict__ ab, unsigned long long* __restrict__ aw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int64_t v = mem[i], base = mpre[i];
    const int64_t beg = off[v], d = off[v + 1] - beg;
    for (int64_t j = lane; j < d; j += 32) {
      ab[base + j] = newid[labels[cols[beg + j]]];
      aw[base + j] = (unsigned long long)W::get(w, beg + j);
    }
  }
}

// ------------------------------------------------------------------ classes

// cnt: [0] warp segments, [1] CTA segments, [2] large segments, [3] chunks.
__global__ void k_ag_class_count(const int64_t* __restrict__ sstart, int64_t k, unsigned long long* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long c[4] = {0, 0, 0, 0};
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < k; a += stride) {
    const int64_t len = sstart[a + 1] - sstart[a];
    if (len <= AG_WARP_MAX) {
      ++c[0];
    } else if (len <= AG_CTA_MAX) {
      ++c[1];
    } else {
      ++c[2];
      c[3] += (unsigned long long)((len + AG_CHUNK - 1) / AG_CHUNK);
    }
  }
  for (int j = 0; j < 4; ++j)
    if (c[j]) atomicAdd(&cnt[j], c[j]);
}

__global__ void k_ag_class_fill(const int64_t* __restrict__ sstart, int64_t k, unsigned long long* cur,
                                int32_t* __restrict__ wl, int32_t* __restrict__ cl, int32_t* __restrict__ ll,
                                int32_t* __restrict__ ch_seg, int64_t* __restrict__ ch_off) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < k; a += stride) {
    const int64_t len = sstart[a + 1] - sstart[a];
    if (len <= AG_WARP_MAX) {
      wl[atomicAdd(&cur[0], 1ull)] = (int32_t)a;
    } else if (len <= AG_CTA_MAX) {
      cl[atomicAdd(&cur[1], 1ull)] = (int32_t)a;
    } else {
      ll[atomicAdd(&cur[2], 1ull)] = (int32_t)a;
      const int64_t nc = (len + AG_CHUNK - 1) / AG_CHUNK;
      const unsigned long long p = atomicAdd(&cur[3], (unsigned long long)nc);
      for (int64_t j = 0; j < nc; ++j) {
        ch_seg[p + j] = (int32_t)a;
        ch_off[p + j] = j * AG_CHUNK;
      }
    }
  }
}

// ------------------------------------------------------------------ shared-memory combining

// Open addressing in a 2^lg-slot table holding at most half that many keys,
// so a free slot is always found; a claimed slot joins the occupied list.
__device__ __forceinline__ void tab_insert(int32_t* keys, unsigned long long* vals, uint16_t* occ, int* occ_n,
                                           unsigned lg, int32_t key, unsigned long long w) {
  const unsigned mask = (1u << lg) - 1u;
  unsigned h = ((uint32_t)key * 2654435761u) >> (32 - lg);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int32_t prev = atomicCAS(&keys[h], AG_EMPTY, key);
    if (prev == AG_EMPTY || prev == key) {
      atomicAdd(&vals[h], w);
      if (prev == AG_EMPTY) occ[atomicAdd(occ_n, 1)] = (uint16_t)h;
      return;
    }
    h = (h + 1) & mask;
  }
}

// A warp inserts `len` entries starting at p: equal keys of one load are
// combined first (match), so a key repeated across the warp costs one atomic.
__device__ __forceinline__ void warp_insert(const int32_t* __restrict__ ab, const unsigned long long* __restrict__ aw,
                                            int64_t p, int64_t len, int32_t* keys, unsigned long long* vals,
                                            uint16_t* occ, int* occ_n, unsigned lg, unsigned long long* stage,
                                            int lane) {
  for (int64_t j = lane; j - lane < len; j += 32) {  // the whole warp iterates together
    const bool ok = j < len;
    const int32_t key = ok ? ab[p + j] : (int32_t)(0x80000000u | (unsigned)lane);
    const unsigned long long wt = ok ? aw[p + j] : 0ull;
    const unsigned peers = __match_any_sync(FULL, key);
    stage[lane] = wt;
    __syncwarp();
    if (ok && (__ffs(peers) - 1) == lane) {
      unsigned long long sum = 0;
      unsigned m = peers;
      while (m) {
        sum += stage[__ffs(m) - 1];
        m &= m - 1;
      }
      tab_insert(keys, vals, occ, occ_n, lg, key, sum);
    }
    __syncwarp();
  }
}

// Warp per small segment: combine, then write the distinct entries back at
// the segment start and record their number.
__global__ void __launch_bounds__(NT) k_ag_warp(const int64_t* __restrict__ sstart, const int32_t* __restrict__ wl,
                                                int64_t nw, int32_t* ab, unsigned long long* aw,
                                                int64_t* __restrict__ ucnt) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long* vals = (unsigned long long*)smem + (size_t)wid * AG_WCAP;
  int32_t* keys = (int32_t*)(smem + (size_t)NW * AG_WCAP * 8) + (size_t)wid * AG_WCAP;
  unsigned long long* stage = (unsigned long long*)(smem + (size_t)NW * AG_WCAP * 12) + (size_t)wid * 32;
  uint16_t* occ = (uint16_t*)(smem + (size_t)NW * AG_WCAP * 12 + (size_t)NW * 32 * 8) + (size_t)wid * AG_WCAP;
  __shared__ int occ_n[NW];
  for (int j = lane; j < AG_WCAP; j += 32) {
    keys[j] = AG_EMPTY;
    vals[j] = 0;
  }
  if (lane == 0) occ_n[wid] = 0;
  __syncwarp();
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t q = warp; q < nw; q += nwarps) {
    const int32_t a = wl[q];
    const int64_t p = sstart[a], len = sstart[a + 1] - p;
    const unsigned lg = lg_for(2 * len);
    warp_insert(ab, aw, p, len, keys, vals, occ, &occ_n[wid], lg, stage, lane);
    __syncwarp();
    const int nocc = occ_n[wid];
    for (int j = lane; j < nocc; j += 32) {
      const int slot = occ[j];
      ab[p + j] = keys[slot];
      aw[p + j] = vals[slot];
      keys[slot] = AG_EMPTY;
      vals[slot] = 0;
    }
    if (lane == 0) {
      ucnt[a] = nocc;
      occ_n[wid] = 0;
    }
    __syncwarp();
  }
}

// CTA per block of up to AG_CTA_MAX arcs: a whole medium segment, or one chunk
// of a large segment (then the chunk's distinct count goes to dch and to the
// segment's upper bound ub).
template <bool CHUNK>
__global__ void __launch_bounds__(AG_CNT) k_ag_cta(const int64_t* __restrict__ sstart, const int32_t* __restrict__ list,
                                               const int64_t* __restrict__ ch_off, int64_t nitems, int32_t* ab,
                                               unsigned long long* aw, int64_t* __restrict__ ucnt,
                                               int32_t* __restrict__ dch, unsigned long long* __restrict__ ub) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* vals = (unsigned long long*)smem;
  int32_t* keys = (int32_t*)(smem + (size_t)AG_CCAP * 8);
  unsigned long long* stage = (unsigned long long*)(smem + (size_t)AG_CCAP * 12) + (threadIdx.x >> 5) * 32;
  uint16_t* occ = (uint16_t*)(smem + (size_t)AG_CCAP * 12 + (size_t)(AG_CNT / 32) * 32 * 8);
  __shared__ int occ_n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < AG_CCAP; j += AG_CNT) {
    keys[j] = AG_EMPTY;
    vals[j] = 0;
  }
  if (threadIdx.x == 0) occ_n = 0;
  __syncthreads();
  for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int32_t a = list[it];
    int64_t p = sstart[a], len = sstart[a + 1] - p;
    if (CHUNK) {
      p += ch_off[it];
      len = len - ch_off[it] < AG_CHUNK ? len - ch_off[it] : AG_CHUNK;
    }
    const unsigned lg = lg_for(2 * len);
    // warps take interleaved 32-entry rows of the block
    for (int64_t j = (int64_t)wid * 32; j < len; j += AG_CNT) {
      const int64_t jj = j + lane;
      const bool ok = jj < len;
      const int32_t key = ok ? ab[p + jj] : (int32_t)(0x80000000u | (unsigned)lane);
      const unsigned long long wt = ok ? aw[p + jj] : 0ull;
      const unsigned peers = __match_any_sync(FULL, key);
      stage[lane] = wt;
      __syncwarp();
      if (ok && (__ffs(peers) - 1) == lane) {
        unsigned long long sum = 0;
        unsigned m = peers;
        while (m) {
          sum += stage[__ffs(m) - 1];
          m &= m - 1;
        }
        tab_insert(keys, vals, occ, &occ_n, lg, key, sum);
      }
      __syncwarp();
    }
    __syncthreads();  // every entry read and inserted before the block is overwritten
    const int nocc = occ_n;
    for (int j = threadIdx.x; j < nocc; j += AG_CNT) {
      const int slot = occ[j];
      ab[p + j] = keys[slot];
      aw[p + j] = vals[slot];
      keys[slot] = AG_EMPTY;
      vals[slot] = 0;
    }
    if (threadIdx.x == 0) {
      if (CHUNK) {
        dch[it] = nocc;
        atomicAdd(&ub[a], (unsigned long long)nocc);
      } else {
        ucnt[a] = nocc;
      }
      occ_n = 0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ large segments

// Global table of a large segment: 2^lg >= 2 x (its upper bound of distinct
// keys) slots, at least AG_SLICE, placed at toff[a]; its slices are owned by a.
__global__ void k_ag_tables_size(const int32_t* __restrict__ ll, int64_t nl, const unsigned long long* __restrict__ ub,
                                 int32_t* __restrict__ tlg, int64_t* __restrict__ toff, unsigned long long* total) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nl; q += stride) {
    const int32_t a = ll[q];
    unsigned lg = lg_for(2 * (int64_t)ub[a]);
    if (lg < 10) lg = 10;  // AG_SLICE
    tlg[a] = (int32_t)lg;
    toff[a] = (int64_t)atomicAdd(total, 1ull << lg);
  }
}

__global__ void k_ag_tables_own(const int32_t* __restrict__ ll, int64_t nl, const int32_t* __restrict__ tlg,
                                const int64_t* __restrict__ toff, int32_t* __restrict__ owner) {
  for (int64_t q = blockIdx.x; q < nl; q += gridDim.x) {
    const int32_t a = ll[q];
    const int64_t s0 = toff[a] / AG_SLICE, ns = ((int64_t)1 << tlg[a]) / AG_SLICE;
    for (int64_t j = threadIdx.x; j < ns; j += blockDim.x) owner[s0 + j] = a;
  }
}

// CTA per chunk: its distinct entries into the segment's global table.
__global__ void __launch_bounds__(NT) k_ag_merge(const int64_t* __restrict__ sstart, const int32_t* __restrict__ ch_seg,
                                                 const int64_t* __restrict__ ch_off, const int32_t* __restrict__ dch,
                                                 int64_t nch, const int32_t* __restrict__ ab,
                                                 const unsigned long long* __restrict__ aw,
                                                 const int32_t* __restrict__ tlg, const int64_t* __restrict__ toff,
                                                 int32_t* gk, unsigned long long* gv) {
  for (int64_t it = blockIdx.x; it < nch; it += gridDim.x) {
    const int32_t a = ch_seg[it];
    const int64_t p = sstart[a] + ch_off[it];
    const int d = dch[it];
    const unsigned lg = (unsigned)tlg[a];
    const uint64_t mask = ((uint64_t)1 << lg) - 1;
    int32_t* keys = gk + toff[a];
    unsigned long long* vals = gv + toff[a];
    for (int j = threadIdx.x; j < d; j += NT) {
      const int32_t key = ab[p + j];
      const unsigned long long w = aw[p + j];
      uint64_t h = ((uint64_t)(uint32_t)key * 0x9E3779B97F4A7C15ull) >> (64 - lg);
      for (uint64_t probe = 0; probe <= mask; ++probe) {
        const int32_t prev = atomicCAS(&keys[h], AG_EMPTY, key);
        if (prev == AG_EMPTY || prev == key) {
          atomicAdd(&vals[h], w);
          break;
        }
        h = (h + 1) & mask;
      }
    }
  }
}

// CTA per AG_SLICE slots of the global tables: the live entries go back into
// their segment (in any order).
__global__ void __launch_bounds__(NT) k_ag_extract(const int32_t* __restrict__ owner, int64_t nslices,
                                                   const int32_t* __restrict__ gk, const unsigned long long* __restrict__ gv,
                                                   const int64_t* __restrict__ sstart, int32_t* ab,
                                                   unsigned long long* aw, int64_t* ucnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t sl = blockIdx.x; sl < nslices; sl += gridDim.x) {
    const int32_t a = owner[sl];
    const int64_t p = sstart[a];
    for (int j0 = 0; j0 < AG_SLICE; j0 += NT) {  // whole warps per step (the ballot needs them)
      const int64_t slot = sl * AG_SLICE + j0 + threadIdx.x;
      const int32_t key = gk[slot];
      const bool live = key != AG_EMPTY;
      const unsigned bal = __ballot_sync(FULL, live);
      unsigned long long base = 0;
      if (lane == 0 && bal) base = (unsigned long long)atomicAdd((unsigned long long*)&ucnt[a], (unsigned long long)__popc(bal));
      base = __shfl_sync(FULL, base, 0);
      if (live) {
        const int64_t q = p + (int64_t)base + __popc(bal & ((1u << lane) - 1u));
        ab[q] = key;
        aw[q] = gv[slot];
      }
    }
  }
}

// Warp per community: its distinct entries into the coarse CSR.
__global__ void __launch_bounds__(NT) k_ag_compact(const int64_t* __restrict__ sstart, const int64_t* __restrict__ ucnt,
                                                   const int64_t* __restrict__ coff, int64_t k,
                                                   const int32_t* __restrict__ ab, const unsigned long long* __restrict__ aw,
                                                   int32_t* __restrict__ ccols, int64_t* __restrict__ cw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t a = warp; a < k; a += nwarps) {
    const int64_t p = sstart[a], d = ucnt[a], o = coff[a];
    for (int64_t j = lane; j < d; j += 32) {
      ccols[o + j] = ab[p + j];
      cw[o + j] = (int64_t)aw[p + j];
    }
  }
}

}  // namespace

// Inside aggregate_hash: a CUDA error frees the scratch before returning.
#define AG_CHECK(call)                                         \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return fail(set_cuda_error(_e));    \
  } while (0)

int aggregate_hash(cd_graph* g, const int32_t* labels_dev, const int32_t* newid_dev, int64_t k,
                   cd_graph** coarse_out) {
  cudaStream_t s = g->stream;
  const int64_t n = g->n, m = g->nnz;
  const int bits = [&] {
    int b = 0;
    while (((int64_t)1 << b) < k) ++b;
    return b;
  }();
  int rc = CD_OK;
  // scratch
  uint64_t *vk = nullptr, *vk2 = nullptr;
  int64_t *vv = nullptr, *vv2 = nullptr, *mpre = nullptr, *sstart = nullptr, *ucnt = nullptr, *coff = nullptr;
  int64_t *tot = nullptr, *ch_off = nullptr, *toff = nullptr;
  int32_t *ab = nullptr, *wl = nullptr, *cl = nullptr, *ll = nullptr, *ch_seg = nullptr, *dch = nullptr;
  int32_t *tlg = nullptr, *owner = nullptr, *gk = nullptr;
  unsigned long long *aw = nullptr, *cnt = nullptr, *ub = nullptr, *gv = nullptr;
  int64_t* coarse_off = nullptr;
  int32_t* ccols = nullptr;
  int64_t* cw = nullptr;
  auto cleanup = [&]() {
    void* ps[] = {vk, vk2, vv, vv2, mpre, sstart, ucnt, coff, tot, ch_off, toff, ab, wl, cl, ll, ch_seg, dch,
                  tlg, owner, gk, aw, cnt, ub, gv};
    for (void* p : ps) dev_free(p, s);
  };
  auto fail = [&](int r) {
    cleanup();
    dev_free(coarse_off, s);
    dev_free(ccols, s);
    dev_free(cw, s);
    return r;
  };
  if ((rc = dev_alloc_t(&vk, n, s)) || (rc = dev_alloc_t(&vk2, n, s)) || (rc = dev_alloc_t(&vv, n, s)) ||
      (rc = dev_alloc_t(&vv2, n, s)) || (rc = dev_alloc_t(&mpre, n, s)) || (rc = dev_alloc_t(&sstart, k + 1, s)) ||
      (rc = dev_alloc_t(&ucnt, k, s)) || (rc = dev_alloc_t(&coff, k, s)) || (rc = dev_alloc_t(&tot, 1, s)) ||
      (rc = dev_alloc_t(&ab, m, s)) || (rc = dev_alloc_t(&aw, m, s)) || (rc = dev_alloc_t(&cnt, 8, s)))
    return fail(rc);
  const int wbytes = g->wkind == W_UNIT ? 0 : g->wkind == W_I32 ? 4 : 8;

  // 1-2: members by community, segments, scatter
  uint64_t* sk = vk;
  int64_t* sv = vv;
  {
    KTimer t(g, K_SORT, (double)n * 32 * ((bits + 7) / 8));
    if (n > 0) CD_LAUNCH(k_ag_vkeys<<<gcap((n + NT - 1) / NT), NT, 0, s>>>(labels_dev, newid_dev, n, vk, vv));
    if ((rc = radix_sort_pairs(vk, vv, vk2, vv2, n, bits, s, &sk, &sv))) return fail(rc);
  }
  {
    KTimer t(g, K_AGG_EMIT, (double)n * (8 + 16 + 8 + 8) + (double)m * (4 + 4 + 4 + wbytes + 4 + 8));
    if (n > 0) CD_LAUNCH(k_ag_mdeg<<<gcap((n + NT - 1) / NT), NT, 0, s>>>(g->off, sv, n, mpre));
    if ((rc = exclusive_scan_i64(mpre, mpre, n, tot, s))) return fail(rc);
    if (n > 0) CD_LAUNCH(k_ag_heads<<<gcap((n + NT - 1) / NT), NT, 0, s>>>(sk, mpre, n, sstart));
    AG_CHECK(cudaMemcpyAsync(sstart + k, tot, 8, cudaMemcpyDeviceToDevice, s));
    if (m > 0) {
      const unsigned gr = gcap((n + NW - 1) / NW);
      if (g->wkind == W_UNIT)
        CD_LAUNCH(k_ag_scatter<WUnit><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, labels_dev, newid_dev, sv, mpre, n, ab, aw));
      else if (g->wkind == W_I32)
        CD_LAUNCH(k_ag_scatter<WI32><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, labels_dev, newid_dev, sv, mpre, n, ab, aw));
      else
        CD_LAUNCH(k_ag_scatter<WI64><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, labels_dev, newid_dev, sv, mpre, n, ab, aw));
    }
  }
  // the vertex-sort buffers are no longer needed
  dev_free(vk, s);
  dev_free(vk2, s);
  dev_free(vv, s);
  dev_free(vv2, s);
  vk = vk2 = nullptr;
  vv = vv2 = nullptr;

  int64_t nseg = 0;
  {
    KTimer t(g, K_AGG_REDUCE, (double)m * 2 * (4 + 8) + (double)k * 32);
    // 3: classes
    unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    AG_CHECK(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
    if (k > 0) CD_LAUNCH(k_ag_class_count<<<gcap((k + NT - 1) / NT), NT, 0, s>>>(sstart, k, cnt));
    AG_CHECK(cudaMemcpyAsync(h, cnt, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    AG_CHECK(cudaStreamSynchronize(s));
    const int64_t nw = (int64_t)h[0], nc = (int64_t)h[1], nl = (int64_t)h[2], nch = (int64_t)h[3];
    if ((rc = dev_alloc_t(&wl, nw, s)) || (rc = dev_alloc_t(&cl, nc, s)) || (rc = dev_alloc_t(&ll, nl, s)) ||
        (rc = dev_alloc_t(&ch_seg, nch, s)) || (rc = dev_alloc_t(&ch_off, nch, s)) || (rc = dev_alloc_t(&dch, nch, s)))
      return fail(rc);
    AG_CHECK(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
    if (k > 0) CD_LAUNCH(k_ag_class_fill<<<gcap((k + NT - 1) / NT), NT, 0, s>>>(sstart, k, cnt, wl, cl, ll, ch_seg, ch_off));
    if (nl > 0) {
      if ((rc = dev_alloc_t(&ub, k, s)) || (rc = dev_alloc_t(&tlg, k, s)) || (rc = dev_alloc_t(&toff, k, s)))
        return fail(rc);
      AG_CHECK(cudaMemsetAsync(ub, 0, k * sizeof(unsigned long long), s));
      AG_CHECK(cudaMemsetAsync(ucnt, 0, k * sizeof(int64_t), s));  // large segments count by atomics
    }
    const size_t wsm = (size_t)NW * AG_WCAP * 12 + (size_t)NW * 32 * 8 + (size_t)NW * AG_WCAP * 2;
    const size_t csm = (size_t)AG_CCAP * 12 + (size_t)(AG_CNT / 32) * 32 * 8 + (size_t)AG_CCAP * 2;
    AG_CHECK(cudaFuncSetAttribute(k_ag_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
    AG_CHECK(cudaFuncSetAttribute(k_ag_cta<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
    AG_CHECK(cudaFuncSetAttribute(k_ag_cta<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
    if (nw > 0) CD_LAUNCH(k_ag_warp<<<gcap((nw + NW - 1) / NW, 152 * 4), NT, wsm, s>>>(sstart, wl, nw, ab, aw, ucnt));
    if (nc > 0)
      CD_LAUNCH(k_ag_cta<false><<<gcap(nc, 152 * 2), AG_CNT, csm, s>>>(sstart, cl, nullptr, nc, ab, aw, ucnt, nullptr, nullptr));
    if (nl > 0) {
      CD_LAUNCH(k_ag_cta<true><<<gcap(nch, 152 * 2), AG_CNT, csm, s>>>(sstart, ch_seg, ch_off, nch, ab, aw, ucnt, dch, ub));
      AG_CHECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
      CD_LAUNCH(k_ag_tables_size<<<gcap((nl + NT - 1) / NT), NT, 0, s>>>(ll, nl, ub, tlg, toff, cnt));
      unsigned long long slots = 0;
      AG_CHECK(cudaMemcpyAsync(&slots, cnt, sizeof(slots), cudaMemcpyDeviceToHost, s));
      AG_CHECK(cudaStreamSynchronize(s));
      const int64_t nslices = (int64_t)slots / AG_SLICE;
      if ((rc = dev_alloc_t(&gk, (int64_t)slots, s)) || (rc = dev_alloc_t(&gv, (int64_t)slots, s)) ||
          (rc = dev_alloc_t(&owner, nslices, s)))
        return fail(rc);
      AG_CHECK(cudaMemsetAsync(gk, 0xff, slots * sizeof(int32_t), s));
      AG_CHECK(cudaMemsetAsync(gv, 0, slots * sizeof(unsigned long long), s));
      CD_LAUNCH(k_ag_tables_own<<<gcap(nl, 152 * 8), NT, 0, s>>>(ll, nl, tlg, toff, owner));
      CD_LAUNCH(k_ag_merge<<<gcap(nch, 152 * 8), NT, 0, s>>>(sstart, ch_seg, ch_off, dch, nch, ab, aw, tlg, toff, gk, gv));
      CD_LAUNCH(k_ag_extract<<<gcap(nslices, 152 * 8), NT, 0, s>>>(owner, nslices, gk, gv, sstart, ab, aw, ucnt));
    }
    // 4: compact into the coarse CSR
    if ((rc = exclusive_scan_i64(ucnt, coff, k, tot, s))) return fail(rc);
    AG_CHECK(cudaMemcpyAsync(&nseg, tot, 8, cudaMemcpyDeviceToHost, s));
    AG_CHECK(cudaStreamSynchronize(s));
    if ((rc = dev_alloc_t(&coarse_off, k + 1, s)) || (rc = dev_alloc_t(&ccols, nseg + COL_PAD, s)) ||
        (rc = dev_alloc_t(&cw, nseg, s)))
      return fail(rc);
    AG_CHECK(cudaMemcpyAsync(coarse_off, coff, k * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    AG_CHECK(cudaMemcpyAsync(coarse_off + k, tot, 8, cudaMemcpyDeviceToDevice, s));
    AG_CHECK(cudaMemsetAsync(ccols + nseg, 0, COL_PAD * sizeof(int32_t), s));
    if (k > 0 && nseg > 0)
      CD_LAUNCH(k_ag_compact<<<gcap((k + NW - 1) / NW), NT, 0, s>>>(sstart, ucnt, coff, k, ab, aw, ccols, cw));
    if (cudaGetLastError() != cudaSuccess) return fail(CD_ECUDA);
  }
  cleanup();
  cd_graph* c = nullptr;
  rc = graph_adopt(s, k, nseg, coarse_off, ccols, cw, W_I64, &c, nullptr, nullptr, g);
  if (rc) return rc;
  c->timing = g->timing;
  c->ktiming = g->ktiming;
  c->cols_distinct = true;  // one arc per pair of communities
  *coarse_out = c;
  return CD_OK;
}

#undef AG_CHECK

}  // namespace cd
