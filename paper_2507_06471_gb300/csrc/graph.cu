// Graph ingest (Sec. II-A): device copy of a symmetric CSR, validation,
// weighted degrees deg_w(v) (loops counted twice) and vol(V); static degree
// bins for the scan kernels and the global hash tables of hub vertices.
//
// Internal weight convention: a loop arc v->v carries 2L, so that deg_w(v) is
// the plain row sum and aggregation/modularity sum arc weights without special
// cases. Upload doubles loop arcs; cd_graph_download halves them back.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>

#include <mutex>

#include "common.cuh"

namespace cd {

const char* const kKernelNames[K_COUNT] = {
    "ingest",     "scan_tile4", "scan_tile8", "scan_tile16", "scan_tile32", "scan_warp",
    "scan_blk128", "hub_build", "hub_eval",   "apply_moves", "renumber",    "agg_emit",
    "radix_sort", "agg_reduce", "modularity", "hub_mark", "frontier", "scan_blk512", "hub_prepare"};

static thread_local int g_last_cuda = 0;
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int set_cuda_error(cudaError_t e) {
  g_last_cuda = (int)e;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return CD_ENOMEM;
  }
  return CD_ECUDA;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  // keep freed blocks in the device's default pool (threads may race here)
  static std::once_flag pool_set;
  std::call_once(pool_set, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    return set_cuda_error(e);
  }
  return CD_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

KTimer::KTimer(cd_graph* g_, int k_, double bytes_, cudaStream_t st_) : g(g_), k(k_), bytes(bytes_), st(st_) {
  if (g && g->ktiming) {
    if (!st) st = g->stream;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
}

KTimer::~KTimer() {
  if (g && g->ktiming) {
    cudaEventRecord(b, st);
    g->pending.push_back({k, {a, b}});
    g->pending_bytes.push_back(bytes);
  }
}

void profile_reset(cd_graph* g) {
  for (int k = 0; k < K_COUNT; ++k) {
    memset(&g->prof[k], 0, sizeof(cd_kernel_profile));
    snprintf(g->prof[k].name, sizeof(g->prof[k].name), "%s", kKernelNames[k]);
  }
}

int profile_flush(cd_graph* g) {
  if (g->pending.empty()) return CD_OK;
  CD_CHECK(cudaStreamSynchronize(g->stream));
  for (size_t i = 0; i < g->pending.size(); ++i) {
    auto& p = g->pending[i];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    cd_kernel_profile& kp = g->prof[p.first];
    kp.launches += 1;
    kp.total_ms += ms;
    kp.alg_bytes += g->pending_bytes[i];
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  g->pending.clear();
  g->pending_bytes.clear();
  return CD_OK;
}

namespace {

constexpr int NT = 256;
constexpr int NSTATS = 5 + NBINS;

__device__ __forceinline__ void fail(int32_t* status, int code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ int bin_of(int64_t d, int t_warp = WARP_MAX, int t_hub = BLOCK_MAX) {
  if (d <= 4) return B_T4;
  if (d <= 8) return B_T8;
  if (d <= 16) return B_T16;
  if (d <= 32) return B_T32;
  if (d <= t_warp) return B_WARP;
  if (d > t_hub) return B_HUB;
  return d <= BLK1_MAX ? B_BLK1 : B_BLK4;
}

__global__ void k_bin_count(const int64_t* __restrict__ off, int64_t n, int t_warp, int t_hub,
                            unsigned long long* counts) {
  __shared__ unsigned long long sb[NBINS];
  if (threadIdx.x < NBINS) sb[threadIdx.x] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int64_t d = off[v + 1] - off[v];
    if (d > 0) atomicAdd(&sb[bin_of(d, t_warp, t_hub)], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < NBINS && sb[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sb[threadIdx.x]);
}

template <class OffT>
__global__ void k_offsets_check(const OffT* __restrict__ in, int64_t n, int64_t nnz,
                                int64_t* __restrict__ out, int32_t* status) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
    int64_t a = (int64_t)in[i];
    out[i] = a;
    if (a < 0 || a > nnz) fail(status, CD_ENOTSYM);
    if (i < n && (int64_t)in[i + 1] < a) fail(status, CD_ENOTSYM);
    if (i == 0 && a != 0) fail(status, CD_ENOTSYM);
    if (i == n && a != nnz) fail(status, CD_ENOTSYM);
  }
}

// Ingest: bounds-check columns and weights, deg_w with loops twice, loop
// count, vol(V), per-bin vertex counts, and whether every row's columns are
// strictly increasing (then no row repeats a column). stats: [0] vol,
// [1] loops, [2] isolated, [3] largest deg_w, [4..4+NBINS) bin counts,
// [4+NBINS] rows not strictly increasing.
//
// Load balance: each lane owns one vertex of its warp's 32 consecutive ones
// and sums a row of at most INGEST_LANE arcs alone; the warp sums the rows of
// up to INGEST_WARP arcs one at a time with coalesced loads; longer rows are
// listed for k_ingest_big (a CTA per row).
constexpr int64_t HUB_LOG_DIV = 4;  // budget of logged hub updates per round: hub arcs / 4
constexpr int INGEST_LANE = 32;
constexpr int INGEST_WARP = 4096;
constexpr int ST_UNSORTED = 4 + NBINS;

struct RowSum {
  long long s, loops;
  bool unsorted;
};

template <class W>
__device__ __forceinline__ void ingest_arc(const int32_t* __restrict__ cols, const void* w, int64_t n, int64_t v,
                                           int64_t e, int64_t beg, int loops_twice, RowSum& r, int32_t* status) {
  const int32_t u = cols[e];
  const int64_t x = W::get(w, e);
  if (u < 0 || u >= n) fail(status, CD_EBOUNDS);
  if (x < 1) fail(status, CD_EINVAL);
  r.s += x;
  if (u == v) {
    if (loops_twice) r.s += x;  // input convention: the loop arc carries L
    ++r.loops;
  }
  if (e > beg && cols[e - 1] >= u) r.unsorted = true;
}

__device__ __forceinline__ void ingest_stats(unsigned long long* sb, int64_t d, long long s) {
  atomicMax(&sb[3], (unsigned long long)s);
  if (d == 0)
    atomicAdd(&sb[2], 1ull);
  else
    atomicAdd(&sb[4 + bin_of(d)], 1ull);
}

template <class W>
__global__ void __launch_bounds__(NT) k_ingest(const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ cols, const void* w,
                                               int64_t n, int loops_twice, int64_t* __restrict__ degw,
                                               unsigned long long* stats, int32_t* status,
                                               int32_t* big, unsigned long long* nbig) {
  __shared__ unsigned long long sb[NSTATS];
  for (int i = threadIdx.x; i < NSTATS; i += NT) sb[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  unsigned long long my_vol = 0, my_loops = 0;
  bool my_unsorted = false;
  for (int64_t v0 = warp * 32; v0 < n; v0 += nwarps * 32) {  // whole warps iterate together
    const int64_t v = v0 + lane;
    const bool ok = v < n;
    const int64_t beg = ok ? off[v] : 0, end = ok ? off[v + 1] : 0;
    const int64_t d = end - beg;
    RowSum r{0, 0, false};
    if (d <= INGEST_LANE) {
      for (int64_t e = beg; e < end; ++e) ingest_arc<W>(cols, w, n, v, e, beg, loops_twice, r, status);
      if (ok) {
        degw[v] = r.s;
        my_vol += (unsigned long long)r.s;
        my_loops += (unsigned long long)r.loops;
        my_unsorted |= r.unsorted;
        ingest_stats(sb, d, r.s);
      }
    } else if (d > INGEST_WARP) {
      big[atomicAdd(nbig, 1ull)] = (int32_t)v;
    }
    unsigned todo = __ballot_sync(FULL, d > INGEST_LANE && d <= INGEST_WARP);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t vv = v0 + src;
      const int64_t b = __shfl_sync(FULL, beg, src), en = __shfl_sync(FULL, end, src);
      RowSum q{0, 0, false};
      for (int64_t e = b + lane; e < en; e += 32) ingest_arc<W>(cols, w, n, vv, e, b, loops_twice, q, status);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        q.s += __shfl_xor_sync(FULL, q.s, o);
        q.loops += __shfl_xor_sync(FULL, q.loops, o);
      }
      my_unsorted |= q.unsorted;
      if (lane == src) {
        degw[vv] = q.s;
        my_vol += (unsigned long long)q.s;
        my_loops += (unsigned long long)q.loops;
        ingest_stats(sb, en - b, q.s);
      }
    }
  }
  atomicAdd(&sb[0], my_vol);
  atomicAdd(&sb[1], my_loops);
  if (my_unsorted) sb[ST_UNSORTED] = 1;
  __syncthreads();
  if (threadIdx.x < NSTATS && sb[threadIdx.x]) {
    if (threadIdx.x == 3)
      atomicMax(&stats[3], sb[3]);
    else
      atomicAdd(&stats[threadIdx.x], sb[threadIdx.x]);
  }
}

// The rows k_ingest listed (more than INGEST_WARP arcs): a CTA per row.
template <class W>
__global__ void __launch_bounds__(NT) k_ingest_big(const int64_t* __restrict__ off,
                                                   const int32_t* __restrict__ cols, const void* w,
                                                   int64_t n, int loops_twice, int64_t* __restrict__ degw,
                                                   unsigned long long* stats, int32_t* status,
                                                   const int32_t* __restrict__ big,
                                                   const unsigned long long* __restrict__ nbig) {
  __shared__ long long red[2][NT / 32];
  __shared__ int uns;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nb = (int64_t)*nbig;
  for (int64_t q = blockIdx.x; q < nb; q += gridDim.x) {
    const int64_t v = big[q];
    const int64_t beg = off[v], end = off[v + 1];
    if (threadIdx.x == 0) uns = 0;
    RowSum r{0, 0, false};
    for (int64_t e = beg + threadIdx.x; e < end; e += NT) ingest_arc<W>(cols, w, n, v, e, beg, loops_twice, r, status);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r.s += __shfl_xor_sync(FULL, r.s, o);
      r.loops += __shfl_xor_sync(FULL, r.loops, o);
    }
    if (lane == 0) {
      red[0][wid] = r.s;
      red[1][wid] = r.loops;
    }
    __syncthreads();
    if (r.unsorted) uns = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long s = 0, loops = 0;
      for (int i = 0; i < NT / 32; ++i) {
        s += red[0][i];
        loops += red[1][i];
      }
      degw[v] = s;
      atomicAdd(&stats[0], (unsigned long long)s);
      if (loops) atomicAdd(&stats[1], (unsigned long long)loops);
      atomicMax(&stats[3], (unsigned long long)s);
      atomicAdd(&stats[4 + bin_of(end - beg)], 1ull);
      if (uns) atomicOr(&stats[ST_UNSORTED], 1ull);
    }
    __syncthreads();
  }
}

// Internal weights with loop arcs doubled (int64).
template <class W>
__global__ void __launch_bounds__(NT) k_double_loops(const int64_t* __restrict__ off,
                                                     const int32_t* __restrict__ cols,
                                                     const void* w, int64_t n,
                                                     int64_t* __restrict__ w64) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps)
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) {
      int64_t x = W::get(w, e);
      w64[e] = cols[e] == v ? 2 * x : x;
    }
}

__global__ void __launch_bounds__(NT) k_bin_fill(const int64_t* __restrict__ off, int64_t n, int t_warp,
                                                 int t_hub, const int64_t* __restrict__ bin_base,
                                                 unsigned long long* cursor,
                                                 int32_t* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t limit = (n + 31) / 32 * 32;  // whole warps iterate together
  for (int64_t v = start; v < limit; v += stride) {
    int b = -1;
    if (v < n) {
      int64_t d = off[v + 1] - off[v];
      if (d > 0) b = bin_of(d, t_warp, t_hub);
    }
#pragma unroll
    for (int bb = 0; bb < NBINS; ++bb) {
      unsigned m = __ballot_sync(FULL, b == bb);
      if (!m) continue;
      unsigned long long pos = 0;
      int first = __ffs(m) - 1;
      if (lane == first) pos = atomicAdd(&cursor[bb], (unsigned long long)__popc(m));
      pos = __shfl_sync(FULL, pos, first);
      if (b == bb) list[bin_base[bb] + (int64_t)pos + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
    }
  }
}

__global__ void k_hub_bits(const int32_t* __restrict__ hubs, int64_t nh, uint32_t* hub_bits) {
  int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h < nh) {
    const int32_t v = hubs[h];
    atomicOr(&hub_bits[v >> 5], 1u << (v & 31));
  }
}

// Hubs are numbered in increasing vertex id, so the number of vertex u is its
// rank among the hubs: hub_pref[u / 32] (hubs below 32 (u / 32)) plus the hub
// bits below u in its word. hub_pref[w] = lower bound of 32 w in the sorted list.
__global__ void k_hub_pref(const int32_t* __restrict__ hubs, int64_t nh, int64_t nwords, uint32_t* hub_pref) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += stride) {
    int64_t lo = 0, hi = nh;  // first hub with vertex >= 32 w
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if ((int64_t)hubs[mid] < 32 * w) lo = mid + 1; else hi = mid;
    }
    hub_pref[w] = (uint32_t)lo;
  }
}

__global__ void k_gather_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ vs,
                              int64_t m, int64_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    int32_t v = vs[i];
    out[2 * i] = off[v];
    out[2 * i + 1] = off[v + 1];
  }
}

__global__ void k_download_w(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                             const void* w, int wkind, int64_t n, int64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps)
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) {
      int64_t x = wkind == W_UNIT ? 1 : wkind == W_I32 ? (int64_t)((const int32_t*)w)[e]
                                                       : ((const int64_t*)w)[e];
      out[e] = cols[e] == v ? x / 2 : x;  // loop arcs are stored doubled (2L)
    }
}

__global__ void k_narrow_w(const int64_t* __restrict__ w64, int64_t nnz, int32_t* __restrict__ w32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) w32[e] = (int32_t)w64[e];
}

__global__ void k_labels_check(const int32_t* __restrict__ lab, int64_t n, int32_t* status) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (lab[i] < 0 || lab[i] >= n) fail(status, CD_EINVAL);
}

unsigned grid_cap_u(int64_t blocks, int64_t cap) {
  if (blocks < 1) blocks = 1;
  return (unsigned)(blocks < cap ? blocks : cap);
}

unsigned grid_for(int64_t work, int per_block = NT) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

int read_status(cd_graph* g) {
  int32_t st = 0;
  CD_CHECK(cudaMemcpyAsync(&st, g->status, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  CD_CHECK(cudaStreamSynchronize(g->stream));
  if (st) CD_CHECK(cudaMemsetAsync(g->status, 0, sizeof(int32_t), g->stream));
  return st;
}

void free_arrays(cd_graph* g) {
  cudaStream_t s = g->stream;
  void* ps[] = {g->off,          g->cols,          g->w,            g->degw,         g->bin_list,
                g->act_list,     g->act_cnt,       g->full_cnt,     g->act_ev,       g->act_small,
                g->hub_cc,       g->hub_live,
                g->hub_pref,      g->hub_bits,      g->hub_tab,       g->hub_slot,
                g->hub_item_hub,  g->hub_item_arc, g->hub_ev_hub,   g->hub_ev_slot,
                g->hub_ev_first, g->hub_part,      g->hub_cur,      g->hub_hascur,   g->hub_done,
                g->hub_mv,       g->hub_rb,       g->hub_used,     g->hub_item_first,
                g->hub_flist,    g->hub_fcnt,     g->hub_cl,       g->hub_ccnt,
                g->hub_blist,    g->hub_mlist,     g->hub_lcnt,     g->C,            g->sigma,        g->csize,
                g->hub_log,
                g->sigma32,
                g->flag[0],      g->flag[1],       g->mv_v,         g->mv_c,         g->mv_a,
                g->ctr,          g->status,        g->gid,          g->gbase,        g->gvol,
                g->gfrozen,      g->gcnt};
  for (void* p : ps) dev_free(p, s);
  if (g->h_ctr) cudaFreeHost(g->h_ctr);
}

void free_bins(cd_graph* g) {
  cudaStream_t s = g->stream;
  void* ps[] = {g->bin_list,     g->act_list,    g->act_cnt,      g->full_cnt,  g->act_ev,
                g->act_small,    g->hub_cc,       g->hub_live,
                g->hub_pref,      g->hub_bits,     g->hub_tab,   g->hub_slot,
                g->hub_item_hub, g->hub_item_arc, g->hub_ev_hub,  g->hub_ev_slot, g->hub_ev_first,
                g->hub_part,     g->hub_cur,     g->hub_hascur,   g->hub_done,  g->hub_mv,
                g->hub_rb,       g->hub_used,     g->hub_item_first, g->hub_blist,
                g->hub_flist,    g->hub_fcnt,     g->hub_cl,       g->hub_ccnt,
                g->hub_mlist,    g->hub_lcnt,     g->hub_log};
  for (void* p : ps) dev_free(p, s);
  g->bin_list = nullptr;
  g->act_list = nullptr;
  g->act_cnt = nullptr;
  g->full_cnt = nullptr;
  g->act_ev = nullptr;
  g->act_small = nullptr;
  g->hub_cc = nullptr;
  g->hub_live = nullptr;
  g->hub_pref = nullptr;
  g->hub_bits = nullptr;
  g->hub_tab = nullptr;
  g->hub_slot = nullptr;
  g->hub_item_hub = nullptr;
  g->hub_item_arc = nullptr;
  g->hub_ev_hub = nullptr;
  g->hub_ev_slot = nullptr;
  g->hub_ev_first = nullptr;
  g->hub_part = nullptr;
  g->hub_cur = nullptr;
  g->hub_hascur = nullptr;
  g->hub_done = nullptr;
  g->hub_mv = nullptr;
  g->hub_rb = nullptr;
  g->hub_flist = nullptr;
  g->hub_fcnt = nullptr;
  g->hub_cl = nullptr;
  g->hub_ccnt = nullptr;
  g->hub_used = nullptr;
  g->hub_item_first = nullptr;
  g->hub_blist = nullptr;
  g->hub_mlist = nullptr;
  g->hub_lcnt = nullptr;
  g->hub_log = nullptr;
  g->hub_log_cap = 0;
  g->nhubs = g->hub_slots = g->hub_items = g->hub_eval_items = 0;
}

int build_bins(cd_graph* g);

// Scalars, bins and hub structures of a graph whose CSR, weights and deg_w
// are in place; stats from k_ingest.
int finish_graph(cd_graph* g, const unsigned long long* stats) {
  g->cols_distinct = stats[ST_UNSORTED] == 0;  // strictly increasing rows; aggregation sets it for coarse rows
  g->vol = (int64_t)stats[0];
  g->n_isolated = (int64_t)stats[2];
  g->max_degw = (int64_t)stats[3];
  if (stats[0] >= (1ull << 62)) return CD_EOVERFLOW;
  return build_bins(g);
}

// Degree bins for (t_warp, t_hub), and the hub histograms' layout.
int build_bins(cd_graph* g) {
  cudaStream_t s = g->stream;
  int rc;
  {
    unsigned long long* d_cnt = nullptr;
    unsigned long long h_cnt[NBINS] = {};
    if ((rc = dev_alloc_t(&d_cnt, NBINS, s))) return rc;
    CD_CHECK(cudaMemsetAsync(d_cnt, 0, NBINS * sizeof(unsigned long long), s));
    if (g->n > 0)
      CD_LAUNCH(k_bin_count<<<grid_for(g->n), NT, 0, s>>>(g->off, g->n, g->t_warp, g->t_hub, d_cnt));
    CD_CHECK(cudaMemcpyAsync(h_cnt, d_cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, s));
    CD_CHECK(cudaStreamSynchronize(s));
    dev_free(d_cnt, s);
    g->bin_start[0] = 0;
    for (int b = 0; b < NBINS; ++b) g->bin_start[b + 1] = g->bin_start[b] + (int64_t)h_cnt[b];
  }
  int64_t listed = g->bin_start[NBINS];
  rc = dev_alloc_t(&g->bin_list, listed, s);
  if (rc) return rc;
  if ((rc = dev_alloc_t(&g->act_list, listed, s))) return rc;
  if ((rc = dev_alloc_t(&g->act_cnt, NBINS + 2, s))) return rc;
  if ((rc = dev_alloc_t(&g->full_cnt, NBINS + 2, s))) return rc;
  int64_t* d_base = nullptr;
  unsigned long long* d_cur = nullptr;
  if ((rc = dev_alloc_t(&d_base, NBINS, s))) return rc;
  if ((rc = dev_alloc_t(&d_cur, NBINS, s))) return rc;
  CD_CHECK(cudaMemcpyAsync(d_base, g->bin_start, NBINS * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CD_CHECK(cudaMemsetAsync(d_cur, 0, NBINS * sizeof(unsigned long long), s));
  if (g->n > 0)
    CD_LAUNCH(k_bin_fill<<<grid_for(g->n), NT, 0, s>>>(g->off, g->n, g->t_warp, g->t_hub, d_base, d_cur,
                                                       g->bin_list));
  CD_CHECK(cudaGetLastError());
  // hubs: host-side layout of tables and work items
  int64_t nh = g->bin_start[B_HUB + 1] - g->bin_start[B_HUB];
  g->nhubs = nh;
  if (nh > 0) {
    {  // hubs in increasing vertex id (their number is their rank)
      std::vector<int32_t> hv(nh);
      int32_t* dl = g->bin_list + g->bin_start[B_HUB];
      CD_CHECK(cudaMemcpyAsync(hv.data(), dl, nh * 4, cudaMemcpyDeviceToHost, s));
      CD_CHECK(cudaStreamSynchronize(s));
      std::sort(hv.begin(), hv.end());
      CD_CHECK(cudaMemcpyAsync(dl, hv.data(), nh * 4, cudaMemcpyHostToDevice, s));
      CD_CHECK(cudaStreamSynchronize(s));  // hv dies here
    }
    int64_t* d_rows = nullptr;
    if ((rc = dev_alloc_t(&d_rows, 2 * nh, s))) return rc;
    CD_LAUNCH(k_gather_rows<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(g->off, g->bin_list + g->bin_start[B_HUB],
                                                              nh, d_rows));
    std::vector<int64_t> rows(2 * nh);
    CD_CHECK(cudaMemcpyAsync(rows.data(), d_rows, 2 * nh * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CHECK(cudaStreamSynchronize(s));
    dev_free(d_rows, s);
    std::vector<int64_t> tab(nh + 1, 0), item_arc, ev_first(nh + 1, 0), ev_slot, item_first(nh + 1, 0);
    std::vector<int32_t> item_hub, ev_hub;
    std::vector<int64_t> cc(nh);
    for (int64_t h = 0; h < nh; ++h) {
      int64_t beg = rows[2 * h], deg = rows[2 * h + 1] - beg;
      int64_t cap = deg + deg / 2 + 64;  // live labels <= deg; the rest absorbs labels that come and go
      tab[h + 1] = tab[h] + cap;
      item_first[h] = (int64_t)item_hub.size();
      for (int64_t a = 0; a < deg; a += HUB_CHUNK) {
        item_hub.push_back((int32_t)h);
        item_arc.push_back(beg + a);
      }
      ev_first[h] = (int64_t)ev_hub.size();
      for (int64_t e = 0; e < cap; e += HUB_SLICE) {
        ev_hub.push_back((int32_t)h);
        ev_slot.push_back(e);
      }
    }
    ev_first[nh] = (int64_t)ev_hub.size();
    item_first[nh] = (int64_t)item_hub.size();
    g->hub_slots = tab[nh];
    g->hub_items = (int64_t)item_hub.size();
    g->hub_eval_items = (int64_t)ev_hub.size();
    if ((rc = dev_alloc_t(&g->act_ev, g->hub_eval_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->act_small, nh, s))) return rc;  // any hub whose table in use is small
    if ((rc = dev_alloc_t(&g->hub_cc, nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_live, nh, s))) return rc;
    for (int64_t h = 0; h < nh; ++h) cc[h] = tab[h + 1] - tab[h];  // every table starts at its allocation
    CD_CHECK(cudaMemcpyAsync(g->hub_cc, cc.data(), nh * 8, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemsetAsync(g->hub_live, 0, nh * 4, s));
    if ((rc = dev_alloc_t(&g->hub_pref, (g->n + 31) / 32, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_bits, (g->n + 31) / 32, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_tab, nh + 1, s))) return rc;
    g->hub_wide = g->max_degw >= ((int64_t)1 << 32) ? 1 : 0;
    if ((rc = dev_alloc_t(&g->hub_slot, g->hub_slots * (1 + g->hub_wide), s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_item_hub, g->hub_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_item_arc, g->hub_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_ev_hub, g->hub_eval_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_ev_slot, g->hub_eval_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_ev_first, nh + 1, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_part, 3 * g->hub_eval_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_cur, nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_hascur, nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_done, nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_mv, 3 * nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_rb, nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_flist, 2 * nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_fcnt, 2, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_cl, 5 * nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_ccnt, 5, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_used, nh, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_item_first, nh + 1, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_blist, g->hub_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_mlist, g->hub_items, s))) return rc;
    if ((rc = dev_alloc_t(&g->hub_lcnt, 2, s))) return rc;
    {  // a round applies at most hub_arcs / HUB_LOG_DIV logged updates (random probes
       // into the tables cost about as much as rebuilding the hubs); the hub of
       // every update beyond that budget is rebuilt from its row instead
      const int64_t hub_arcs = tab[nh] * 2 / 3;
      g->hub_log_cap = std::max<int64_t>(1, hub_arcs / HUB_LOG_DIV);
      if ((rc = dev_alloc_t(&g->hub_log, 2 * g->hub_log_cap, s))) return rc;
    }
    CD_CHECK(cudaMemcpyAsync(g->hub_tab, tab.data(), (nh + 1) * 8, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemcpyAsync(g->hub_item_hub, item_hub.data(), item_hub.size() * 4, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemcpyAsync(g->hub_item_arc, item_arc.data(), item_arc.size() * 8, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemcpyAsync(g->hub_ev_hub, ev_hub.data(), ev_hub.size() * 4, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemcpyAsync(g->hub_ev_slot, ev_slot.data(), ev_slot.size() * 8, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemcpyAsync(g->hub_ev_first, ev_first.data(), (nh + 1) * 8, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemcpyAsync(g->hub_item_first, item_first.data(), (nh + 1) * 8, cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaMemsetAsync(g->hub_rb, 0, nh * 4, s));
    CD_CHECK(cudaMemsetAsync(g->hub_used, 0, nh * 4, s));
    CD_CHECK(cudaMemsetAsync(g->hub_lcnt, 0, 2 * 8, s));
    CD_CHECK(cudaMemsetAsync(g->hub_fcnt, 0, 2 * 8, s));
    CD_CHECK(cudaMemsetAsync(g->hub_ccnt, 0, 5 * 8, s));
    CD_CHECK(cudaMemsetAsync(g->hub_cur, 0, nh * 8, s));
    CD_CHECK(cudaMemsetAsync(g->hub_hascur, 0, nh * 4, s));
    CD_CHECK(cudaMemsetAsync(g->hub_done, 0, nh * 4, s));
    CD_CHECK(cudaMemsetAsync(g->hub_bits, 0, (g->n + 31) / 32 * 4, s));
    CD_LAUNCH(k_hub_bits<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(g->bin_list + g->bin_start[B_HUB], nh,
                                                                      g->hub_bits));
    CD_LAUNCH(k_hub_pref<<<grid_for((g->n + 31) / 32), NT, 0, s>>>(g->bin_list + g->bin_start[B_HUB], nh,
                                                                   (g->n + 31) / 32, g->hub_pref));
    CD_CHECK(cudaStreamSynchronize(s));  // the host vectors above die here
  }
  {
    unsigned long long full[NBINS + 2];
    for (int b = 0; b < NBINS; ++b) full[b] = (unsigned long long)(g->bin_start[b + 1] - g->bin_start[b]);
    full[NBINS] = full[NBINS + 1] = 0;  // hub evaluate work is routed per round
    CD_CHECK(cudaMemcpyAsync(g->full_cnt, full, sizeof(full), cudaMemcpyHostToDevice, s));
    CD_CHECK(cudaStreamSynchronize(s));  // `full` lives on this stack frame
  }
  dev_free(d_base, s);
  dev_free(d_cur, s);
  return CD_OK;
}

int ingest(cd_graph* g, int loops_twice, unsigned long long* stats_host) {
  cudaStream_t s = g->stream;
  unsigned long long* d_stats = nullptr;
  int rc = dev_alloc_t(&d_stats, NSTATS, s);
  if (rc) return rc;
  CD_CHECK(cudaMemsetAsync(d_stats, 0, (NSTATS) * sizeof(unsigned long long), s));
  int32_t* big = nullptr;
  unsigned long long* nbig = nullptr;
  const int64_t big_cap = g->nnz / (INGEST_WARP + 1) + 1;  // rows longer than INGEST_WARP arcs, at most
  if ((rc = dev_alloc_t(&big, big_cap, s)) || (rc = dev_alloc_t(&nbig, 1, s))) {
    dev_free(big, s);
    dev_free(d_stats, s);
    return rc;
  }
  CD_CHECK(cudaMemsetAsync(nbig, 0, sizeof(unsigned long long), s));
  {
    KTimer t(g, K_UPLOAD, (double)g->nnz * (4 + (g->wkind == W_I32 ? 4 : g->wkind == W_I64 ? 8 : 0)) +
                              (double)g->n * 16);
    if (g->n > 0) {
      const unsigned gr = grid_for((g->n + 31) / 32 * 32);
      const unsigned gb = grid_cap_u(big_cap, 152 * 8);
#define CD_INGEST(WT)                                                                                      \
  CD_LAUNCH(k_ingest<WT><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, g->n, loops_twice, g->degw, d_stats,     \
                                           g->status, big, nbig));                                         \
  CD_LAUNCH(k_ingest_big<WT><<<gb, NT, 0, s>>>(g->off, g->cols, g->w, g->n, loops_twice, g->degw, d_stats, \
                                               g->status, big, nbig))
      if (g->wkind == W_UNIT) {
        CD_INGEST(WUnit);
      } else if (g->wkind == W_I32) {
        CD_INGEST(WI32);
      } else {
        CD_INGEST(WI64);
      }
#undef CD_INGEST
    }
  }
  dev_free(big, s);
  dev_free(nbig, s);
  CD_CHECK(cudaGetLastError());
  CD_CHECK(cudaMemcpyAsync(stats_host, d_stats, (NSTATS) * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  dev_free(d_stats, s);
  CD_CHECK(cudaStreamSynchronize(s));
  return CD_OK;
}

}  // namespace

int rebin(cd_graph* g, int t_warp, int t_hub) {
  if (t_warp < 32 || t_warp > WARP_MAX || t_hub < t_warp || t_hub > BLK4_MAX) return CD_EINVAL;
  g->bins_set = true;
  if (t_warp == g->t_warp && t_hub == g->t_hub && g->bin_list) return CD_OK;
  CD_CHECK(cudaStreamSynchronize(g->stream));
  free_bins(g);
  g->t_warp = t_warp;
  g->t_hub = t_hub;
  return build_bins(g);
}

int ensure_run_state(cd_graph* g) {
  if (g->C) return CD_OK;
  cudaStream_t s = g->stream;
  int rc;
  if ((rc = dev_alloc_t(&g->C, g->n, s))) return rc;
  if ((rc = dev_alloc_t(&g->sigma, g->n, s))) return rc;
  if ((rc = dev_alloc_t(&g->csize, g->n, s))) return rc;
  if ((rc = dev_alloc_t(&g->flag[0], (g->n + 31) / 32 + 1, s))) return rc;
  if ((rc = dev_alloc_t(&g->flag[1], (g->n + 31) / 32 + 1, s))) return rc;
  if ((rc = dev_alloc_t(&g->mv_v, g->n, s))) return rc;
  if ((rc = dev_alloc_t(&g->mv_c, g->n, s))) return rc;
  if ((rc = dev_alloc_t(&g->mv_a, g->n, s))) return rc;
  if ((rc = dev_alloc_t(&g->ctr, C_COUNT, s))) return rc;
  if (!g->h_ctr) CD_CHECK(cudaMallocHost(&g->h_ctr, C_COUNT * sizeof(int64_t)));
  return CD_OK;
}

int check_labels(cd_graph* g, const int32_t* labels_dev) {
  if (g->n == 0) return CD_OK;
  CD_LAUNCH(k_labels_check<<<grid_for(g->n), NT, 0, g->stream>>>(labels_dev, g->n, g->status));
  CD_CHECK(cudaGetLastError());
  int st = read_status(g);
  return st ? st : CD_OK;
}

// Takes ownership of device arrays already in the internal convention (loop
// arcs carry 2L). If degw_pre is given (with its ingest stats) it is adopted
// too; otherwise deg_w is computed as the plain row sum.
int graph_adopt(cudaStream_t s, int64_t n, int64_t nnz, int64_t* off, int32_t* cols, void* w,
                int wkind, cd_graph** out, int64_t* degw_pre, const unsigned long long* stats_pre,
                const cd_graph* like) {
  cd_graph* g = new cd_graph();
  if (like) {
    g->t_warp = like->t_warp;
    g->t_hub = like->t_hub;
    g->bins_set = like->bins_set;
    if (!g->bins_set && nnz >= COARSE_HUB_ARCS && g->t_hub > COARSE_T_HUB && g->t_warp <= COARSE_T_HUB)
      g->t_hub = COARSE_T_HUB;
  }
  g->stream = s;
  g->n = n;
  g->nnz = nnz;
  g->off = off;
  g->cols = cols;
  g->w = w;
  g->wkind = wkind;
  g->degw = degw_pre;
  profile_reset(g);
  int rc = dev_alloc_t(&g->status, 1, s);
  if (!rc && cudaMemsetAsync(g->status, 0, 4, s) != cudaSuccess) rc = CD_ECUDA;
  unsigned long long stats[NSTATS] = {};
  if (stats_pre) {
    memcpy(stats, stats_pre, sizeof(stats));
  } else {
    if (!rc) rc = dev_alloc_t(&g->degw, n, s);
    if (!rc) rc = ingest(g, 0, stats);
    if (!rc) {
      int st = read_status(g);
      if (st) rc = st;
    }
  }
  // 64-bit weights whose every row sum (loops doubled included) is below 2^31
  // are kept in 32 bits: every arc weight is at most its row's deg_w
  if (!rc && g->wkind == W_I64 && g->w && nnz > 0 && stats[3] < (1ull << 31)) {
    int32_t* w32 = nullptr;
    rc = dev_alloc_t(&w32, nnz, s);
    if (!rc) {
      CD_LAUNCH(k_narrow_w<<<grid_for(nnz), NT, 0, s>>>((const int64_t*)g->w, nnz, w32));
      dev_free(g->w, s);
      g->w = w32;
      g->wkind = W_I32;
    }
  }
  if (!rc) rc = finish_graph(g, stats);
  if (rc) {
    free_arrays(g);
    delete g;
    return rc;
  }
  *out = g;
  return CD_OK;
}

}  // namespace cd

using namespace cd;

extern "C" {

int cd_params_default(cd_params* p) {
  if (!p) return CD_EINVAL;
  p->max_iter = 100;
  p->max_levels = 64;
  p->threshold = 0;
  p->tie_keep_current = 1;
  p->singleton_rule = 1;
  p->use_frontier = 1;
  p->timing = 0;
  p->sched_seed = 0x5EED5EEDull;
  p->aggregation = 0;
  p->asynchronous = 0;
  p->device_loop = 1;
  return CD_OK;
}

int cd_last_cuda_error(void) { return g_last_cuda; }

int64_t cd_launch_count(void) { return (int64_t)g_launches.load(); }

const char* cd_status_string(int st) {
  switch (st) {
    case CD_OK: return "ok";
    case CD_EINVAL: return "invalid argument (null pointer, size, weight < 1 or label out of range)";
    case CD_EBOUNDS: return "column id outside [0, n)";
    case CD_ENOMEM: return "device allocation failed";
    case CD_ECUDA: return "CUDA runtime error";
    case CD_EOVERFLOW: return "size overflow (vol(V) >= 2^62 or n >= 2^31)";
    case CD_ETIMEOUT: return "bounded device wait ran out";
    case CD_ENOTSYM: return "malformed CSR offsets";
    default: return "unknown status";
  }
}

int cd_csr_upload(const void* offsets, int offsets_is_i64, const int32_t* cols, const int32_t* w,
                  int64_t n, int64_t nnz, int ptrs_on_device, void* stream, cd_graph** out) {
  if (!out || n < 0 || nnz < 0 || !offsets || (nnz > 0 && !cols)) return CD_EINVAL;
  if (n >= (int64_t)INT32_MAX) return CD_EOVERFLOW;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cd_graph tmp;
  tmp.stream = s;
  tmp.n = n;
  tmp.nnz = nnz;
  profile_reset(&tmp);
  int rc = dev_alloc_t(&tmp.status, 1, s);
  int32_t* d_cols = nullptr;
  int64_t* d_off = nullptr;
  int32_t* d_w = nullptr;
  void* d_off_in = nullptr;
  if (!rc) rc = dev_alloc_t(&d_off, n + 1, s);
  if (!rc) rc = dev_alloc_t(&d_cols, nnz + COL_PAD, s);
  if (!rc && cudaMemsetAsync(d_cols + nnz, 0, COL_PAD * sizeof(int32_t), s) != cudaSuccess) rc = CD_ECUDA;
  if (!rc && w) rc = dev_alloc_t(&d_w, nnz, s);
  size_t ob = (size_t)(n + 1) * (offsets_is_i64 ? 8 : 4);
  if (!rc) rc = dev_alloc(&d_off_in, ob, s);
  auto cleanup = [&]() {
    dev_free(d_cols, s);
    dev_free(d_off, s);
    dev_free(d_w, s);
    dev_free(d_off_in, s);
    dev_free(tmp.status, s);
  };
  if (rc) {
    cleanup();
    return rc;
  }
  if (cudaMemsetAsync(tmp.status, 0, 4, s) != cudaSuccess ||
      cudaMemcpyAsync(d_off_in, offsets, ob, kind, s) != cudaSuccess ||
      (nnz > 0 && cudaMemcpyAsync(d_cols, cols, (size_t)nnz * 4, kind, s) != cudaSuccess) ||
      (w && nnz > 0 && cudaMemcpyAsync(d_w, w, (size_t)nnz * 4, kind, s) != cudaSuccess)) {
    int e = set_cuda_error(cudaGetLastError());
    cleanup();
    return e;
  }
  if (offsets_is_i64)
    CD_LAUNCH(k_offsets_check<int64_t><<<grid_for(n + 1), NT, 0, s>>>((const int64_t*)d_off_in, n, nnz, d_off,
                                                            tmp.status));
  else
    CD_LAUNCH(k_offsets_check<int32_t><<<grid_for(n + 1), NT, 0, s>>>((const int32_t*)d_off_in, n, nnz, d_off,
                                                            tmp.status));
  int32_t st = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&st, tmp.status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cleanup();
    return CD_ECUDA;
  }
  dev_free(d_off_in, s);
  d_off_in = nullptr;
  if (st) {
    cleanup();
    return st;
  }
  // validate columns and weights, count loops, compute deg_w
  tmp.off = d_off;
  tmp.cols = d_cols;
  tmp.w = d_w;
  tmp.wkind = d_w ? W_I32 : W_UNIT;
  rc = dev_alloc_t(&tmp.degw, n, s);
  unsigned long long stats[NSTATS] = {};
  if (!rc) rc = ingest(&tmp, 1, stats);
  if (!rc && cudaMemcpyAsync(&st, tmp.status, 4, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess && st)
    rc = st;
  dev_free(tmp.status, s);
  tmp.status = nullptr;
  if (rc) {
    dev_free(tmp.degw, s);
    dev_free(d_cols, s);
    dev_free(d_off, s);
    dev_free(d_w, s);
    return rc;
  }
  // loops: switch to int64 weights with loop arcs doubled
  void* wint = d_w;
  int wk = d_w ? W_I32 : W_UNIT;
  if (stats[1] > 0) {
    int64_t* w64 = nullptr;
    rc = dev_alloc_t(&w64, nnz, s);
    if (rc) {
      dev_free(tmp.degw, s);
      dev_free(d_cols, s);
      dev_free(d_off, s);
      dev_free(d_w, s);
      return rc;
    }
    if (d_w)
      CD_LAUNCH(k_double_loops<WI32><<<grid_for(n * 32), NT, 0, s>>>(d_off, d_cols, d_w, n, w64));
    else
      CD_LAUNCH(k_double_loops<WUnit><<<grid_for(n * 32), NT, 0, s>>>(d_off, d_cols, nullptr, n, w64));
    dev_free(d_w, s);
    wint = w64;
    wk = W_I64;
  }
  return graph_adopt(s, n, nnz, d_off, d_cols, wint, wk, out, tmp.degw, stats);
}

int cd_graph_free(cd_graph* g) {
  if (!g) return CD_OK;
  free_arrays(g);
  for (auto& p : g->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  cudaStreamSynchronize(g->stream);
  delete g;
  return CD_OK;
}

int cd_graph_info(const cd_graph* g, int64_t* n, int64_t* nnz, int64_t* vol) {
  if (!g) return CD_EINVAL;
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (vol) *vol = g->vol;
  return CD_OK;
}

int cd_graph_download(const cd_graph* g, int64_t* off, int32_t* cols, int64_t* w, int on_device) {
  if (!g || !off || (g->nnz > 0 && !cols)) return CD_EINVAL;
  cudaStream_t s = g->stream;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CD_CHECK(cudaMemcpyAsync(off, g->off, (g->n + 1) * 8, k, s));
  if (g->nnz > 0) CD_CHECK(cudaMemcpyAsync(cols, g->cols, g->nnz * 4, k, s));
  if (w && g->nnz > 0) {
    int64_t* tmp = nullptr;
    int rc = dev_alloc_t(&tmp, g->nnz, s);
    if (rc) return rc;
    CD_LAUNCH(k_download_w<<<grid_for(g->n * 32), NT, 0, s>>>(g->off, g->cols, g->w, g->wkind, g->n, tmp));
    CD_CHECK(cudaMemcpyAsync(w, tmp, g->nnz * 8, k, s));
    dev_free(tmp, s);
  }
  CD_CHECK(cudaStreamSynchronize(s));
  return CD_OK;
}

int cd_trace_get(const cd_graph* g, cd_round_trace* out, int32_t cap, int32_t* count) {
  if (!g || !count) return CD_EINVAL;
  *count = (int32_t)g->trace.size();
  for (int32_t i = 0; i < cap && i < (int32_t)g->trace.size(); ++i) out[i] = g->trace[i];
  return CD_OK;
}

int cd_profile_get(const cd_graph* g, cd_kernel_profile* out, int32_t cap, int32_t* count) {
  if (!g || !count) return CD_EINVAL;
  *count = K_COUNT;
  for (int32_t i = 0; i < cap && i < K_COUNT; ++i) out[i] = g->prof[i];
  return CD_OK;
}

}  // extern "C"
