// Louvain aggregation (Algorithm 3, Aggregation), exact modularity (Sec.
// II-C) and the Louvain driver (Algorithm 3).
//
// Aggregation: communities are renumbered 0..k-1 in ascending id order (a
// used-flag array and an exclusive scan); every arc u->v becomes the 64-bit key
// (A << b) | B with A = new(C[u]), B = new(C[v]) and its weight as value; a
// stable LSD radix sort over the 2b key bits groups equal keys in (A, B)
// order; a segmented reduce (exclusive scans of head flags and of the weights)
// sums every run into one coarse arc. Rows come out sorted by column. Weights
// of the coarse graph are int64; a loop (A,A) collects every arc inside A, i.e.
// twice A's internal weight, which is the internal convention for loops.
//
// Modularity: Q = (I vol - S) / vol^2 with I = sum of arc weights inside
// communities (loop arcs carry 2L) and S = sum_c vol(c)^2 accumulated exactly
// in 128 bits; only the final quotient is FP64.
#include <algorithm>

#include "common.cuh"

namespace cd {
namespace {

constexpr int NT = 256;

unsigned grid_cap(int64_t blocks, int64_t cap = 152 * 16) {
  if (blocks < 1) blocks = 1;
  return (unsigned)(blocks < cap ? blocks : cap);
}

__global__ void k_mark_used(const int32_t* __restrict__ labels, int64_t n, uint8_t* used) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    used[labels[v]] = 1;
}

__global__ void k_fix_unused(const uint8_t* __restrict__ used, int64_t n, int32_t* newid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride)
    if (!used[c]) newid[c] = -1;
}

// Warp per vertex: one (key, weight) pair per arc.
template <class W>
__global__ void __launch_bounds__(NT) k_agg_emit(const int64_t* __restrict__ off,
                                                 const int32_t* __restrict__ cols, const void* w,
                                                 int64_t n, const int32_t* __restrict__ labels,
                                                 const int32_t* __restrict__ newid, int bits,
                                                 uint64_t* __restrict__ keys,
                                                 int64_t* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const uint64_t A = (uint64_t)newid[labels[v]];
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) {
      const uint64_t B = (uint64_t)newid[labels[cols[e]]];
      keys[e] = (A << bits) | B;
      vals[e] = W::get(w, e);
    }
  }
}

// Heads of runs: the coarse column, the row count, and minus the weight
// prefix at the run start (the tail kernel adds the prefix at the run end).
__global__ void k_agg_heads(const uint64_t* __restrict__ keys, const int64_t* __restrict__ hx,
                            const int64_t* __restrict__ pre, int64_t m, int bits,
                            int32_t* __restrict__ ccols, int64_t* __restrict__ cw,
                            unsigned long long* rowcnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint64_t mask = bits ? ((1ull << bits) - 1ull) : 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    if (i > 0 && keys[i] == keys[i - 1]) continue;
    const int64_t seg = hx[i];
    ccols[seg] = (int32_t)(keys[i] & mask);
    cw[seg] = -pre[i];
    atomicAdd(&rowcnt[keys[i] >> bits], 1ull);
  }
}

__global__ void k_agg_tails(const uint64_t* __restrict__ keys, const int64_t* __restrict__ hx,
                            const int64_t* __restrict__ pre, const int64_t* __restrict__ vals,
                            int64_t m, int64_t* __restrict__ cw) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    if (i + 1 < m && keys[i + 1] == keys[i]) continue;
    const int64_t head = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
    const int64_t seg = hx[i] + head - 1;
    cw[seg] += pre[i] + vals[i];
  }
}

__global__ void k_compose(int32_t* labels0, int64_t n0, const int32_t* __restrict__ C,
                          const int32_t* __restrict__ newid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += stride)
    labels0[v] = newid[C[labels0[v]]];
}

__global__ void k_iota(int32_t* a, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    a[v] = (int32_t)v;
}

// ------------------------------------------------------------------ modularity

__global__ void k_mod_vol(const int32_t* __restrict__ labels, const int64_t* __restrict__ degw,
                          int64_t n, unsigned long long* volc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    atomicAdd(&volc[labels[v]], (unsigned long long)degw[v]);
}

// acc[0..1]: 128-bit unsigned accumulator (low, high) for sum vol(c)^2;
// acc[2]: I, the weight of arcs inside communities.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* acc, unsigned __int128 x) {
  const unsigned long long lo = (unsigned long long)x, hi = (unsigned long long)(x >> 64);
  const unsigned long long old = atomicAdd(&acc[0], lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(&acc[1], hi + carry);
}

__global__ void __launch_bounds__(NT) k_mod_sq(const unsigned long long* __restrict__ volc,
                                               int64_t n, unsigned long long* acc) {
  __shared__ unsigned __int128 part[NT];
  unsigned __int128 s = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const unsigned long long x = volc[c];
    s += (unsigned __int128)x * x;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && part[0]) atomic_add_u128(acc, part[0]);
}

template <class W>
__global__ void __launch_bounds__(NT) k_mod_internal(const int64_t* __restrict__ off,
                                                     const int32_t* __restrict__ cols, const void* w,
                                                     int64_t n, const int32_t* __restrict__ labels,
                                                     unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  int64_t s = 0;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t a = labels[v];
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
      if (labels[cols[e]] == a) s += W::get(w, e);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if (lane == 0 && s) atomicAdd(&acc[2], (unsigned long long)s);
}

int ceil_log2_host(int64_t x) {
  int b = 0;
  while (((int64_t)1 << b) < x) ++b;
  return b;
}

}  // namespace

int renumber(cd_graph* g, const int32_t* labels_dev, int32_t* newid_dev, int64_t* k_out) {
  cudaStream_t s = g->stream;
  const int64_t n = g->n;
  if (n == 0) {
    *k_out = 0;
    return CD_OK;
  }
  uint8_t* used = nullptr;
  int64_t* total = nullptr;
  int rc = dev_alloc_t(&used, n, s);
  if (!rc) rc = dev_alloc_t(&total, 1, s);
  if (rc) {
    dev_free(used, s);
    return rc;
  }
  {
    KTimer t(g, K_RENUMBER, (double)n * (4 + 1 + 1 + 4 + 1));
    CD_CHECK(cudaMemsetAsync(used, 0, n, s));
    CD_LAUNCH(k_mark_used<<<grid_cap((n + NT - 1) / NT), NT, 0, s>>>(labels_dev, n, used));
    rc = exclusive_scan_u8_to_i32(used, newid_dev, n, total, s);
    if (!rc) CD_LAUNCH(k_fix_unused<<<grid_cap((n + NT - 1) / NT), NT, 0, s>>>(used, n, newid_dev));
  }
  int64_t k = 0;
  if (!rc && cudaMemcpyAsync(&k, total, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess)
    *k_out = k;
  else if (!rc)
    rc = set_cuda_error(cudaGetLastError());
  dev_free(used, s);
  dev_free(total, s);
  return rc;
}

int aggregate(cd_graph* g, const int32_t* labels_dev, const int32_t* newid_dev, int64_t k,
              cd_graph** coarse_out, int mode) {
  if (mode == 0 && g->n > 0 && k > 0) return aggregate_hash(g, labels_dev, newid_dev, k, coarse_out);
  cudaStream_t s = g->stream;
  const int64_t n = g->n, m = g->nnz;
  const int bits = ceil_log2_host(k);  // B < k fits in `bits` bits
  int rc = CD_OK;
  uint64_t *keys = nullptr, *keys2 = nullptr;
  int64_t *vals = nullptr, *vals2 = nullptr;
  int64_t *coff = nullptr, *cw = nullptr, *nseg_dev = nullptr;
  int32_t* ccols = nullptr;
  unsigned long long* rowcnt = nullptr;
  auto cleanup = [&]() {
    dev_free(keys, s);
    dev_free(keys2, s);
    dev_free(vals, s);
    dev_free(vals2, s);
    dev_free(rowcnt, s);
    dev_free(nseg_dev, s);
  };
  if ((rc = dev_alloc_t(&keys, m, s)) || (rc = dev_alloc_t(&keys2, m, s)) ||
      (rc = dev_alloc_t(&vals, m, s)) || (rc = dev_alloc_t(&vals2, m, s)) ||
      (rc = dev_alloc_t(&rowcnt, k, s)) || (rc = dev_alloc_t(&nseg_dev, 1, s))) {
    cleanup();
    return rc;
  }
  const int wbytes = g->wkind == W_UNIT ? 0 : g->wkind == W_I32 ? 4 : 8;
  if (m > 0) {
    KTimer t(g, K_AGG_EMIT, (double)n * (8 + 4 + 4) + (double)m * (4 + 4 + 4 + wbytes + 16));
    const unsigned gr = grid_cap(n * 32 / NT + 1);
    if (g->wkind == W_UNIT)
      CD_LAUNCH(k_agg_emit<WUnit><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, labels_dev, newid_dev, bits, keys, vals));
    else if (g->wkind == W_I32)
      CD_LAUNCH(k_agg_emit<WI32><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, labels_dev, newid_dev, bits, keys, vals));
    else
      CD_LAUNCH(k_agg_emit<WI64><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, labels_dev, newid_dev, bits, keys, vals));
  }
  uint64_t* sk = keys;
  int64_t* sv = vals;
  {
    KTimer t(g, K_SORT, (double)m * 32 * ((2 * bits + 7) / 8));
    rc = radix_sort_pairs(keys, vals, keys2, vals2, m, 2 * bits, s, &sk, &sv);
  }
  if (rc) {
    cleanup();
    return rc;
  }
  // the other pair of buffers is free again: reuse it for the two scans
  int64_t* hx = (int64_t*)(sk == keys ? keys2 : keys);
  int64_t* pre = sv == vals ? vals2 : vals;
  int64_t nseg = 0;
  {
    KTimer t(g, K_AGG_REDUCE, (double)m * (8 * 3 + 8 * 3) + (double)k * 16);
    rc = exclusive_scan_head(sk, hx, m, nseg_dev, s);
    if (!rc) rc = exclusive_scan_i64(sv, pre, m, nullptr, s);
    if (!rc && cudaMemcpyAsync(&nseg, nseg_dev, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = CD_ECUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = CD_ECUDA;
    if (!rc) rc = dev_alloc_t(&coff, k + 1, s);
    if (!rc) rc = dev_alloc_t(&ccols, nseg + COL_PAD, s);
    if (!rc && cudaMemsetAsync(ccols + nseg, 0, COL_PAD * sizeof(int32_t), s) != cudaSuccess) rc = CD_ECUDA;
    if (!rc) rc = dev_alloc_t(&cw, nseg, s);
    if (!rc) {
      cudaMemsetAsync(rowcnt, 0, k * sizeof(unsigned long long), s);
      if (m > 0) {
        CD_LAUNCH(k_agg_heads<<<grid_cap((m + NT - 1) / NT), NT, 0, s>>>(sk, hx, pre, m, bits, ccols, cw, rowcnt));
        CD_LAUNCH(k_agg_tails<<<grid_cap((m + NT - 1) / NT), NT, 0, s>>>(sk, hx, pre, sv, m, cw));
      }
      // offsets = exclusive scan of the row counts
      rc = exclusive_scan_i64((const int64_t*)rowcnt, coff, k, nseg_dev, s);
      if (!rc) cudaMemcpyAsync(coff + k, nseg_dev, 8, cudaMemcpyDeviceToDevice, s);
      if (cudaGetLastError() != cudaSuccess) rc = CD_ECUDA;
    }
  }
  cleanup();
  if (rc) {
    dev_free(coff, s);
    dev_free(ccols, s);
    dev_free(cw, s);
    return rc;
  }
  cd_graph* c = nullptr;
  rc = graph_adopt(s, k, nseg, coff, ccols, cw, W_I64, &c, nullptr, nullptr, g);
  if (rc) return rc;
  c->timing = g->timing;
  c->ktiming = g->ktiming;
  c->cols_distinct = true;  // one arc per pair of communities
  *coarse_out = c;
  return CD_OK;
}

int modularity(cd_graph* g, const int32_t* labels_dev, double* q_out) {
  cudaStream_t s = g->stream;
  const int64_t n = g->n;
  if (g->vol == 0) {
    *q_out = 0.0;
    return CD_OK;
  }
  unsigned long long *volc = nullptr, *acc = nullptr;
  int rc = dev_alloc_t(&volc, n, s);
  if (!rc) rc = dev_alloc_t(&acc, 3, s);
  if (rc) {
    dev_free(volc, s);
    return rc;
  }
  {
    const int wbytes = g->wkind == W_UNIT ? 0 : g->wkind == W_I32 ? 4 : 8;
    KTimer t(g, K_MODULARITY, (double)n * (8 + 4 + 4 + 8 + 8 + 8) + (double)g->nnz * (4 + 4 + wbytes));
    cudaMemsetAsync(volc, 0, n * 8, s);
    cudaMemsetAsync(acc, 0, 3 * 8, s);
    CD_LAUNCH(k_mod_vol<<<grid_cap((n + NT - 1) / NT), NT, 0, s>>>(labels_dev, g->degw, n, volc));
    CD_LAUNCH(k_mod_sq<<<grid_cap((n + NT - 1) / NT, 152 * 4), NT, 0, s>>>(volc, n, acc));
    const unsigned gr = grid_cap(n * 32 / NT + 1);
    if (g->wkind == W_UNIT)
      CD_LAUNCH(k_mod_internal<WUnit><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, labels_dev, acc));
    else if (g->wkind == W_I32)
      CD_LAUNCH(k_mod_internal<WI32><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, labels_dev, acc));
    else
      CD_LAUNCH(k_mod_internal<WI64><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, labels_dev, acc));
  }
  unsigned long long h[3] = {0, 0, 0};
  CD_CHECK(cudaGetLastError());
  CD_CHECK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  CD_CHECK(cudaStreamSynchronize(s));
  dev_free(volc, s);
  dev_free(acc, s);
  const unsigned __int128 S = ((unsigned __int128)h[1] << 64) | h[0];
  const i128 num = (i128)(int64_t)h[2] * g->vol - (i128)S;
  const i128 den = (i128)g->vol * g->vol;
  *q_out = (double)num / (double)den;
  return CD_OK;
}

}  // namespace cd

using namespace cd;

namespace {

int stage_labels(cd_graph* g, const int32_t* labels, int on_device, int32_t** dev, bool* owned) {
  *owned = false;
  if (on_device) {
    *dev = const_cast<int32_t*>(labels);
    return CD_OK;
  }
  int rc = dev_alloc_t(dev, g->n, g->stream);
  if (rc) return rc;
  *owned = true;
  if (g->n > 0)
    CD_CHECK(cudaMemcpyAsync(*dev, labels, g->n * 4, cudaMemcpyHostToDevice, g->stream));
  return CD_OK;
}

void merge_stats(cd_graph* into, const cd_graph* from) {
  into->trace.insert(into->trace.end(), from->trace.begin(), from->trace.end());
  for (int k = 0; k < K_COUNT; ++k) {
    into->prof[k].launches += from->prof[k].launches;
    into->prof[k].total_ms += from->prof[k].total_ms;
    into->prof[k].alg_bytes += from->prof[k].alg_bytes;
  }
}

}  // namespace

extern "C" {

int cd_modularity(cd_graph* g, const int32_t* labels, int on_device, double* q_out) {
  if (!g || !q_out || (!labels && g->n > 0)) return CD_EINVAL;
  int32_t* d = nullptr;
  bool owned = false;
  int rc = stage_labels(g, labels, on_device, &d, &owned);
  if (!rc) rc = check_labels(g, d);
  if (!rc) rc = modularity(g, d, q_out);
  if (owned) dev_free(d, g->stream);
  if (!rc) rc = profile_flush(g);
  return rc;
}

int cd_louvain_aggregate(cd_graph* g, const int32_t* labels, int on_device, cd_graph** coarse_out,
                         int32_t* newid_out, int64_t* k_out) {
  if (!g || !coarse_out || (!labels && g->n > 0)) return CD_EINVAL;
  *coarse_out = nullptr;
  int32_t* d = nullptr;
  int32_t* newid = nullptr;
  bool owned = false;
  int64_t k = 0;
  int rc = stage_labels(g, labels, on_device, &d, &owned);
  if (!rc) rc = check_labels(g, d);
  if (!rc) rc = dev_alloc_t(&newid, g->n, g->stream);
  if (!rc) rc = renumber(g, d, newid, &k);
  if (!rc) rc = aggregate(g, d, newid, k, coarse_out);
  if (!rc && newid_out && g->n > 0)
    if (cudaMemcpyAsync(newid_out, newid, g->n * 4,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        g->stream) != cudaSuccess)
      rc = CD_ECUDA;
  if (!rc && k_out) *k_out = k;
  dev_free(newid, g->stream);
  if (owned) dev_free(d, g->stream);
  if (cudaStreamSynchronize(g->stream) != cudaSuccess && !rc) rc = CD_ECUDA;
  if (!rc) rc = profile_flush(g);
  return rc;
}

int cd_louvain_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
                   int32_t* levels_out, double* q_out) {
  int rc = begin_run(g, p);
  if (rc) return rc;
  if (!labels_out && g->n > 0) return CD_EINVAL;
  cudaStream_t s = g->stream;
  const int64_t n0 = g->n;
  int32_t* labels0 = nullptr;
  if ((rc = dev_alloc_t(&labels0, n0, s))) return rc;
  if (n0 > 0) CD_LAUNCH(k_iota<<<grid_cap((n0 + NT - 1) / NT), NT, 0, s>>>(labels0, n0));
  cd_graph* cur = g;
  int32_t levels = 0;
  int32_t* newid = nullptr;
  bool settled = false;  // the last level ended with every vertex of `cur` in its own community
  for (int32_t lvl = 0; lvl < p->max_levels && !rc; ++lvl) {
    rc = run_local_move(cur, opts_from(p, lvl), 0, nullptr, nullptr);
    if (rc) break;
    int64_t k = 0;
    if ((rc = dev_alloc_t(&newid, cur->n, s))) break;
    if ((rc = renumber(cur, cur->C, newid, &k))) break;
    if (n0 > 0) CD_LAUNCH(k_compose<<<grid_cap((n0 + NT - 1) / NT), NT, 0, s>>>(labels0, n0, cur->C, newid));
    levels = lvl + 1;
    if (k == cur->n) {  // done: every vertex is its own community
      settled = true;
      break;
    }
    cd_graph* coarse = nullptr;
    rc = aggregate(cur, cur->C, newid, k, &coarse, p->aggregation);
    dev_free(newid, s);
    newid = nullptr;
    if (rc) break;
    if (cur != g) {
      profile_flush(cur);
      merge_stats(g, cur);
      cd_graph_free(cur);
    }
    cur = coarse;
  }
  dev_free(newid, s);
  // Q of the input partition equals Q of the last graph under its final
  // partition: aggregation keeps every community's volume and internal
  // weight exactly (integers), so the same quotient follows from a far
  // smaller graph. That partition is the last local move's if the run settled
  // there, else (max_levels reached after an aggregation) the coarse
  // vertices themselves.
  double q = 0.0;
  if (!rc) {
    if (settled) {
      rc = modularity(cur, cur->C, &q);
    } else {
      int32_t* ident = nullptr;
      if (!(rc = dev_alloc_t(&ident, cur->n, s))) {
        if (cur->n > 0) CD_LAUNCH(k_iota<<<grid_cap((cur->n + NT - 1) / NT), NT, 0, s>>>(ident, cur->n));
        rc = modularity(cur, ident, &q);
        dev_free(ident, s);
      }
    }
  }
  if (cur != g) {
    profile_flush(cur);
    merge_stats(g, cur);
    cd_graph_free(cur);
  }
  if (!rc && n0 > 0)
    if (cudaMemcpyAsync(labels_out, labels0, n0 * 4,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = CD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = CD_ECUDA;
  dev_free(labels0, s);
  if (!rc) rc = profile_flush(g);
  if (!rc) {
    if (levels_out) *levels_out = levels;
    if (q_out) *q_out = q;
  }
  return rc;
}

}  // extern "C"
