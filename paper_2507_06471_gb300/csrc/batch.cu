// Batched mode: many independent graphs packed block-diagonally into one CSR
// and solved by the same kernels, one launch per kernel and round for all of
// them. Every graph's result is the one a solo run of that graph gives:
//   - gains use the graph's own vol(V), the coin draws with graph-local ids;
//   - LPA freezes a graph after its own round with dN <= threshold;
//   - Louvain runs the levels in lockstep; a graph whose level left every
//     vertex in its own community (Algorithm 3's done test) is frozen for the
//     remaining levels; the coarse graph of all graphs is the union of their
//     coarse graphs, because communities never span two graphs;
//   - modularity (Sec. II-C) is reported per graph.
#include <algorithm>

#include "common.cuh"

namespace cd {
namespace {

constexpr int NT = 256;

unsigned grid_cap(int64_t blocks, int64_t cap = 152 * 16) {
  if (blocks < 1) blocks = 1;
  return (unsigned)(blocks < cap ? blocks : cap);
}

__global__ void k_batch_gid(const int64_t* __restrict__ gbase, int64_t nb, int64_t n, int32_t* gid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    int64_t lo = 0, hi = nb;  // last b with gbase[b] <= v
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (gbase[mid] <= v) lo = mid; else hi = mid;
    }
    gid[v] = (int32_t)lo;
  }
}

// Warp per vertex: every arc must stay inside the vertex's graph.
__global__ void __launch_bounds__(NT) k_batch_check(const int64_t* __restrict__ off,
                                                    const int32_t* __restrict__ cols,
                                                    const int32_t* __restrict__ gid, int64_t n,
                                                    int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t b = gid[v];
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
      if (gid[cols[e]] != b) atomicCAS(status, 0, CD_EINVAL);
  }
}

__global__ void k_batch_vol(const int64_t* __restrict__ degw, const int32_t* __restrict__ gid, int64_t n,
                            unsigned long long* gvol) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    atomicAdd(&gvol[gid[v]], (unsigned long long)degw[v]);
}

// graph of each coarse vertex: the graph of any member of the community
__global__ void k_batch_coarse_gid(const int32_t* __restrict__ C, const int32_t* __restrict__ newid,
                                   const int32_t* __restrict__ gid, int64_t n, int32_t* gid_c) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    gid_c[newid[C[v]]] = gid[v];
}

// communities per graph (a used community id c is a vertex of c's graph)
__global__ void k_batch_kcount(const int32_t* __restrict__ newid, const int32_t* __restrict__ gid, int64_t n,
                               unsigned long long* kcnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride)
    if (newid[c] >= 0) atomicAdd(&kcnt[gid[c]], 1ull);
}

// out[v] = lab[v] - base[gid[v]]: labels local to each graph
__global__ void k_batch_localize(const int32_t* __restrict__ lab, const int32_t* __restrict__ gid,
                                 const int64_t* __restrict__ base, int64_t n, int32_t* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    out[v] = (int32_t)(lab[v] - base[gid[v]]);
}

__global__ void k_iota32(int32_t* a, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) a[v] = (int32_t)v;
}

__global__ void k_compose32(int32_t* labels0, int64_t n0, const int32_t* __restrict__ C,
                            const int32_t* __restrict__ newid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += stride)
    labels0[v] = newid[C[labels0[v]]];
}

// ---- per-graph modularity: I_b, S_b = sum over b's communities of vol(c)^2

__global__ void k_bmod_vol(const int32_t* __restrict__ lab, const int64_t* __restrict__ degw,
                           const int32_t* __restrict__ gid, int64_t n, unsigned long long* volc,
                           int32_t* cgid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    atomicAdd(&volc[lab[v]], (unsigned long long)degw[v]);
    cgid[lab[v]] = gid[v];
  }
}

__global__ void k_bmod_sq(const unsigned long long* __restrict__ volc, const int32_t* __restrict__ cgid,
                          int64_t n, unsigned long long* S) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const unsigned long long x = volc[c];
    if (!x) continue;
    const unsigned __int128 sq = (unsigned __int128)x * x;
    const unsigned long long lo = (unsigned long long)sq, hi = (unsigned long long)(sq >> 64);
    unsigned long long* acc = S + 2 * cgid[c];
    const unsigned long long old = atomicAdd(&acc[0], lo);
    const unsigned long long carry = old + lo < old ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&acc[1], hi + carry);
  }
}

template <class W>
__global__ void __launch_bounds__(NT) k_bmod_internal(const int64_t* __restrict__ off,
                                                      const int32_t* __restrict__ cols, const void* w,
                                                      int64_t n, const int32_t* __restrict__ lab,
                                                      const int32_t* __restrict__ gid,
                                                      unsigned long long* I) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t a = lab[v];
    int64_t s = 0;
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
      if (lab[cols[e]] == a) s += W::get(w, e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0 && s) atomicAdd(&I[gid[v]], (unsigned long long)s);
  }
}

void free_batches(cd_graph* g) {
  dev_free(g->gid, g->stream);
  dev_free(g->gbase, g->stream);
  dev_free(g->gvol, g->stream);
  dev_free(g->gfrozen, g->stream);
  dev_free(g->gcnt, g->stream);
  g->gid = nullptr;
  g->gbase = g->gvol = g->gcnt = nullptr;
  g->gfrozen = nullptr;
  g->nb = 0;
  g->h_gbase.clear();
}

// Attach a partition into nb graphs (gbase on the host). gid_dev, if given,
// is copied (and trusted); else derived from gbase and every arc is checked
// to stay in its block. gvol_dev, if given, is copied; else summed from deg_w.
int set_batches(cd_graph* g, const std::vector<int64_t>& gbase, const int32_t* gid_dev,
                const int64_t* gvol_dev) {
  cudaStream_t s = g->stream;
  const int64_t nb = (int64_t)gbase.size() - 1;
  free_batches(g);
  int rc;
  if ((rc = dev_alloc_t(&g->gid, g->n, s)) || (rc = dev_alloc_t(&g->gbase, nb + 1, s)) ||
      (rc = dev_alloc_t(&g->gvol, nb, s)) || (rc = dev_alloc_t(&g->gfrozen, nb, s)) ||
      (rc = dev_alloc_t(&g->gcnt, nb, s)))
    return rc;
  g->nb = nb;
  g->h_gbase = gbase;
  CD_CHECK(cudaMemcpyAsync(g->gbase, gbase.data(), (nb + 1) * 8, cudaMemcpyHostToDevice, s));
  CD_CHECK(cudaMemsetAsync(g->gfrozen, 0, nb, s));
  if (g->n > 0) {
    if (gid_dev) {
      CD_CHECK(cudaMemcpyAsync(g->gid, gid_dev, g->n * 4, cudaMemcpyDeviceToDevice, s));
    } else {
      CD_LAUNCH(k_batch_gid<<<grid_cap((g->n + NT - 1) / NT), NT, 0, s>>>(g->gbase, nb, g->n, g->gid));
      CD_LAUNCH(k_batch_check<<<grid_cap(g->n * 32 / NT + 1), NT, 0, s>>>(g->off, g->cols, g->gid, g->n,
                                                                          g->status));
    }
  }
  if (gvol_dev) {
    CD_CHECK(cudaMemcpyAsync(g->gvol, gvol_dev, nb * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    CD_CHECK(cudaMemsetAsync(g->gvol, 0, nb * 8, s));
    if (g->n > 0)
      CD_LAUNCH(k_batch_vol<<<grid_cap((g->n + NT - 1) / NT), NT, 0, s>>>(g->degw, g->gid, g->n,
                                                                         (unsigned long long*)g->gvol));
  }
  CD_CHECK(cudaGetLastError());
  int32_t st = 0;
  CD_CHECK(cudaMemcpyAsync(&st, g->status, 4, cudaMemcpyDeviceToHost, s));
  CD_CHECK(cudaStreamSynchronize(s));
  if (st) {
    CD_CHECK(cudaMemsetAsync(g->status, 0, 4, s));
    free_batches(g);
    return st;
  }
  return CD_OK;
}

// Per-graph modularity of global labels `lab` (values in [0, n)).
int batch_modularity(cd_graph* g, const int32_t* lab, std::vector<double>& q) {
  cudaStream_t s = g->stream;
  const int64_t n = g->n, nb = g->nb;
  unsigned long long *volc = nullptr, *S = nullptr, *I = nullptr;
  int32_t* cgid = nullptr;
  int rc;
  if ((rc = dev_alloc_t(&volc, n, s)) || (rc = dev_alloc_t(&cgid, n, s)) || (rc = dev_alloc_t(&S, 2 * nb, s)) ||
      (rc = dev_alloc_t(&I, nb, s)))
    return rc;
  {
    const int wbytes = g->wkind == W_UNIT ? 0 : g->wkind == W_I32 ? 4 : 8;
    KTimer t(g, K_MODULARITY, (double)n * 40 + (double)g->nnz * (8 + wbytes));
    CD_CHECK(cudaMemsetAsync(volc, 0, n * 8, s));
    CD_CHECK(cudaMemsetAsync(S, 0, 2 * nb * 8, s));
    CD_CHECK(cudaMemsetAsync(I, 0, nb * 8, s));
    if (n > 0) {
      CD_LAUNCH(k_bmod_vol<<<grid_cap((n + NT - 1) / NT), NT, 0, s>>>(lab, g->degw, g->gid, n, volc, cgid));
      CD_LAUNCH(k_bmod_sq<<<grid_cap((n + NT - 1) / NT), NT, 0, s>>>(volc, cgid, n, S));
      const unsigned gr = grid_cap(n * 32 / NT + 1);
      if (g->wkind == W_UNIT)
        CD_LAUNCH(k_bmod_internal<WUnit><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, lab, g->gid, I));
      else if (g->wkind == W_I32)
        CD_LAUNCH(k_bmod_internal<WI32><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, lab, g->gid, I));
      else
        CD_LAUNCH(k_bmod_internal<WI64><<<gr, NT, 0, s>>>(g->off, g->cols, g->w, n, lab, g->gid, I));
    }
  }
  std::vector<unsigned long long> hS(2 * nb), hI(nb);
  std::vector<int64_t> hvol(nb);
  CD_CHECK(cudaGetLastError());
  CD_CHECK(cudaMemcpyAsync(hS.data(), S, 2 * nb * 8, cudaMemcpyDeviceToHost, s));
  CD_CHECK(cudaMemcpyAsync(hI.data(), I, nb * 8, cudaMemcpyDeviceToHost, s));
  CD_CHECK(cudaMemcpyAsync(hvol.data(), g->gvol, nb * 8, cudaMemcpyDeviceToHost, s));
  CD_CHECK(cudaStreamSynchronize(s));
  dev_free(volc, s);
  dev_free(cgid, s);
  dev_free(S, s);
  dev_free(I, s);
  q.assign(nb, 0.0);
  for (int64_t b = 0; b < nb; ++b) {
    if (hvol[b] == 0) continue;
    const unsigned __int128 Sb = ((unsigned __int128)hS[2 * b + 1] << 64) | hS[2 * b];
    const i128 num = (i128)(int64_t)hI[b] * hvol[b] - (i128)Sb;
    const i128 den = (i128)hvol[b] * hvol[b];
    q[b] = (double)num / (double)den;
  }
  return CD_OK;
}

void merge_into(cd_graph* into, cd_graph* from) {
  profile_flush(from);
  into->trace.insert(into->trace.end(), from->trace.begin(), from->trace.end());
  for (int k = 0; k < K_COUNT; ++k) {
    into->prof[k].launches += from->prof[k].launches;
    into->prof[k].total_ms += from->prof[k].total_ms;
    into->prof[k].alg_bytes += from->prof[k].alg_bytes;
  }
}

int copy_out(cudaStream_t s, void* dst, const void* src, size_t bytes, int on_device) {
  if (bytes == 0) return CD_OK;
  CD_CHECK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return CD_OK;
}

}  // namespace

void release_batches(cd_graph* g) { free_batches(g); }

}  // namespace cd

using namespace cd;

extern "C" {

int cd_graph_set_batches(cd_graph* g, const int64_t* vstart, int64_t n_graphs, int on_device) {
  if (!g || !vstart || n_graphs < 1 || n_graphs > INT32_MAX) return CD_EINVAL;
  std::vector<int64_t> gb(n_graphs + 1);
  if (on_device) {
    CD_CHECK(cudaMemcpyAsync(gb.data(), vstart, (n_graphs + 1) * 8, cudaMemcpyDeviceToHost, g->stream));
    CD_CHECK(cudaStreamSynchronize(g->stream));
  } else {
    std::copy(vstart, vstart + n_graphs + 1, gb.begin());
  }
  if (gb[0] != 0 || gb[n_graphs] != g->n) return CD_EINVAL;
  for (int64_t b = 0; b < n_graphs; ++b)
    if (gb[b + 1] < gb[b]) return CD_EINVAL;
  return set_batches(g, gb, nullptr, nullptr);
}

int cd_batch_lpa_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
                     int32_t* rounds_out) {
  int rc = begin_run(g, p);
  if (rc) return rc;
  if (g->nb == 0 || (!labels_out && g->n > 0)) return CD_EINVAL;
  std::vector<int32_t> rounds;
  RunOpts o = opts_from(p, 0);
  o.batched = true;
  if ((rc = run_lpa_batched(g, o, rounds))) return rc;
  int32_t* loc = nullptr;
  if ((rc = dev_alloc_t(&loc, g->n, g->stream))) return rc;
  if (g->n > 0)
    CD_LAUNCH(k_batch_localize<<<grid_cap((g->n + NT - 1) / NT), NT, 0, g->stream>>>(g->C, g->gid, g->gbase,
                                                                                    g->n, loc));
  rc = copy_out(g->stream, labels_out, loc, g->n * 4, on_device);
  dev_free(loc, g->stream);
  CD_CHECK(cudaStreamSynchronize(g->stream));
  if (rc) return rc;
  if (rounds_out) std::copy(rounds.begin(), rounds.end(), rounds_out);
  return CD_OK;
}

int cd_batch_louvain_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
                         int32_t* levels_out, double* q_out) {
  int rc = begin_run(g, p);
  if (rc) return rc;
  if (g->nb == 0 || (!labels_out && g->n > 0)) return CD_EINVAL;
  cudaStream_t s = g->stream;
  const int64_t n0 = g->n, nb = g->nb;
  int32_t *labels0 = nullptr, *newid = nullptr, *gid_c = nullptr;
  unsigned long long* kcnt = nullptr;
  if ((rc = dev_alloc_t(&labels0, n0, s)) || (rc = dev_alloc_t(&kcnt, nb, s))) return rc;
  if (n0 > 0) CD_LAUNCH(k_iota32<<<grid_cap((n0 + NT - 1) / NT), NT, 0, s>>>(labels0, n0));
  std::vector<uint8_t> done(nb, 0);
  std::vector<int32_t> levels(nb, 0);
  bool emitted = false;
  std::vector<unsigned long long> hk(nb);
  cd_graph* cur = g;
  for (int32_t lvl = 0; lvl < p->max_levels && !rc; ++lvl) {
    CD_CHECK(cudaMemcpyAsync(cur->gfrozen, done.data(), nb, cudaMemcpyHostToDevice, s));
    RunOpts o = opts_from(p, lvl);
    o.batched = true;
    if ((rc = run_local_move(cur, o, 0, nullptr, nullptr))) break;
    int64_t k = 0;
    if ((rc = dev_alloc_t(&newid, cur->n, s))) break;
    if ((rc = renumber(cur, cur->C, newid, &k))) break;
    if (n0 > 0) CD_LAUNCH(k_compose32<<<grid_cap((n0 + NT - 1) / NT), NT, 0, s>>>(labels0, n0, cur->C, newid));
    CD_CHECK(cudaMemsetAsync(kcnt, 0, nb * 8, s));
    if (cur->n > 0)
      CD_LAUNCH(k_batch_kcount<<<grid_cap((cur->n + NT - 1) / NT), NT, 0, s>>>(newid, cur->gid, cur->n, kcnt));
    CD_CHECK(cudaMemcpyAsync(hk.data(), kcnt, nb * 8, cudaMemcpyDeviceToHost, s));
    CD_CHECK(cudaStreamSynchronize(s));
    bool all = true;
    std::vector<int64_t> gbase_c(nb + 1, 0);
    for (int64_t b = 0; b < nb; ++b) {
      if (!done[b]) {
        levels[b] = lvl + 1;
        if ((int64_t)hk[b] == cur->h_gbase[b + 1] - cur->h_gbase[b]) done[b] = 1;  // no merge: done
      }
      all = all && done[b];
      gbase_c[b + 1] = gbase_c[b] + (int64_t)hk[b];
    }
    if (all || lvl + 1 == p->max_levels) {
      // final labels are ids of the renumbered communities: make them local
      int64_t* cb = nullptr;
      if ((rc = dev_alloc_t(&cb, nb + 1, s))) break;
      CD_CHECK(cudaMemcpyAsync(cb, gbase_c.data(), (nb + 1) * 8, cudaMemcpyHostToDevice, s));
      int32_t* loc = nullptr;
      if ((rc = dev_alloc_t(&loc, n0, s))) break;
      if (n0 > 0)
        CD_LAUNCH(k_batch_localize<<<grid_cap((n0 + NT - 1) / NT), NT, 0, s>>>(labels0, g->gid, cb, n0, loc));
      rc = copy_out(s, labels_out, loc, n0 * 4, on_device);
      CD_CHECK(cudaStreamSynchronize(s));
      dev_free(loc, s);
      dev_free(cb, s);
      emitted = true;
      break;
    }
    // union of the graphs' coarse graphs, with the partition carried over
    cd_graph* coarse = nullptr;
    if ((rc = aggregate(cur, cur->C, newid, k, &coarse, p->aggregation))) break;
    if ((rc = dev_alloc_t(&gid_c, k, s))) break;
    if (cur->n > 0)
      CD_LAUNCH(k_batch_coarse_gid<<<grid_cap((cur->n + NT - 1) / NT), NT, 0, s>>>(cur->C, newid, cur->gid,
                                                                                  cur->n, gid_c));
    rc = set_batches(coarse, gbase_c, gid_c, cur->gvol);
    dev_free(gid_c, s);
    gid_c = nullptr;
    dev_free(newid, s);
    newid = nullptr;
    if (rc) {
      cd_graph_free(coarse);
      break;
    }
    if (cur != g) {
      merge_into(g, cur);
      release_batches(cur);
      cd_graph_free(cur);
    }
    cur = coarse;
  }
  dev_free(newid, s);
  if (cur != g) {
    merge_into(g, cur);
    release_batches(cur);
    cd_graph_free(cur);
  }
  if (!rc && !emitted && n0 > 0) {  // no level ran: every vertex its own community
    int32_t* loc = nullptr;
    if (!(rc = dev_alloc_t(&loc, n0, s))) {
      CD_LAUNCH(k_batch_localize<<<grid_cap((n0 + NT - 1) / NT), NT, 0, s>>>(labels0, g->gid, g->gbase, n0, loc));
      rc = copy_out(s, labels_out, loc, n0 * 4, on_device);
      if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = CD_ECUDA;
      dev_free(loc, s);
    }
  }
  std::vector<double> q;
  if (!rc) rc = batch_modularity(g, labels0, q);
  dev_free(labels0, s);
  dev_free(kcnt, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = CD_ECUDA;
  if (!rc) rc = profile_flush(g);
  if (rc) return rc;
  if (levels_out) std::copy(levels.begin(), levels.end(), levels_out);
  if (q_out) std::copy(q.begin(), q.end(), q_out);
  return CD_OK;
}

}  // extern "C"
