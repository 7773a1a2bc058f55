// The neighbour-community scan and the synchronous round loops of
// Label Propagation (Algorithm 1, PLPMove) and Louvain local moving
// (Algorithm 2, gain of Eq. deltaQ).
//
// Per examined vertex v the scan accumulates, for every community c among v's
// neighbours (loops excluded), k_{v,c} = sum of w(v,u) over u in N(v) with
// C[u] = c, and picks
//   LPA:     the c of largest k_{v,c}; the current label is kept if it
//            attains the maximum (tie_keep_current), else the smallest c;
//   Louvain: the c != A = C[v] of largest g(c) = vol(V) k_{v,c} - deg_w(v)
//            Sigma_tot[c] (smallest c on ties) and moves iff
//            G = g(c) - vol(V) k_{v,A} + deg_w(v) (Sigma_tot[A] - deg_w(v)) > 0,
//            where G = dQ_{v->c} vol(V)^2 / 2 (Eq. deltaQ, exact in 128 bits).
// A vertex whose decision differs from its label commits only if the pinned
// SplitMix64 coin says so; otherwise it defers and stays active.
//
// Degree bins (per graph, thresholds t_warp <= t_hub, defaults 256 and
// 1024): degrees 1-4/5-8/9-16/17-32 use TILE lanes per vertex and group equal
// labels with __match_any_sync; 33..t_warp a warp with a shared-memory
// open-addressing table; up to t_hub 128 threads (degree <= 1024) or a whole
// 512-thread CTA (<= 4096) with a shared-memory table;
// larger degrees (hubs) keep persistent label histograms in global memory,
// updated by their neighbours' moves, and many CTAs evaluate slices of a
// hub's histogram with the last one deciding.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace cd {
namespace {

constexpr int NT = 256;  // threads of the tile and hub-evaluate kernels
constexpr int NW = NT / 32;
constexpr int WARP_CAP_SLOTS = 2 * WARP_MAX;   // table slots per warp-bin vertex
constexpr int BLK1_CAP_SLOTS = 2 * BLK1_MAX;   // per 128-thread group
constexpr int BLK4_CAP_SLOTS = 2 * BLK4_MAX;   // per 512-thread CTA

// ------------------------------------------------------------------ coin

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): draw number ctr of the
// stream with state `seed`; the move commits iff bit 63 is set.
__device__ __forceinline__ bool commit_coin(uint64_t seed, int level, int round, int32_t v) {
  uint64_t ctr = ((uint64_t)(uint32_t)level << 48) | ((uint64_t)(uint32_t)round << 32) | (uint32_t)v;
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (z >> 63) != 0;
}

// ------------------------------------------------------------------ keys

template <bool LOUV, bool NK> struct KeyOf { typedef int64_t T; };
template <> struct KeyOf<true, false> { typedef i128 T; };

__device__ __forceinline__ int64_t shfl_xor_key(int64_t x, int o) {
  return __shfl_xor_sync(FULL, (long long)x, o);
}
__device__ __forceinline__ i128 shfl_xor_key(i128 x, int o) {
  unsigned long long lo = (unsigned long long)x, hi = (unsigned long long)(x >> 64);
  lo = __shfl_xor_sync(FULL, lo, o);
  hi = __shfl_xor_sync(FULL, hi, o);
  return (i128)(((unsigned __int128)hi << 64) | lo);
}

// Is candidate (k1, c1) preferred over (k0, c0)? Larger key, then smaller id.
template <class K>
__device__ __forceinline__ bool better(K k1, int32_t c1, K k0, int32_t c0) {
  if (c1 == NOCAND) return false;
  if (c0 == NOCAND) return true;
  return k1 > k0 || (k1 == k0 && c1 < c0);
}

template <class K>
__device__ __forceinline__ void reduce_best(K& k, int32_t& c, int width) {
  for (int o = width / 2; o > 0; o >>= 1) {
    K ok = shfl_xor_key(k, o);
    int32_t oc = __shfl_xor_sync(FULL, c, o);
    if (better(ok, oc, k, c)) {
      k = ok;
      c = oc;
    }
  }
}

struct ScanCtx {
  const int64_t* off;
  const int32_t* cols;
  const void* w;
  const int64_t* degw;
  int64_t vol;
  const int32_t* C;
  const int64_t* sigma;
  const uint32_t* sigma32;  // 32-bit copy of sigma for the gathers (vol(V) < 2^31, synchronous), or null
  const int32_t* csize;
  const uint32_t* flag_cur;  // bitmaps of n bits: examined this round / next round
  uint32_t* flag_nxt;
  int all_active;
  int mark;  // maintain the next-round flags (frontier on)
  int32_t* mv_v;
  int32_t* mv_c;
  unsigned long long* ctr;
  int32_t* status;
  uint64_t seed;
  int level, round, tie_keep, singleton_rule;
  int32_t* mv_a;
  // hubs
  const int32_t* hub_list;
  const uint32_t* hub_pref;
  const uint32_t* hub_bits;
  const int64_t* hub_tab;
  int64_t* hub_cc;                   // per hub: slots in use, [0, hub_cc) of its allocation (the rest empty)
  int32_t* hub_live;                 // per hub: live entries counted by this round's evaluate items
  unsigned long long* hub_slot;
  int hub_wide;
  const int32_t* hub_item_hub;
  const int64_t* hub_item_arc;
  const int32_t* hub_ev_hub;
  const int64_t* hub_ev_slot;
  const int64_t* hub_ev_first;
  int64_t* hub_part;
  int64_t* hub_cur;
  int32_t* hub_hascur;
  int32_t* hub_done;
  int32_t* hub_mv;
  int32_t* hub_rb;                   // per hub: 1 = rebuild from its row, 2 = compact, before its next evaluation
  int32_t* hub_flist_w;              // hubs flagged this round (read back at the start of the next)
  unsigned long long* hub_fcnt_w;
  const int32_t* hub_flist_r;        // hubs flagged in the previous round
  const unsigned long long* hub_fcnt_r;
  int32_t* hub_used;                 // per hub: slots claimed since its last build
  const int64_t* hub_item_first;     // nhubs+1: first build/mark item of each hub
  int32_t* hub_blist;                // build items of the hubs being rebuilt this round
  int32_t* hub_mlist;                // mark items of the hubs that moved this round
  unsigned long long* hub_lcnt;      // [0] build items, [1] mark items
  int32_t* hub_cl;                   // 5 x nhubs: hubs rebuilt per build class (one CTA small/large, clusters of 2, 4, 8)
  unsigned long long* hub_ccnt;      // 5: their counts
  const int32_t* ev_list;            // evaluate items (of large hubs) to run this round
  const unsigned long long* ev_cnt;  // their number
  const int32_t* small_list;         // small hubs (one warp each) to evaluate this round
  const unsigned long long* small_cnt;
  const int32_t* hub_act;            // hubs examined this round (null: every hub)
  const unsigned long long* hub_act_cnt;
  int hub_upd;  // 0: neighbour moves do not update hub histograms (every hub is rebuilt next round)
  int64_t n_items, nhubs, n_ev_items;
  unsigned long long* hub_log;  // hub-histogram updates of this round, applied after the scans (null: at once)
  unsigned long long* hub_log_cnt;
  int64_t hub_log_cap;
  // asynchronous mode: a committed move is applied at once through these
  int async_mode;
  int32_t* C_w;
  int64_t* sigma_w;  // null for LPA
  int32_t* csize_w;
  // device-side round loop: the round number and the hub-update switch are
  // read from device memory (null: the host-side values above apply)
  const int32_t* round_p;
  const int32_t* hub_upd_p;
  // batched mode (gid == nullptr: one graph)
  const int32_t* gid;
  const int64_t* gbase;
  const int64_t* gvol;
  const uint8_t* gfrozen;
  unsigned long long* gcnt;
};

__device__ __forceinline__ int round_of(const ScanCtx& s) { return s.round_p ? *s.round_p : s.round; }
__device__ __forceinline__ bool hub_upd_of(const ScanCtx& s) {
  return s.hub_upd_p ? *s.hub_upd_p != 0 : s.hub_upd != 0;
}

// Flag vertex u for the next round (a bit in an L2-resident bitmap).
__device__ __forceinline__ void flag_next(const ScanCtx& s, int32_t u) {
  atomicOr(&s.flag_nxt[u >> 5], 1u << (u & 31));
}

// vol(V) of the graph v belongs to, and v's id inside that graph (the coin
// uses graph-local ids so that a batched run draws what a solo run draws).
__device__ __forceinline__ int64_t vol_of(const ScanCtx& s, int32_t v) {
  return s.gid ? s.gvol[s.gid[v]] : s.vol;
}
__device__ __forceinline__ int32_t local_id(const ScanCtx& s, int32_t v) {
  return s.gid ? v - (int32_t)s.gbase[s.gid[v]] : v;
}
// A vertex that wants to change label (moved or deferred) counts toward its
// graph's stop test.
__device__ __forceinline__ void count_change(const ScanCtx& s, int32_t v) {
  if (s.gcnt) atomicAdd(&s.gcnt[s.gid[v]], 1ull);
}

// Sigma_tot[c] for a candidate: from the 32-bit copy when there is one
// (half the bytes of the random gather).
template <bool NK>
__device__ __forceinline__ int64_t sig_of(const ScanCtx& s, int32_t c) {
  if constexpr (NK) {
    if (s.sigma32) return (int64_t)s.sigma32[c];
  }
  return s.sigma[c];
}

template <bool LOUV, bool NK>
__device__ __forceinline__ typename KeyOf<LOUV, NK>::T cand_key(const ScanCtx& s, int32_t c, int64_t k,
                                                            int64_t d, int64_t vol) {
  if constexpr (LOUV && NK)
    return vol * k - d * sig_of<NK>(s, c);  // each product < 2^62 when vol(V) < 2^31
  else if constexpr (LOUV)
    return (i128)vol * k - (i128)d * s.sigma[c];
  else
    return k;
}

// The same key with Sigma_tot[c] already loaded.
template <bool LOUV, bool NK>
__device__ __forceinline__ typename KeyOf<LOUV, NK>::T cand_key_sg(int64_t sig, int64_t k, int64_t d, int64_t vol) {
  if constexpr (LOUV && NK)
    return vol * k - d * sig;
  else if constexpr (LOUV)
    return (i128)vol * k - (i128)d * sig;
  else
    return k;
}

// Final decision of vertex v from the best candidate.
template <bool LOUV, bool NK>
__device__ __forceinline__ int32_t decide(const ScanCtx& s, int32_t v, int32_t cur,
                                          typename KeyOf<LOUV, NK>::T bk, int32_t bc, bool has_cur,
                                          int64_t kcur, int64_t vol) {
  if (bc == NOCAND) return cur;
  if constexpr (!LOUV) {
    if (s.tie_keep && has_cur && kcur == bk) return cur;
    return bc;
  } else {
    int64_t d = s.degw[v];
    i128 G = (i128)bk - (i128)vol * kcur + (i128)d * (s.sigma[cur] - d);
    if (G <= 0) return cur;  // only strictly positive gains
    if (s.singleton_rule && s.csize[cur] == 1 && s.csize[bc] == 1 && bc > cur) return cur;
    return bc;
  }
}

// Asynchronous mode: v's move from `cur` to `target` takes effect now.
__device__ __forceinline__ void apply_now(const ScanCtx& s, int32_t v, int32_t cur, int32_t target) {
  s.C_w[v] = target;
  if (s.sigma_w) {
    const int64_t d = s.degw[v];
    atomicAdd((unsigned long long*)&s.sigma_w[cur], (unsigned long long)(-d));
    atomicAdd((unsigned long long*)&s.sigma_w[target], (unsigned long long)d);
    atomicSub(&s.csize_w[cur], 1);
    atomicAdd(&s.csize_w[target], 1);
  }
}

// One thread acts on a decision: append a committed move or count a deferral.
// Returns 1 if the move was deferred.
__device__ __forceinline__ int act_single(const ScanCtx& s, int32_t v, int32_t cur, int32_t target) {
  if (target == cur) return 0;
  if (s.mark) flag_next(s, v);
  count_change(s, v);
  if (commit_coin(s.seed, s.level, round_of(s), local_id(s, v))) {
    unsigned long long pos = atomicAdd(&s.ctr[C_MOVES], 1ull);
    s.mv_v[pos] = v;
    s.mv_c[pos] = target;
    s.mv_a[pos] = cur;
    if (s.async_mode) apply_now(s, v, cur, target);
    return 0;
  }
  return 1;
}

__device__ __forceinline__ void flush_counters(const ScanCtx& s, int bin, int64_t act, int64_t arcs,
                                               int64_t cands, int64_t def, int64_t marcs) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    act += __shfl_xor_sync(FULL, act, o);
    arcs += __shfl_xor_sync(FULL, arcs, o);
    cands += __shfl_xor_sync(FULL, cands, o);
    def += __shfl_xor_sync(FULL, def, o);
    marcs += __shfl_xor_sync(FULL, marcs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (act) atomicAdd(&s.ctr[C_BIN0 + 3 * bin], (unsigned long long)act);
    if (arcs) atomicAdd(&s.ctr[C_BIN0 + 3 * bin + 1], (unsigned long long)arcs);
    if (cands) atomicAdd(&s.ctr[C_BIN0 + 3 * bin + 2], (unsigned long long)cands);
    if (def) atomicAdd(&s.ctr[C_DEFERRED], (unsigned long long)def);
    if (marcs) atomicAdd(&s.ctr[C_MARCS], (unsigned long long)marcs);
  }
}

__device__ __forceinline__ bool is_active(const ScanCtx& s, int32_t v) {
  if (s.gfrozen && s.gfrozen[s.gid[v]]) return false;
  return s.all_active || ((s.flag_cur[v >> 5] >> (v & 31)) & 1u);
}

// Group weight of the lanes in `peers` (equal labels): popcount for unit
// weights, else a sum over the warp's staging row.
template <class W>
__device__ __forceinline__ int64_t group_sum(unsigned peers, int64_t wt, int64_t* stage) {
  if constexpr (W::unit) {
    return (int64_t)__popc(peers);
  } else {
    const int lane = threadIdx.x & 31;
    stage[lane] = wt;
    __syncwarp();
    int64_t s = 0;
    unsigned m = peers;
    while (m) {
      s += stage[__ffs(m) - 1];
      m &= m - 1;
    }
    __syncwarp();
    return s;
  }
}

// ------------------------------------------------------------------ hub histograms

constexpr unsigned long long SLOT_EMPTY = ~0ull;

// Flag hub h for the start of the next round: HUB_REBUILD (an update was
// lost; it is rebuilt from its row and not updated until then) or
// HUB_COMPACT (it is consistent but too full; its live entries are rehashed).
// A hub is queued once, when it is first flagged.
constexpr int32_t HUB_REBUILD = 1, HUB_COMPACT = 2;

__device__ __forceinline__ void hub_flag(const ScanCtx& s, int32_t h, int32_t how) {
  const int32_t old = how == HUB_REBUILD ? atomicExch(&s.hub_rb[h], HUB_REBUILD) : atomicCAS(&s.hub_rb[h], 0, how);
  if (old == 0) s.hub_flist_w[atomicAdd(s.hub_fcnt_w, 1ull)] = h;
}

// Slot of `label` in a table of `cap` slots (hub histograms, here and in the
// shared-memory layouts built for them).
__device__ __forceinline__ int64_t hub_home(int32_t label, int64_t cap) {
  return (int64_t)(((uint64_t)((uint32_t)label * 2654435761u) * (uint64_t)cap) >> 32);
}

// An update gives up after HUB_PROBE_MAX probes (the hub is rebuilt), and a
// hub whose claimed slots pass 7/8 of its capacity is compacted: labels that
// leave keep their slot (count 0), so a table fills up over the rounds and
// linear-probe chains would otherwise grow without bound.
constexpr int HUB_PROBE_MAX = 64;
constexpr int64_t HUB_SKIP_DIV = 16;     // Louvain (measured: 4 and 64 slower)
constexpr int64_t HUB_SKIP_DIV_LPA = 4;  // LPA (measured: 16 slower by 12%)

// k_{h,label} += w in hub h's histogram (w may be negative: a neighbour left
// `label`; the count then stays >= 0). A packed slot is updated with one
// 64-bit atomic: the count lives in the low word and never carries or borrows
// into the label. A build (BUILD) probes the whole table, which at most two
// thirds of its slots can fill; an update gives up after HUB_PROBE_MAX probes
// or when a label to decrement is missing, and then flags the hub.
template <bool BUILD>
__device__ __forceinline__ void hub_hist_add(const ScanCtx& s, int32_t h, int32_t label, int64_t w) {
  if (!BUILD && s.hub_rb[h] == HUB_REBUILD) return;
  const int64_t base = s.hub_tab[h];
  const int64_t cap = s.hub_cc[h];
  const int64_t lim = BUILD ? cap : (cap < HUB_PROBE_MAX ? cap : HUB_PROBE_MAX);
  int64_t slot = hub_home(label, cap);
  bool claimed = false;
  if (!s.hub_wide) {
    unsigned long long* words = s.hub_slot + base;
    for (int64_t probe = 0; probe < lim; ++probe) {
      unsigned long long cur = words[slot];
      if (cur == SLOT_EMPTY) {
        if (w <= 0) break;
        cur = atomicCAS(&words[slot], SLOT_EMPTY,
                        ((unsigned long long)(uint32_t)label << 32) | (unsigned long long)(uint32_t)w);
        if (cur == SLOT_EMPTY) {
          claimed = true;
          break;
        }
      }
      if ((int32_t)(cur >> 32) == label) {
        atomicAdd(&words[slot], (unsigned long long)w);
        return;
      }
      slot = slot + 1 == cap ? 0 : slot + 1;
    }
  } else {
    unsigned long long* words = s.hub_slot + 2 * base;  // (label, count) pairs
    for (int64_t probe = 0; probe < lim; ++probe) {
      unsigned long long cur = words[2 * slot];
      if (cur == SLOT_EMPTY) {
        if (w <= 0) break;
        cur = atomicCAS(&words[2 * slot], SLOT_EMPTY, (unsigned long long)(uint32_t)label);
        if (cur == SLOT_EMPTY) {
          claimed = true;
          cur = (uint32_t)label;
        }
      }
      if ((int32_t)(uint32_t)cur == label) {
        atomicAdd(&words[2 * slot + 1], (unsigned long long)w);
        if (!claimed) return;
        break;
      }
      slot = slot + 1 == cap ? 0 : slot + 1;
    }
  }
  if (claimed) {
    const int32_t used = atomicAdd(&s.hub_used[h], 1) + 1;
    if (!BUILD && (int64_t)used * 8 > cap * 7) hub_flag(s, h, HUB_COMPACT);
    return;
  }
  hub_flag(s, h, HUB_REBUILD);
}

// Read slot i of a hub table at `base`: (label or -1 if empty, count).
__device__ __forceinline__ void hub_slot_read(const ScanCtx& s, int64_t base, int64_t i, int32_t& c,
                                              int64_t& k) {
  if (!s.hub_wide) {
    const unsigned long long x = s.hub_slot[base + i];
    c = x == SLOT_EMPTY ? -1 : (int32_t)(x >> 32);
    k = (int64_t)(x & 0xffffffffull);
  } else {
    const unsigned long long x = s.hub_slot[2 * (base + i)];
    c = x == SLOT_EMPTY ? -1 : (int32_t)(uint32_t)x;
    k = (int64_t)s.hub_slot[2 * (base + i) + 1];
  }
}

// A committed move of a neighbour of u (label A -> c over an arc of weight
// w) changes u's histogram if u is a hub. The hub bitmap (n bits) stays in L2.
__device__ __forceinline__ void hub_neighbour_moved(const ScanCtx& s, int32_t u, int32_t A, int32_t c,
                                                    int64_t w) {
  if (!hub_upd_of(s)) return;
  const uint32_t bits = __ldg(&s.hub_bits[u >> 5]);
  if (!((bits >> (u & 31)) & 1u)) return;
  const int32_t h = (int32_t)(__ldg(&s.hub_pref[u >> 5]) + __popc(bits & ((1u << (u & 31)) - 1u)));
  if (s.hub_log) {
    // appended as (h, A) and (c, w) words by the lanes that got here together;
    // applied by k_hub_apply_log with every thread busy
    cg::coalesced_group grp = cg::coalesced_threads();
    unsigned long long pos = 0;
    if (grp.thread_rank() == 0) pos = atomicAdd(s.hub_log_cnt, (unsigned long long)grp.size());
    pos = grp.shfl(pos, 0) + grp.thread_rank();
    if ((int64_t)pos < s.hub_log_cap) {
      s.hub_log[2 * pos] = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)A;
      s.hub_log[2 * pos + 1] = ((unsigned long long)(uint32_t)c << 32) | (unsigned long long)(uint32_t)w;
    } else {
      hub_flag(s, h, HUB_REBUILD);  // log full: rebuild this hub from its row instead
    }
    return;
  }
  hub_hist_add<false>(s, h, A, -w);
  hub_hist_add<false>(s, h, c, w);
}

// The round's logged hub-histogram updates, one thread per record.
__global__ void __launch_bounds__(NT) k_hub_apply_log(ScanCtx s) {
  const int64_t nrec = (int64_t)*(volatile unsigned long long*)s.hub_log_cnt;
  const int64_t m = nrec < s.hub_log_cap ? nrec : s.hub_log_cap;
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < m; i += stride) {
    const unsigned long long a = s.hub_log[2 * i], b = s.hub_log[2 * i + 1];
    const int32_t h = (int32_t)(a >> 32), A = (int32_t)(uint32_t)a, c = (int32_t)(b >> 32);
    const int64_t w = (int64_t)(b & 0xffffffffull);
    hub_hist_add<false>(s, h, A, -w);
    hub_hist_add<false>(s, h, c, w);
  }
}

// ------------------------------------------------------------------ tiles

// TILE lanes per vertex, one arc per lane (degree <= TILE).
template <int TILE, bool LOUV, class W, bool NK>
__global__ void __launch_bounds__(NT, 6) k_scan_tile(ScanCtx s, const int32_t* __restrict__ list,
                                                  const unsigned long long* __restrict__ count_p, int bin) {
  typedef typename KeyOf<LOUV, NK>::T K;
  const int64_t count = (int64_t)*count_p;
  __shared__ int64_t stage[NW][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int sub = lane & (TILE - 1);
  const int tbase = lane & ~(TILE - 1);
  const unsigned tmask = TILE == 32 ? FULL : (((1u << TILE) - 1u) << tbase);
  constexpr int VPW = 32 / TILE;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  int64_t n_act = 0, n_arcs = 0, n_cand = 0, n_def = 0, n_marcs = 0;
  for (int64_t base = warp * VPW; base < count; base += nwarps * VPW) {
    const int64_t i = base + lane / TILE;
    const bool valid = i < count;
    const int32_t v = valid ? list[i] : 0;
    const bool act = valid && is_active(s, v);
    int64_t beg = 0;
    int d = 0;
    if (act) {
      beg = s.off[v];
      d = (int)(s.off[v + 1] - beg);
    }
    const bool has = act && sub < d;
    const int32_t u = has ? s.cols[beg + sub] : v;
    const int64_t wt = has ? W::get(s.w, beg + sub) : 0;
    const bool cand = has && u != v;
    const int32_t lbl = cand ? s.C[u] : (int32_t)(0x80000000u | (unsigned)lane);
    const unsigned peers = __match_any_sync(FULL, lbl) & tmask;
    const int64_t gsum = group_sum<W>(peers, wt, stage[wid]);
    const bool leader = cand && (__ffs(peers) - 1) == lane;
    const int32_t cur = act ? s.C[v] : 0;
    const unsigned cm = __ballot_sync(FULL, cand && lbl == cur) & tmask;
    int64_t kcur = __shfl_sync(FULL, gsum, cm ? __ffs(cm) - 1 : lane);
    if (!cm) kcur = 0;
    const int64_t dv = (LOUV && act) ? s.degw[v] : 0;
    const int64_t volv = (LOUV && act) ? vol_of(s, v) : 0;
    const bool ok = leader && (!LOUV || lbl != cur);
    K bk = ok ? cand_key<LOUV, NK>(s, lbl, gsum, dv, volv) : K(0);
    int32_t bc = ok ? lbl : NOCAND;
    reduce_best(bk, bc, TILE);
    int32_t target = cur;
    if (act) target = decide<LOUV, NK>(s, v, cur, bk, bc, cm != 0, kcur, volv);
    const bool want = act && target != cur;
    const bool commit = want && commit_coin(s.seed, s.level, round_of(s), local_id(s, v));
    if (want && sub == 0) count_change(s, v);
    const unsigned am = __ballot_sync(FULL, commit && sub == 0);
    if (am) {
      const int first = __ffs(am) - 1;
      unsigned long long pos0 = 0;
      if (lane == first) pos0 = atomicAdd(&s.ctr[C_MOVES], (unsigned long long)__popc(am));
      pos0 = __shfl_sync(FULL, pos0, first);
      if (commit && sub == 0) {
        const unsigned long long pos = pos0 + __popc(am & ((1u << lane) - 1u));
        s.mv_v[pos] = v;
        s.mv_c[pos] = target;
        s.mv_a[pos] = cur;
        if (s.async_mode) apply_now(s, v, cur, target);
      }
    }
    if (s.mark) {
      if (commit && has) flag_next(s, u);  // the neighbours of a moved vertex
      if (want && sub == 0) flag_next(s, v);
    }
    if (s.nhubs > 0 && commit && cand) hub_neighbour_moved(s, u, cur, target, wt);
    if (sub == 0 && act) {
      ++n_act;
      n_arcs += d;
      if (want && !commit) ++n_def;
      if (commit) n_marcs += d;
    }
    if (leader) ++n_cand;  // every distinct neighbour label, the vertex's own included
  }
  flush_counters(s, bin, n_act, n_arcs, n_cand, n_def, n_marcs);
}

// ------------------------------------------------------------------ shared-memory tables

// Open addressing with linear probing; capacity 2^lg >= 2 x the arcs inserted,
// so a free slot is always found within `cap` probes. A newly claimed slot is
// appended to the table's occupied list, so that reading the table costs the
// number of distinct labels rather than its capacity.
template <class V>
__device__ __forceinline__ void smem_insert(int32_t* keys, V* vals, uint16_t* occ, int* occ_n,
                                            unsigned lg, int32_t key, V w, int32_t* status) {
  const unsigned mask = (1u << lg) - 1u;
  unsigned h = ((uint32_t)key * 2654435761u) >> (32 - lg);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int32_t prev = atomicCAS(&keys[h], EMPTY, key);
    if (prev == EMPTY || prev == key) {
      atomicAdd(vals + h, w);
      if (prev == EMPTY) occ[atomicAdd(occ_n, 1)] = (uint16_t)h;
      return;
    }
    h = (h + 1) & mask;
  }
  atomicCAS(status, 0, CD_ETIMEOUT);  // table full: impossible with cap >= 2 deg
}

__device__ __forceinline__ unsigned ceil_log2(int64_t x) {
  unsigned lg = 0;
  while (((int64_t)1 << lg) < x) ++lg;
  return lg < 1 ? 1 : lg;
}

// Synchronise the GROUP threads sharing a table: a warp, the whole CTA, or a
// named barrier (ids 1..15) for a sub-CTA group.
template <int GROUP, int NTB>
__device__ __forceinline__ void group_sync(int gid) {
  if constexpr (GROUP == 32)
    __syncwarp();
  else if constexpr (GROUP == NTB)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "n"(GROUP) : "memory");
}

// Insert the arcs [beg, end) of vertex v into a group's table. Columns are
// read 16 bytes at a time (4 arcs per lane, 4 label gathers in flight); equal
// labels inside a warp are combined with __match_any_sync before the atomics.
// Column arrays carry COL_PAD spare entries, so a 16-byte load that starts
// before `end` stays inside the allocation.
template <class W, class V, int GROUP>
__device__ __forceinline__ void group_insert(const ScanCtx& s, int32_t v, int64_t beg, int64_t end,
                                             int gl, int32_t* keys, V* vals, uint16_t* occ, int* occ_n,
                                             unsigned lg, int64_t* stage) {
  const int lane = threadIdx.x & 31;
  const int wig = gl >> 5;
  const int64_t a0 = beg & ~(int64_t)3;
  for (int64_t wb = a0 + (int64_t)wig * 128; wb < end; wb += (int64_t)GROUP * 4) {
    const int64_t base = wb + 4 * lane;
    const int4 c4 = base < end ? __ldg(reinterpret_cast<const int4*>(s.cols + base)) : make_int4(0, 0, 0, 0);
    const int32_t cs[4] = {c4.x, c4.y, c4.z, c4.w};
    int32_t lbl[4];
    int64_t wt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t e = base + j;
      const bool has = e >= beg && e < end;
      const bool cand = has && cs[j] != v;
      lbl[j] = cand ? s.C[cs[j]] : (int32_t)(0x80000000u | (unsigned)(lane * 4 + j));
      wt[j] = (has && !W::unit) ? W::get(s.w, e) : 1;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned peers = __match_any_sync(FULL, lbl[j]);
      const int64_t gsum = group_sum<W>(peers, wt[j], stage);
      if (lbl[j] >= 0 && (__ffs(peers) - 1) == lane)
        smem_insert(keys, vals, occ, occ_n, lg, lbl[j], (V)gsum, s.status);
    }
  }
}

// Read a group's table through its occupied list: every listed slot is a
// candidate; the slot is cleared for the next vertex.
template <bool LOUV, class V, int GROUP, bool NK>
__device__ __forceinline__ void group_eval(const ScanCtx& s, int32_t cur, int64_t dv, int64_t vol,
                                           int gl, int32_t* keys, V* vals, const uint16_t* occ, int nocc,
                                           typename KeyOf<LOUV, NK>::T& bk, int32_t& bc, bool& hc,
                                           int64_t& kc, int64_t& ncand) {
  constexpr int EB = 2;  // candidates per thread per batch: the Sigma_tot gathers go out together
  for (int j0 = gl; j0 < nocc; j0 += EB * GROUP) {
    int32_t c[EB];
    int64_t k[EB], sg[EB];
#pragma unroll
    for (int q = 0; q < EB; ++q) {
      const int j = j0 + q * GROUP;
      c[q] = -1;
      k[q] = 0;
      if (j < nocc) {
        const int slot = occ[j];
        c[q] = keys[slot];
        k[q] = (int64_t)vals[slot];
        keys[slot] = EMPTY;
        vals[slot] = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < EB; ++q) sg[q] = (LOUV && c[q] >= 0) ? sig_of<NK>(s, c[q]) : 0;
#pragma unroll
    for (int q = 0; q < EB; ++q) {
      if (c[q] < 0) continue;
      ++ncand;
      if (c[q] == cur) {
        hc = true;
        kc = k[q];
        if (LOUV) continue;
      }
      const typename KeyOf<LOUV, NK>::T key = cand_key_sg<LOUV, NK>(sg[q], k[q], dv, vol);
      if (better(key, c[q], bk, bc)) {
        bk = key;
        bc = c[q];
      }
    }
  }
}

// What a scan needs of a vertex before reading its row.
struct VHdr {
  int64_t beg, end, dv, vol;
  int32_t cur;
  bool act;
};

template <bool LOUV>
__device__ __forceinline__ VHdr load_hdr(const ScanCtx& s, int32_t v, bool valid) {
  VHdr h;
  h.act = valid && is_active(s, v);
  h.beg = valid ? s.off[v] : 0;
  h.end = valid ? s.off[v + 1] : 0;
  h.cur = valid ? s.C[v] : 0;
  h.dv = (LOUV && valid) ? s.degw[v] : 0;
  h.vol = (LOUV && valid) ? vol_of(s, v) : 0;
  return h;
}

// GROUP threads per vertex (a warp, or a named-barrier group of 128 or 512
// threads), each group with its own CAP-slot shared-memory table.
template <bool LOUV, class W, class V, int GROUP, int NTB, int CAP, int BIN, bool PF, bool NK>
__global__ void __launch_bounds__(NTB, GROUP == 32 ? ((LOUV || !W::unit) ? 4 : 5) : 2)
    k_scan_group(ScanCtx s, const int32_t* __restrict__ list, const unsigned long long* __restrict__ count_p) {
  typedef typename KeyOf<LOUV, NK>::T K;
  const int64_t count = (int64_t)*count_p;
  constexpr int GPB = NTB / GROUP;  // groups per CTA
  constexpr int WPG = GROUP / 32;   // warps per group
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ K red_k[GPB][WPG];
  __shared__ int32_t red_c[GPB][WPG];
  __shared__ int64_t red_kc[GPB][WPG];
  __shared__ int32_t red_hc[GPB][WPG];
  __shared__ int occ_n[GPB];
  __shared__ int32_t moved_to[GPB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gid = threadIdx.x / GROUP, gl = threadIdx.x % GROUP, wig = gl >> 5;
  V* vals = (V*)smem + (size_t)gid * CAP;
  int32_t* keys = (int32_t*)(smem + (size_t)GPB * CAP * sizeof(V)) + (size_t)gid * CAP;
  int64_t* stage = (int64_t*)(smem + (size_t)GPB * CAP * (sizeof(V) + 4)) + wid * 32;
  uint16_t* occ = (uint16_t*)(smem + (size_t)GPB * CAP * (sizeof(V) + 4) + (size_t)(NTB / 32) * 32 * 8) +
                  (size_t)gid * CAP;
  for (int j = gl; j < CAP; j += GROUP) {
    keys[j] = EMPTY;
    vals[j] = 0;
  }
  if (gl == 0) occ_n[gid] = 0;
  group_sync<GROUP, NTB>(gid);
  int64_t n_act = 0, n_arcs = 0, n_cand = 0, n_def = 0, n_marcs = 0;
  // Software pipeline over the group's vertices: while vertex i is processed,
  // the header of vertex i + stride (activity, row bounds, label, deg_w) and
  // the list entry of vertex i + 2 stride are already in flight.
  const int64_t stride = (int64_t)gridDim.x * GPB;
  int64_t i = (int64_t)blockIdx.x * GPB + gid;
  int32_t v_nx = 0, v_nn = 0;
  VHdr h_nx{};
  if constexpr (PF) {
    v_nx = i < count ? list[i] : 0;
    h_nx = load_hdr<LOUV>(s, v_nx, i < count);
    v_nn = i + stride < count ? list[i + stride] : 0;
  }
  for (; i < count; i += stride) {
    int32_t v;
    VHdr h;
    if constexpr (PF) {
      v = v_nx;
      h = h_nx;
      v_nx = v_nn;
      h_nx = load_hdr<LOUV>(s, v_nx, i + stride < count);
      v_nn = i + 2 * stride < count ? list[i + 2 * stride] : 0;
    } else {
      v = list[i];
      h = load_hdr<LOUV>(s, v, true);
    }
    if (!h.act) continue;  // uniform within the group
    const int64_t beg = h.beg, end = h.end;
    const int64_t d = end - beg;
    const unsigned lg = ceil_log2(2 * d);
    const int32_t cur = h.cur;
    group_insert<W, V, GROUP>(s, v, beg, end, gl, keys, vals, occ, &occ_n[gid], lg, stage);
    group_sync<GROUP, NTB>(gid);
    const int64_t dv = h.dv;
    const int64_t volv = h.vol;
    const int nocc = occ_n[gid];
    K bk = K(0);
    int32_t bc = NOCAND;
    bool hc = false;
    int64_t kc = 0;
    group_eval<LOUV, V, GROUP, NK>(s, cur, dv, volv, gl, keys, vals, occ, nocc, bk, bc, hc, kc, n_cand);
    reduce_best(bk, bc, 32);
    unsigned hm = __ballot_sync(FULL, hc);
    if (hm) kc = __shfl_sync(FULL, kc, __ffs(hm) - 1);
    if constexpr (WPG > 1) {
      if (lane == 0) {
        red_k[gid][wig] = bk;
        red_c[gid][wig] = bc;
        red_hc[gid][wig] = hm != 0;
        red_kc[gid][wig] = kc;
      }
      group_sync<GROUP, NTB>(gid);
      if (wig == 0) {
        bk = lane < WPG ? red_k[gid][lane] : K(0);
        bc = lane < WPG ? red_c[gid][lane] : NOCAND;
        reduce_best(bk, bc, 32);
        hm = __ballot_sync(FULL, lane < WPG && red_hc[gid][lane]);
        kc = hm ? red_kc[gid][__ffs(hm) - 1] : 0;
      }
    }
    if (gl == 0) {
      const int32_t target = decide<LOUV, NK>(s, v, cur, bk, bc, hm != 0, kc, volv);
      const int def = act_single(s, v, cur, target);
      n_def += def;
      ++n_act;
      n_arcs += d;
      if (target != cur && !def) n_marcs += d;
      occ_n[gid] = 0;
      moved_to[gid] = (target != cur && !def) ? target : -1;
    }
    group_sync<GROUP, NTB>(gid);  // tables and reduction slots are reused after this
    // a committed move: flag the neighbours for the next round and update the
    // histograms of neighbouring hubs (their evaluation for this round is done)
    const int32_t to = moved_to[gid];
    if (to >= 0 && (s.mark || s.nhubs > 0))
      for (int64_t e = beg + gl; e < end; e += GROUP) {
        const int32_t u = s.cols[e];
        if (s.mark) flag_next(s, u);
        if (s.nhubs > 0 && u != v) hub_neighbour_moved(s, u, cur, to, W::get(s.w, e));
      }
  }
  flush_counters(s, BIN, n_act, n_arcs, n_cand, n_def, n_marcs);
}

// The warp bin (degrees 33..t_warp): a warp takes vb (a power of two <= 32)
// listed vertices at a time. Lane j < vb loads vertex j's header; the warp
// then scans each active vertex in turn (table inserts and evaluation as in
// k_scan_group) and lane j keeps vertex j's best candidate. The decisions,
// coins and move-list appends then run in parallel, one lane per vertex, and
// the neighbours of the committed moves are flagged (and their hub histograms
// updated) last. vb = 32 on large bins; a small bin takes fewer vertices per
// warp so that its warps still fill the GPU.
template <bool LOUV, class W, class V, bool NK>
__global__ void __launch_bounds__(256, (LOUV || !W::unit) ? 4 : 5)
    k_scan_warp(ScanCtx s, const int32_t* __restrict__ list, const unsigned long long* __restrict__ count_p,
                int vb) {
  typedef typename KeyOf<LOUV, NK>::T K;
  constexpr int CAP = WARP_CAP_SLOTS, WPB = 256 / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int occ_n[WPB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  V* vals = (V*)smem + (size_t)wid * CAP;
  int32_t* keys = (int32_t*)(smem + (size_t)WPB * CAP * sizeof(V)) + (size_t)wid * CAP;
  int64_t* stage = (int64_t*)(smem + (size_t)WPB * CAP * (sizeof(V) + 4)) + wid * 32;
  uint16_t* occ = (uint16_t*)(smem + (size_t)WPB * CAP * (sizeof(V) + 4) + (size_t)WPB * 32 * 8) + (size_t)wid * CAP;
  for (int j = lane; j < CAP; j += 32) {
    keys[j] = EMPTY;
    vals[j] = 0;
  }
  if (lane == 0) occ_n[wid] = 0;
  __syncwarp();
  const int64_t count = (int64_t)*count_p;
  const int64_t warp = ((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * 256) >> 5;
  int64_t n_act = 0, n_arcs = 0, n_cand = 0, n_def = 0, n_marcs = 0;
  for (int64_t base = warp * vb; base < count; base += nwarps * vb) {
    const int64_t i = base + lane;
    const bool in = lane < vb && i < count;
    const int32_t my_v = in ? list[i] : 0;
    const VHdr h = load_hdr<LOUV>(s, my_v, in);
    K my_bk = K(0);
    int32_t my_bc = NOCAND;
    bool my_hc = false;
    int64_t my_kc = 0;
    for (unsigned am = __ballot_sync(FULL, h.act); am; am &= am - 1) {
      const int j = __ffs(am) - 1;
      const int32_t v = __shfl_sync(FULL, my_v, j);
      const int64_t beg = __shfl_sync(FULL, h.beg, j), end = __shfl_sync(FULL, h.end, j);
      const int32_t cur = __shfl_sync(FULL, h.cur, j);
      const int64_t dv = LOUV ? __shfl_sync(FULL, h.dv, j) : 0;
      const int64_t volv = LOUV ? __shfl_sync(FULL, h.vol, j) : 0;
      const unsigned lg = 64 - __clzll((unsigned long long)(2 * (end - beg) - 1));  // 2^lg >= 2 deg
      group_insert<W, V, 32>(s, v, beg, end, lane, keys, vals, occ, &occ_n[wid], lg, stage);
      __syncwarp();
      K bk = K(0);
      int32_t bc = NOCAND;
      bool hc = false;
      int64_t kc = 0;
      group_eval<LOUV, V, 32, NK>(s, cur, dv, volv, lane, keys, vals, occ, occ_n[wid], bk, bc, hc, kc, n_cand);
      reduce_best(bk, bc, 32);
      const unsigned hm = __ballot_sync(FULL, hc);
      if (hm) kc = __shfl_sync(FULL, kc, __ffs(hm) - 1);
      if (lane == j) {
        my_bk = bk;
        my_bc = bc;
        my_hc = hm != 0;
        my_kc = kc;
      }
      __syncwarp();
      if (lane == 0) occ_n[wid] = 0;
      __syncwarp();
    }
    // the batch's decisions, one lane per vertex
    int32_t target = h.cur;
    if (h.act) target = decide<LOUV, NK>(s, my_v, h.cur, my_bk, my_bc, my_hc, my_kc, h.vol);
    const bool want = h.act && target != h.cur;
    const bool commit = want && commit_coin(s.seed, s.level, round_of(s), local_id(s, my_v));
    if (want) count_change(s, my_v);
    const unsigned cm = __ballot_sync(FULL, commit);
    if (cm) {
      const int first = __ffs(cm) - 1;
      unsigned long long pos0 = 0;
      if (lane == first) pos0 = atomicAdd(&s.ctr[C_MOVES], (unsigned long long)__popc(cm));
      pos0 = __shfl_sync(FULL, pos0, first);
      if (commit) {
        const unsigned long long pos = pos0 + __popc(cm & ((1u << lane) - 1u));
        s.mv_v[pos] = my_v;
        s.mv_c[pos] = target;
        s.mv_a[pos] = h.cur;
        if (s.async_mode) apply_now(s, my_v, h.cur, target);
      }
    }
    if (want && s.mark) flag_next(s, my_v);
    if (h.act) {
      ++n_act;
      n_arcs += h.end - h.beg;
      if (!commit && want) ++n_def;
      if (commit) n_marcs += h.end - h.beg;
    }
    // committed moves: flag the neighbours for the next round and update the
    // histograms of neighbouring hubs (their evaluation for this round is done)
    if (s.mark || s.nhubs > 0)
      for (unsigned m = cm; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const int32_t v = __shfl_sync(FULL, my_v, j);
        const int64_t beg = __shfl_sync(FULL, h.beg, j), end = __shfl_sync(FULL, h.end, j);
        const int32_t from = __shfl_sync(FULL, h.cur, j), to = __shfl_sync(FULL, target, j);
        for (int64_t e = beg + lane; e < end; e += 32) {
          const int32_t u = s.cols[e];
          if (s.mark) flag_next(s, u);
          if (s.nhubs > 0 && u != v) hub_neighbour_moved(s, u, from, to, W::get(s.w, e));
        }
      }
  }
  flush_counters(s, B_WARP, n_act, n_arcs, n_cand, n_def, n_marcs);
}

// ------------------------------------------------------------------ hubs
//
// A hub keeps k_{v,c} for every neighbour label c in a persistent histogram:
// built from its row when the run (or level) starts, then updated by every
// committed move of a neighbour (k[old] -= w, k[new] += w). Evaluating a hub
// therefore reads its distinct labels instead of its whole row.

constexpr int HUB_CL_SLOTS = 12288;    // table slots per CTA of a cluster build (96 KB: 2 CTAs per SM)
constexpr int HUB_CL1_SLOTS = 8192;    // a one-CTA build of 512 threads (64 KB: 3 CTAs per SM)
constexpr int HUB_CL0_SLOTS = 4096;    // a one-CTA build of 256 threads (32 KB: 7 CTAs per SM)
constexpr int HUB_NCLASS = 5;          // build classes: one CTA (small, large), clusters of 2, 4, 8
// Build class of a hub table of `cap` packed slots: 0..4, or -1 (too large: chunked global inserts).
__host__ __device__ constexpr int hub_class(int64_t cap) {
  return cap <= HUB_CL0_SLOTS ? 0 : cap <= HUB_CL1_SLOTS ? 1 : cap <= 2 * HUB_CL_SLOTS ? 2
       : cap <= 4 * HUB_CL_SLOTS ? 3 : cap <= 8 * HUB_CL_SLOTS ? 4 : -1;
}
template <int CI> struct HubClass;  // CTAs per cluster, threads per CTA, table slots per CTA
template <> struct HubClass<0> { static constexpr int C = 1, NT = 256, SLOTS = HUB_CL0_SLOTS; };
template <> struct HubClass<1> { static constexpr int C = 1, NT = 512, SLOTS = HUB_CL1_SLOTS; };
template <> struct HubClass<2> { static constexpr int C = 2, NT = 512, SLOTS = HUB_CL_SLOTS; };
template <> struct HubClass<3> { static constexpr int C = 4, NT = 512, SLOTS = HUB_CL_SLOTS; };
template <> struct HubClass<4> { static constexpr int C = 8, NT = 512, SLOTS = HUB_CL_SLOTS; };
template <int CI> constexpr size_t hub_cl_smem() { return (size_t)HubClass<CI>::SLOTS * 8; }
constexpr int HUB_PREP_SLOTS = 12288;  // shared-memory slots of a compaction (live list + new table)
constexpr size_t HUB_PREP_SMEM = (size_t)HUB_PREP_SLOTS * 8;

// A hub's table in use is [0, cc) of its allocation of A = 1.5 deg + 64
// slots; the slots past cc are empty. A rebuild from the row takes all of A
// (the number of distinct labels is not known before it). When an evaluation
// finds at most a quarter of the slots in use holding live entries, the hub
// is queued for compaction, which rehashes them into 2 live + 64 slots. Late
// in a level most hubs' neighbours sit in few communities, so an evaluation
// then reads a few hundred slots instead of 1.5 deg.
constexpr int64_t HUB_SHRINK_MIN = 512;  // tables in use this small are left as they are
__device__ __forceinline__ void hub_maybe_shrink(const ScanCtx& s, int32_t h, int64_t cc, int64_t live) {
  if (!s.hub_wide && cc > HUB_SHRINK_MIN && live * 4 < cc && 3 * live + 64 <= HUB_PREP_SLOTS && s.hub_rb[h] == 0)
    hub_flag(s, h, HUB_COMPACT);
}

// Start of a round, a CTA per hub flagged in the previous round (every hub in
// round 0). COMPACT (packed slots): the live entries (count > 0) are listed at
// the top of shared memory and rehashed below them into a table of 2 live + 64
// slots (at most the allocation), which is written back with coalesced stores
// (the slots it no longer uses are cleared). REBUILD, or too many live entries
// for shared memory: the table goes back to its whole allocation, is cleared
// (unless a cluster build overwrites it whole) and the hub's build is queued.
__global__ void __launch_bounds__(NT) k_hub_prepare(ScanCtx s) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* T = (unsigned long long*)smem;
  __shared__ unsigned long long pos;
  __shared__ int n_live;
  const int64_t nf = (int64_t)*(volatile const unsigned long long*)s.hub_fcnt_r;
  for (int64_t q = blockIdx.x; q < nf; q += gridDim.x) {
    const int32_t h = s.hub_flist_r[q];
    const int64_t base = s.hub_tab[h], cap = s.hub_tab[h + 1] - base;  // the allocation
    const int64_t cc = s.hub_cc[h];                                     // slots in use
    const int64_t i0 = s.hub_item_first[h], ni = s.hub_item_first[h + 1] - i0;
    if (s.hub_rb[h] == HUB_COMPACT && !s.hub_wide) {  // uniform in the CTA
      if (threadIdx.x == 0) n_live = 0;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < cc; i += NT) {
        const unsigned long long x = s.hub_slot[base + i];
        if (x == SLOT_EMPTY || (x & 0xffffffffull) == 0) continue;
        const int j = atomicAdd(&n_live, 1);
        if (j < HUB_PREP_SLOTS) T[HUB_PREP_SLOTS - 1 - j] = x;  // the live list grows down from the top
      }
      __syncthreads();
      const int64_t nl = n_live;
      const int64_t nc = 2 * nl + 64 < cap ? 2 * nl + 64 : cap;
      if (nc + nl <= HUB_PREP_SLOTS) {  // the new table [0, nc) lies below the list
        for (int64_t i = threadIdx.x; i < nc; i += NT) T[i] = SLOT_EMPTY;
        __syncthreads();
        for (int64_t j = threadIdx.x; j < nl; j += NT) {
          const unsigned long long x = T[HUB_PREP_SLOTS - 1 - j];
          int64_t slot = hub_home((int32_t)(x >> 32), nc);
          for (int64_t probe = 0; probe < nc; ++probe) {  // nl < nc: always ends
            if (atomicCAS(&T[slot], SLOT_EMPTY, x) == SLOT_EMPTY) break;
            slot = slot + 1 == nc ? 0 : slot + 1;
          }
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < nc; i += NT) s.hub_slot[base + i] = T[i];
        for (int64_t i = nc + threadIdx.x; i < cc; i += NT) s.hub_slot[base + i] = SLOT_EMPTY;
        if (threadIdx.x == 0) {
          s.hub_cc[h] = nc;
          s.hub_used[h] = (int32_t)nl;
          s.hub_rb[h] = 0;
          atomicAdd(&s.ctr[C_HUB_PSLOTS], (unsigned long long)(2 * cc));  // read and written
        }
        __syncthreads();
        continue;
      }
    }
    if (!s.hub_wide && hub_class(cap) >= 0) {  // one CTA or a cluster builds it and writes the whole table
      if (threadIdx.x == 0) {
        const int c = hub_class(cap);
        s.hub_cc[h] = cap;
        s.hub_used[h] = 0;
        s.hub_rb[h] = HUB_REBUILD;  // cleared by the cluster once built
        s.hub_cl[(int64_t)c * s.nhubs + (int64_t)atomicAdd(&s.hub_ccnt[c], 1ull)] = h;
      }
      __syncthreads();
      continue;
    }
    {  // giant or two-word hubs: cleared here (the slots past cc are empty already),
       // built by items with global inserts
      const int64_t clr = s.hub_wide ? cap : cc;
      if (threadIdx.x == 0) atomicAdd(&s.ctr[C_HUB_PSLOTS], (unsigned long long)clr);
      for (int64_t i = threadIdx.x; i < clr; i += NT) {
        if (!s.hub_wide) {
          s.hub_slot[base + i] = SLOT_EMPTY;
        } else {
          s.hub_slot[2 * (base + i)] = SLOT_EMPTY;
          s.hub_slot[2 * (base + i) + 1] = 0;
        }
      }
    }
    if (threadIdx.x == 0) {
      s.hub_cc[h] = cap;
      s.hub_used[h] = 0;
      s.hub_rb[h] = HUB_REBUILD;  // cleared once built (start of the evaluate kernel)
      pos = atomicAdd(&s.hub_lcnt[0], (unsigned long long)ni);
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < ni; j += NT) s.hub_blist[pos + j] = (int32_t)(i0 + j);
    __syncthreads();
  }
}

constexpr int HUB_NT = 512;

// A hub table of at most C x hub_cl_slots(C) packed slots is rebuilt from the
// hub's row by a cluster of C CTAs: the table is laid out in its final hash
// order across the cluster's shared memories (CTA p holds slots
// [p S, (p+1) S)), every arc's label is added there (remote slots through
// distributed shared memory), and each CTA then writes its part with
// coalesced stores. No global atomics. In shared memory a slot is two 32-bit
// words, the label and its count (packed tables have every count < 2^32), so
// a probe past an occupied slot is a plain 32-bit load, only an empty slot is
// claimed with a compare-and-swap, and the count takes a 32-bit add.
template <int C>
__device__ __forceinline__ bool hub_cl_insert(cg::cluster_group& cl, int32_t* K, uint32_t* V, int64_t cap,
                                              int64_t S, int32_t lbl, uint32_t sum) {
  const uint32_t home = (uint32_t)hub_home(lbl, cap);
  if constexpr (C == 1) {  // the whole table is local
    uint32_t slot = home;
    for (int64_t probe = 0; probe < cap; ++probe) {  // at most 2/3 of the slots fill: always ends
      int32_t k = *(volatile int32_t*)&K[slot];
      if (k == EMPTY) k = atomicCAS(&K[slot], EMPTY, lbl);
      if (k == EMPTY || k == lbl) {
        atomicAdd(&V[slot], sum);
        return k == EMPTY;
      }
      slot = slot + 1 == (uint32_t)cap ? 0 : slot + 1;
    }
  } else {
    // slot = owner * S + local (tables here are < 2^32 slots); probing steps
    // local and carries into the next owner, wrapping at cap
    uint32_t owner = home / (uint32_t)S, local = home - owner * (uint32_t)S;
    for (int64_t probe = 0; probe < cap; ++probe) {  // at most 2/3 of the slots fill: always ends
      int32_t* pk = cl.map_shared_rank(K + local, owner);
      int32_t k = *(volatile int32_t*)pk;
      if (k == EMPTY) k = atomicCAS(pk, EMPTY, lbl);
      if (k == EMPTY || k == lbl) {
        atomicAdd(cl.map_shared_rank(V + local, owner), sum);
        return k == EMPTY;
      }
      if (++local == (uint32_t)S || (int64_t)owner * S + local == cap) {
        local = 0;
        owner = (int64_t)(owner + 1) * S >= cap ? 0 : owner + 1;
      }
    }
  }
  return false;
}

template <class W, int CI>
__global__ void __cluster_dims__(HubClass<CI>::C, 1, 1) __launch_bounds__(HubClass<CI>::NT)
    k_hub_build_cl(ScanCtx s) {
  constexpr int C = HubClass<CI>::C, NTB = HubClass<CI>::NT, SLOTS = HubClass<CI>::SLOTS;
  extern __shared__ __align__(16) unsigned char hsm[];  // SLOTS keys, then as many counts
  int32_t* K = (int32_t*)hsm;
  uint32_t* V = (uint32_t*)(hsm + (size_t)SLOTS * 4);
  __shared__ uint32_t st_w[NTB / 32][32];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t n = (int64_t)*(volatile unsigned long long*)&s.hub_ccnt[CI];
  const int32_t* list = s.hub_cl + (int64_t)CI * s.nhubs;
  // the table starts clean; writing a hub's part out clears it again
  for (int i = threadIdx.x; i < SLOTS; i += NTB) {
    K[i] = EMPTY;
    V[i] = 0;
  }
  if constexpr (C == 1) __syncthreads(); else cl.sync();
  for (int64_t q = blockIdx.x / C; q < n; q += gridDim.x / C) {  // uniform in the cluster
    const int32_t h = list[q];
    const int32_t v = s.hub_list[h];
    const int64_t base = s.hub_tab[h], cap = s.hub_tab[h + 1] - base;
    const int64_t S = (cap + C - 1) / C;  // slots per CTA
    const int64_t mine = cap - rank * S < S ? cap - rank * S : S;
    const int64_t beg = s.off[v], end = s.off[v + 1];
    const int64_t share = (end - beg + C - 1) / C;
    const int64_t a0 = beg + rank * share, a1 = a0 + share < end ? a0 + share : end;
    int claimed = 0;
    constexpr int U = 4;  // arcs per thread per step: their loads and gathers are in flight together
    for (int64_t e0 = a0; e0 < a1; e0 += (int64_t)U * NTB) {  // whole CTAs iterate together
      int32_t nb[U], lbl[U];
      uint32_t w[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int64_t e = e0 + (int64_t)j * NTB + threadIdx.x;
        const bool has = e < a1;
        nb[j] = has ? s.cols[e] : v;
        w[j] = (has && nb[j] != v) ? (uint32_t)W::get(s.w, e) : 0u;
      }
#pragma unroll
      for (int j = 0; j < U; ++j)  // labels are >= 0; a non-candidate gets a lane-unique negative key
        lbl[j] = w[j] ? s.C[nb[j]] : (int32_t)(0x80000000u | (unsigned)lane);
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const bool cand = lbl[j] >= 0;
        const unsigned peers = __match_any_sync(FULL, lbl[j]);
        uint32_t sum;
        if constexpr (W::unit) {
          sum = (uint32_t)__popc(peers);
        } else {
          st_w[wid][lane] = w[j];
          __syncwarp();
          sum = 0;
          unsigned m = peers;
          while (m) {
            sum += st_w[wid][__ffs(m) - 1];
            m &= m - 1;
          }
          __syncwarp();
        }
        if (cand && (__ffs(peers) - 1) == lane && hub_cl_insert<C>(cl, K, V, cap, S, lbl[j], sum)) ++claimed;
      }
    }
    if constexpr (C == 1) __syncthreads(); else cl.sync();  // every insert is done
    for (int64_t i = threadIdx.x; i < mine; i += NTB) {
      const int32_t k = K[i];
      s.hub_slot[base + rank * S + i] =
          k == EMPTY ? SLOT_EMPTY : (((unsigned long long)(uint32_t)k << 32) | (unsigned long long)V[i]);
      K[i] = EMPTY;
      V[i] = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) claimed += __shfl_xor_sync(FULL, claimed, o);
    if (lane == 0 && claimed) atomicAdd(&s.hub_used[h], claimed);
    if (rank == 0 && threadIdx.x == 0) {
      s.hub_rb[h] = 0;
      atomicAdd(&s.ctr[C_HUB_BARCS], (unsigned long long)(end - beg));
      atomicAdd(&s.ctr[C_HUB_BSLOTS], (unsigned long long)cap);
    }
    if constexpr (C == 1) __syncthreads(); else cl.sync();  // parts cleared before the next hub's inserts
  }
}
constexpr int HUB_CAP = 2 * HUB_CHUNK;
static_assert(HUB_CAP == 8192, "hub chunk table");

// Rebuild of the queued hubs too large for a cluster (or with two-word
// slots): every item is one HUB_CHUNK-arc chunk of a hub row, combined in a
// shared-memory table, then added to the hub's histogram with global inserts.
template <class W, class V>
__global__ void __launch_bounds__(HUB_NT) k_hub_build(ScanCtx s) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int occ_n;
  V* vals = (V*)smem;
  int32_t* keys = (int32_t*)(smem + (size_t)HUB_CAP * sizeof(V));
  int64_t* stage = (int64_t*)(smem + (size_t)HUB_CAP * (sizeof(V) + 4)) + (threadIdx.x >> 5) * 32;
  uint16_t* occ = (uint16_t*)(smem + (size_t)HUB_CAP * (sizeof(V) + 4) + (size_t)(HUB_NT / 32) * 32 * 8);
  for (int j = threadIdx.x; j < HUB_CAP; j += HUB_NT) {
    keys[j] = EMPTY;
    vals[j] = 0;
  }
  if (threadIdx.x == 0) occ_n = 0;
  __syncthreads();
  const int64_t nb = (int64_t)*(volatile unsigned long long*)&s.hub_lcnt[0];
  for (int64_t q = blockIdx.x; q < nb; q += gridDim.x) {
    const int32_t it = s.hub_blist[q];
    const int32_t h = s.hub_item_hub[it];
    const int32_t v = s.hub_list[h];
    const int64_t a0 = s.hub_item_arc[it];
    const int64_t rowend = s.off[v + 1];
    const int64_t end = a0 + HUB_CHUNK < rowend ? a0 + HUB_CHUNK : rowend;
    group_insert<W, V, HUB_NT>(s, v, a0, end, threadIdx.x, keys, vals, occ, &occ_n, 13, stage);
    __syncthreads();
    const int nocc = occ_n;
    for (int j = threadIdx.x; j < nocc; j += HUB_NT) {
      const int slot = occ[j];
      const int32_t c = keys[slot];
      const int64_t k = (int64_t)vals[slot];
      keys[slot] = EMPTY;
      vals[slot] = 0;
      hub_hist_add<true>(s, h, c, k);
    }
    if (threadIdx.x == 0) {
      atomicAdd(&s.ctr[C_HUB_BSLOTS], (unsigned long long)nocc);
      atomicAdd(&s.ctr[C_HUB_BARCS], (unsigned long long)(end - a0));
    }
    __syncthreads();
    if (threadIdx.x == 0) occ_n = 0;
    __syncthreads();
  }
}

// Decision of hub h (one thread): act on it, and queue the mark items of a
// committed move (the neighbours are flagged and their hub histograms
// updated by k_hub_mark).
template <bool LOUV, bool NK>
__device__ __forceinline__ void hub_decide(const ScanCtx& s, int32_t h, int32_t v, int32_t cur,
                                           typename KeyOf<LOUV, NK>::T fk, int32_t fc, bool hc, int64_t kc,
                                           int64_t volv, int64_t& n_act, int64_t& n_arcs, int64_t& n_def,
                                           int64_t& n_marcs) {
  const int32_t target = decide<LOUV, NK>(s, v, cur, fk, fc, hc, kc, volv);
  const int def = act_single(s, v, cur, target);
  n_def += def;
  if (target != cur && !def) {
    n_marcs += s.off[v + 1] - s.off[v];
    atomicAdd(&s.ctr[C_HUB_MARCS], (unsigned long long)(s.off[v + 1] - s.off[v]));
    s.hub_mv[3 * h] = 1;
    s.hub_mv[3 * h + 1] = cur;
    s.hub_mv[3 * h + 2] = target;
    const int64_t i0 = s.hub_item_first[h], ni = s.hub_item_first[h + 1] - i0;
    const unsigned long long pos = atomicAdd(&s.hub_lcnt[1], (unsigned long long)ni);
    for (int64_t j = 0; j < ni; ++j) s.hub_mlist[pos + j] = (int32_t)(i0 + j);
  }
  ++n_act;
  n_arcs += s.off[v + 1] - s.off[v];
}

// A small hub (at most HUB_SMALL slots) is evaluated by one warp: no partial
// results, no cross-CTA combination.
template <bool LOUV, bool NK>
__global__ void __launch_bounds__(NT) k_hub_eval_small(ScanCtx s) {
  typedef typename KeyOf<LOUV, NK>::T K;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  const int64_t n = (int64_t)*s.small_cnt;
  int64_t n_act = 0, n_arcs = 0, n_cand = 0, n_def = 0, n_marcs = 0;
  for (int64_t q = warp; q < n; q += nwarps) {
    const int32_t h = s.small_list[q];
    const int32_t v = s.hub_list[h];
    if (!is_active(s, v)) continue;  // uniform within the warp
    const int32_t cur = s.C[v];
    const int64_t dv = LOUV ? s.degw[v] : 0;
    const int64_t volv = LOUV ? vol_of(s, v) : 0;
    const int64_t base = s.hub_tab[h];
    const int64_t cap = s.hub_cc[h];
    K bk = K(0);
    int32_t bc = NOCAND;
    bool hc = false;
    int64_t kc = 0;
    unsigned nl = 0;  // live entries seen by this lane
    constexpr int U = 4;  // slots per lane per batch, then their gathers
    for (int64_t e = lane; e < cap; e += U * 32) {
      int32_t c[U];
      int64_t k[U], sg[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int64_t x = e + (int64_t)j * 32;
        c[j] = -1;
        k[j] = 0;
        if (x < cap) hub_slot_read(s, base, x, c[j], k[j]);
      }
#pragma unroll
      for (int j = 0; j < U; ++j) sg[j] = (LOUV && c[j] >= 0 && k[j] != 0) ? sig_of<NK>(s, c[j]) : 0;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        if (c[j] < 0 || k[j] == 0) continue;
        ++n_cand;
        ++nl;
        if (c[j] == cur) {
          hc = true;
          kc = k[j];
          if (LOUV) continue;
        }
        const K key = cand_key_sg<LOUV, NK>(sg[j], k[j], dv, volv);
        if (better(key, c[j], bk, bc)) {
          bk = key;
          bc = c[j];
        }
      }
    }
    reduce_best(bk, bc, 32);
    const unsigned hm = __ballot_sync(FULL, hc);
    if (hm) kc = __shfl_sync(FULL, kc, __ffs(hm) - 1);
    nl = __reduce_add_sync(FULL, nl);
    if (lane == 0) {
      hub_decide<LOUV, NK>(s, h, v, cur, bk, bc, hm != 0, kc, volv, n_act, n_arcs, n_def, n_marcs);
      hub_maybe_shrink(s, h, cap, nl);
    }
  }
  flush_counters(s, B_HUB, n_act, n_arcs, n_cand, n_def, n_marcs);
}

// Every item scans HUB_SLICE histogram entries of one active hub (the hub's
// first ceil(cc / HUB_SLICE) items are listed); the last item of a hub to
// finish combines the partial bests and decides. Entries with weight 0
// (labels that left the neighbourhood) are not candidates.
template <bool LOUV, bool NK>
__global__ void __launch_bounds__(NT) k_hub_eval(ScanCtx s) {
  typedef typename KeyOf<LOUV, NK>::T K;
  __shared__ K red_k[NW];
  __shared__ int32_t red_c[NW];
  __shared__ int s_last;
  __shared__ unsigned s_live;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_live = 0;
  {
    const int64_t nb = (int64_t)*(volatile unsigned long long*)&s.hub_lcnt[0];
    for (int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x; q < nb; q += (int64_t)gridDim.x * NT) {
      const int32_t it = s.hub_blist[q];
      const int32_t h = s.hub_item_hub[it];
      if (s.hub_item_first[h] == it) s.hub_rb[h] = 0;
    }
  }
  __syncthreads();
  int64_t n_act = 0, n_arcs = 0, n_cand = 0, n_def = 0, n_marcs = 0;
  const int64_t n_ev = (int64_t)*s.ev_cnt;
  for (int64_t q = blockIdx.x; q < n_ev; q += gridDim.x) {
    const int64_t it = s.ev_list[q];
    const int32_t h = s.hub_ev_hub[it];
    const int32_t v = s.hub_list[h];
    if (!is_active(s, v)) continue;  // uniform within the CTA
    const int32_t cur = s.C[v];
    const int64_t dv = LOUV ? s.degw[v] : 0;
    const int64_t volv = LOUV ? vol_of(s, v) : 0;
    const int64_t base = s.hub_tab[h];
    const int64_t cap = s.hub_cc[h];
    const int64_t e0 = s.hub_ev_slot[it];
    const int64_t e1 = e0 + HUB_SLICE < cap ? e0 + HUB_SLICE : cap;
    K bk = K(0);
    int32_t bc = NOCAND;
    unsigned nl = 0;
    constexpr int HB = 6;  // slots per thread per batch: all loads, then all gathers, in flight together
    for (int64_t e = e0 + threadIdx.x; e < e1; e += HB * NT) {
      int32_t c[HB];
      int64_t k[HB], sg[HB];
#pragma unroll
      for (int j = 0; j < HB; ++j) {
        const int64_t x = e + (int64_t)j * NT;
        c[j] = -1;
        k[j] = 0;
        if (x < e1) hub_slot_read(s, base, x, c[j], k[j]);
      }
#pragma unroll
      for (int j = 0; j < HB; ++j) sg[j] = (LOUV && c[j] >= 0 && k[j] != 0) ? sig_of<NK>(s, c[j]) : 0;
#pragma unroll
      for (int j = 0; j < HB; ++j) {
        if (c[j] < 0 || k[j] == 0) continue;  // unused entry, or a label that left
        ++n_cand;
        ++nl;
        if (c[j] == cur) {
          s.hub_cur[h] = k[j];
          s.hub_hascur[h] = 1;
          if (LOUV) continue;
        }
        const K key = cand_key_sg<LOUV, NK>(sg[j], k[j], dv, volv);
        if (better(key, c[j], bk, bc)) {
          bk = key;
          bc = c[j];
        }
      }
    }
    reduce_best(bk, bc, 32);
    nl = __reduce_add_sync(FULL, nl);
    if (lane == 0) {
      red_k[wid] = bk;
      red_c[wid] = bc;
      if (nl) atomicAdd(&s_live, nl);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w2 = 1; w2 < NW; ++w2)
        if (better(red_k[w2], red_c[w2], bk, bc)) {
          bk = red_k[w2];
          bc = red_c[w2];
        }
      const i128 kk = (i128)bk;
      s.hub_part[3 * it] = (int64_t)(kk >> 64);
      s.hub_part[3 * it + 1] = (int64_t)(uint64_t)kk;
      s.hub_part[3 * it + 2] = bc;
      if (s_live) atomicAdd(&s.hub_live[h], (int)s_live);
      __threadfence();
      const int64_t nparts = (cap + HUB_SLICE - 1) / HUB_SLICE;
      s_last = atomicAdd(&s.hub_done[h], 1) == (int)(nparts - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      const volatile int64_t* part = s.hub_part;
      K fk = K(0);
      int32_t fc = NOCAND;
      const int64_t p0 = s.hub_ev_first[h], p1 = p0 + (cap + HUB_SLICE - 1) / HUB_SLICE;
      for (int64_t p = p0; p < p1; ++p) {
        const i128 pk = (i128)(((unsigned __int128)(uint64_t)part[3 * p] << 64) | (uint64_t)part[3 * p + 1]);
        const int32_t pc = (int32_t)part[3 * p + 2];
        if (better((K)pk, pc, fk, fc)) {
          fk = (K)pk;
          fc = pc;
        }
      }
      const bool hc = *((volatile int32_t*)&s.hub_hascur[h]) != 0;
      const int64_t kc = hc ? *((volatile int64_t*)&s.hub_cur[h]) : 0;
      hub_decide<LOUV, NK>(s, h, v, cur, fk, fc, hc, kc, volv, n_act, n_arcs, n_def, n_marcs);
      hub_maybe_shrink(s, h, cap, *(volatile int32_t*)&s.hub_live[h]);
      s.hub_live[h] = 0;
      s.hub_done[h] = 0;
      s.hub_cur[h] = 0;
      s.hub_hascur[h] = 0;
    }
    if (threadIdx.x == 0) s_live = 0;
    __syncthreads();
  }
  flush_counters(s, B_HUB, n_act, n_arcs, n_cand, n_def, n_marcs);
}

// ------------------------------------------------------------------ first round from rows
//
// Round 0 of a run or level that starts from singletons (C[v] = v, Sigma_tot
// = deg_w, every size 1) on a graph whose rows never repeat a column: the
// neighbour label u of arc (v, u) is u itself and k_{v,u} = w(v, u), so the
// decision is an argmax over v's row (LPA: largest w, then smallest u;
// Louvain: largest vol(V) w - deg_w(v) Sigma_tot[u], then smallest u) without
// label gathers or tables. v's own label has weight 0 (loops are not
// neighbours), so G of Eq. deltaQ equals the candidate key. PER threads work
// on a vertex (a sub-warp tile, a warp, or the whole CTA); the decision, the
// coin and the marking of a committed move's neighbours are those of the
// general scan. No hub histogram is built or updated here: round 0 counts as
// a heavy round, so every hub table is built at the start of round 1.
constexpr int FIRST_MARK = 100;  // profile marks of first-round launches: FIRST_MARK + bin

template <bool LOUV, class W, bool NK, int PER>
__global__ void __launch_bounds__(NT) k_first_round(ScanCtx s, const int32_t* __restrict__ list,
                                                    const unsigned long long* __restrict__ count_p, int bin) {
  typedef typename KeyOf<LOUV, NK>::T K;
  static_assert(PER == 4 || PER == 8 || PER == 16 || PER == 32 || PER == NT, "threads per vertex");
  constexpr int TW = PER < 32 ? PER : 32;  // width of the in-warp reduction
  constexpr int GPB = NT / PER;            // vertices per CTA and pass
  __shared__ K red_k[NW];
  __shared__ int32_t red_c[NW];
  __shared__ int32_t moved_to[GPB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gid = threadIdx.x / PER, gl = threadIdx.x % PER;
  const int64_t count = (int64_t)*count_p;
  int64_t n_act = 0, n_arcs = 0, n_cand = 0, n_def = 0, n_marcs = 0;
  // whole CTAs iterate together (the reductions need every lane)
  for (int64_t base = (int64_t)blockIdx.x * GPB; base < count; base += (int64_t)gridDim.x * GPB) {
    const int64_t i = base + gid;
    const bool valid = i < count;
    const int32_t v = valid ? list[i] : 0;
    const bool act = valid && is_active(s, v);
    int64_t beg = 0, end = 0, dv = 0, volv = 0;
    if (act) {
      beg = s.off[v];
      end = s.off[v + 1];
      if (LOUV) {
        dv = s.degw[v];
        volv = vol_of(s, v);
      }
    }
    K bk = K(0);
    int32_t bc = NOCAND;
    for (int64_t e = beg + gl; e < end; e += PER) {
      const int32_t u = s.cols[e];
      if (u == v) continue;
      const int64_t wt = W::get(s.w, e);
      const K key = LOUV ? cand_key<LOUV, NK>(s, u, wt, dv, volv) : K(wt);
      ++n_cand;
      if (better(key, u, bk, bc)) {
        bk = key;
        bc = u;
      }
    }
    reduce_best(bk, bc, TW);
    if constexpr (PER == NT) {
      if (lane == 0) {
        red_k[wid] = bk;
        red_c[wid] = bc;
      }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int w2 = 1; w2 < NW; ++w2)
          if (better(red_k[w2], red_c[w2], bk, bc)) {
            bk = red_k[w2];
            bc = red_c[w2];
          }
    }
    if (gl == 0) {
      bool moved = false;
      if (act) {
        const int32_t target = decide<LOUV, NK>(s, v, v, bk, bc, false, 0, volv);
        const int def = act_single(s, v, v, target);
        n_def += def;
        ++n_act;
        n_arcs += end - beg;
        moved = target != v && !def;
        if (moved) n_marcs += end - beg;
      }
      if constexpr (PER == NT) moved_to[0] = moved ? 1 : 0;
      else if (!moved) end = beg;  // nothing to mark
    }
    if constexpr (PER == NT) {
      __syncthreads();
      if (!moved_to[0]) end = beg;
      __syncthreads();
    } else {
      end = __shfl_sync(FULL, end, lane - gl);  // the tile leader's verdict
    }
    if (s.mark)  // the neighbours of a committed move are examined next round
      for (int64_t e = beg + gl; e < end; e += PER) flag_next(s, s.cols[e]);
  }
  flush_counters(s, bin, n_act, n_arcs, n_cand, n_def, n_marcs);
}

// ------------------------------------------------------------------ device-side round loop
//
// After round 0, the remaining rounds of a run or level can run as one
// captured CUDA graph: a conditional WHILE node whose body is one round. Every
// value the host loop decides per round lives in device memory instead: the
// round number (the coin reads it), whether this round's moves update the hub
// histograms, the trace row, the move totals and the stop test, which clears
// the loop condition.
struct DevLoop {
  int32_t round;    // the round being run
  int32_t hub_upd;  // this round's committed moves update the hub histograms
  int32_t max_iter;
  int32_t pad;
  long long prev_moves;
  long long total_moves;
  unsigned long long alive;  // per-graph stop: graphs still running after this round
};
constexpr int TRACE_W = 6;  // trace row: examined, arcs, moved, deferred, candidate pairs, moved arcs

__global__ void k_loop_begin(DevLoop* dl, int64_t n, int64_t div, int has_hubs) {
  dl->hub_upd = (has_hubs && dl->prev_moves * div > n) ? 0 : 1;
}

// A round whose moves did not update the hub histograms queues every hub for
// a rebuild at the start of the next one.
__global__ void k_queue_all(ScanCtx s, const DevLoop* dl) {
  if (dl->hub_upd) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < s.nhubs; h += stride) {
    s.hub_rb[h] = HUB_REBUILD;
    s.hub_flist_w[h] = (int32_t)h;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *s.hub_fcnt_w = (unsigned long long)s.nhubs;
}

// The hubs flagged this round become the list the next round's preparation reads.
__global__ void k_flist_carry(const int32_t* __restrict__ flist_w, const unsigned long long* fcnt_w,
                              int32_t* __restrict__ flist_r, unsigned long long* fcnt_r) {
  const int64_t nf = (int64_t)*(volatile const unsigned long long*)fcnt_w;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += stride) flist_r[i] = flist_w[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *fcnt_r = (unsigned long long)nf;
}

// Batched runs that stop per graph: a graph stops after its own round with at
// most `threshold` vertices wanting to move (moved + deferred).
__global__ void k_loop_freeze(const unsigned long long* __restrict__ gcnt, uint8_t* gfrozen, int32_t* grounds,
                              int64_t nb, DevLoop* dl, int64_t threshold) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long alive = 0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
    if (gfrozen[b]) continue;
    if ((int64_t)gcnt[b] <= threshold) {
      gfrozen[b] = 1;
      grounds[b] = dl->round + 1;
    } else {
      ++alive;
    }
  }
  if (alive) atomicAdd(&dl->alive, alive);
}

__global__ void k_loop_end(const unsigned long long* __restrict__ ctr, DevLoop* dl, long long* trace, int louv,
                           int64_t threshold, int per_graph, int64_t iso_add, cudaGraphConditionalHandle handle) {
  const long long moves = (long long)ctr[C_MOVES], deferred = (long long)ctr[C_DEFERRED];
  long long act = 0, arcs = 0, cands = 0;
  for (int b = 0; b < NBINS; ++b) {
    act += (long long)ctr[C_BIN0 + 3 * b];
    arcs += (long long)ctr[C_BIN0 + 3 * b + 1];
    cands += (long long)ctr[C_BIN0 + 3 * b + 2];
  }
  long long* t = trace + (int64_t)TRACE_W * dl->round;
  t[0] = act + iso_add;
  t[1] = arcs;
  t[2] = moves;
  t[3] = deferred;
  t[4] = cands;
  t[5] = (long long)ctr[C_MARCS];
  dl->prev_moves = moves;
  dl->total_moves += moves;
  const bool stop = per_graph ? dl->alive == 0 : (louv ? moves + deferred == 0 : moves + deferred <= threshold);
  dl->round += 1;
  if (stop || dl->round >= dl->max_iter) cudaGraphSetConditional(handle, 0);
}

// ------------------------------------------------------------------ frontier

struct BinBounds {
  int64_t b[NBINS + 1];
};

// The active vertices of a round into per-bin lists (bin b at act + b.b[b],
// order arbitrary; the scans do not depend on it); the hub bin's list holds
// hub numbers (k_hub_route turns them into evaluate work once the round's
// preparation has fixed every table's size). Whole warps iterate together
// for the match.
__global__ void __launch_bounds__(NT) k_compact(ScanCtx s, const int32_t* __restrict__ bin_list, BinBounds bb,
                                                int32_t* __restrict__ act, unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t total = bb.b[NBINS];
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t base = (int64_t)blockIdx.x * NT + (threadIdx.x & ~31); base < total; base += stride) {
    const int64_t i = base + lane;
    const bool valid = i < total;
    const int32_t v = valid ? bin_list[i] : 0;
    int bin = -1;
    if (valid && is_active(s, v)) {
      bin = 0;
      while (i >= bb.b[bin + 1]) ++bin;
    }
    const int key = bin;
    const unsigned peers = __match_any_sync(FULL, key);
    const int leader = __ffs(peers) - 1;
    unsigned long long p0 = 0;
    if (key >= 0 && lane == leader) p0 = atomicAdd(&cnt[key], (unsigned long long)__popc(peers));
    p0 = __shfl_sync(FULL, p0, leader);
    // hub h is the h-th entry of the hub bin
    if (key >= 0)
      act[bb.b[key] + (int64_t)p0 + __popc(peers & ((1u << lane) - 1u))] =
          key == B_HUB ? (int32_t)(i - bb.b[B_HUB]) : v;
  }
}

// The evaluate work of the hubs examined this round, by the size of their
// tables after this round's preparation: a hub with at most HUB_SMALL slots in
// use goes to the one-warp list, a larger one's first ceil(cc / HUB_SLICE)
// items to the item list. cnt[0] and cnt[1] count them (zeroed before).
__global__ void __launch_bounds__(NT) k_hub_route(ScanCtx s, int32_t* __restrict__ ev, int32_t* __restrict__ small,
                                                  unsigned long long* __restrict__ cnt) {
  const int64_t n = s.hub_act ? (int64_t)*s.hub_act_cnt : s.nhubs;
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += stride) {
    const int32_t h = s.hub_act ? s.hub_act[i] : (int32_t)i;
    const int64_t cc = s.hub_cc[h];
    if (cc <= HUB_SMALL) {
      small[atomicAdd(&cnt[1], 1ull)] = h;
    } else {
      const int64_t e0 = s.hub_ev_first[h], ne = (cc + HUB_SLICE - 1) / HUB_SLICE;
      const unsigned long long p = atomicAdd(&cnt[0], (unsigned long long)ne);
      for (int64_t j = 0; j < ne; ++j) ev[p + j] = (int32_t)(e0 + j);
    }
  }
}

// ------------------------------------------------------------------ apply

// Thread per committed move (vertex v: A -> c): the new label, and Sigma_tot
// and community sizes for Louvain. (The scan kernels flag the neighbours of
// their committed vertices and update neighbouring hub histograms; moved hubs
// are handled by k_hub_mark.)
// Add `d` to sigma[key] and `one` to csize[key] for every lane with key >= 0,
// one atomic pair per distinct key of the warp: popular target communities
// would otherwise serialise on one address.
__device__ __forceinline__ void warp_add_community(int64_t* sigma, int32_t* csize, int32_t key, int64_t d,
                                                   int32_t one, int64_t* stage) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(FULL, key);
  stage[lane] = d;
  __syncwarp();
  if (key >= 0 && (__ffs(peers) - 1) == lane) {
    int64_t sum = 0;
    unsigned m = peers;
    while (m) {
      sum += stage[__ffs(m) - 1];
      m &= m - 1;
    }
    atomicAdd((unsigned long long*)&sigma[key], (unsigned long long)sum);
    atomicAdd(&csize[key], one * __popc(peers));
  }
  __syncwarp();
}

template <bool LOUV>
__global__ void __launch_bounds__(NT) k_apply_state(ScanCtx s, const unsigned long long* __restrict__ nmoves_p,
                                                    int64_t* sigma, int32_t* csize, int32_t* C) {
  __shared__ int64_t stage[NW][32];
  const int64_t nmoves = (int64_t)*nmoves_p;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * NT;
  // whole warps iterate together (the match needs every lane)
  for (int64_t base = (int64_t)blockIdx.x * NT + wid * 32; base < nmoves; base += stride) {
    const int64_t m = base + lane;
    const bool ok = m < nmoves;
    int32_t v = 0, c = -1, A = -1;
    if (ok) {
      v = s.mv_v[m];
      c = s.mv_c[m];
      C[v] = c;
    }
    if (LOUV) {
      int64_t d = 0;
      if (ok) {
        A = s.mv_a[m];
        d = s.degw[v];
      }
      warp_add_community(sigma, csize, c, d, 1, stage[wid]);
      warp_add_community(sigma, csize, A, -d, -1, stage[wid]);
    }
  }
}

// Moved hubs, one queued item per HUB_CHUNK arcs: flag the neighbours and
// update the histograms of neighbouring hubs.
template <class W>
__global__ void __launch_bounds__(NT) k_hub_mark(ScanCtx s) {
  const int64_t nm = (int64_t)*(volatile unsigned long long*)&s.hub_lcnt[1];
  for (int64_t q = blockIdx.x; q < nm; q += gridDim.x) {
    const int32_t it = s.hub_mlist[q];
    const int32_t h = s.hub_item_hub[it];
    const int32_t A = s.hub_mv[3 * h + 1], c = s.hub_mv[3 * h + 2];
    const int32_t v = s.hub_list[h];
    const int64_t a0 = s.hub_item_arc[it];
    const int64_t rowend = s.off[v + 1];
    const int64_t end = a0 + HUB_CHUNK < rowend ? a0 + HUB_CHUNK : rowend;
    for (int64_t e = a0 + threadIdx.x; e < end; e += NT) {
      const int32_t u = s.cols[e];
      if (s.mark) flag_next(s, u);
      if (u == v) continue;
      hub_neighbour_moved(s, u, A, c, W::get(s.w, e));
    }
  }
}

__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = x;
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long x) { *p = x; }

__global__ void k_sigma32_all(const int64_t* __restrict__ sigma, int64_t n, uint32_t* __restrict__ s32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s32[i] = (uint32_t)sigma[i];
}

// After the moves of a round are applied: refresh the copies of the
// communities they touched (plain stores of the final values).
__global__ void k_sigma32_moves(const int32_t* __restrict__ mv_a, const int32_t* __restrict__ mv_c,
                                const unsigned long long* __restrict__ nmoves_p,
                                const int64_t* __restrict__ sigma, uint32_t* __restrict__ s32) {
  const int64_t nmoves = (int64_t)*nmoves_p;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < nmoves; m += stride) {
    const int32_t a = mv_a[m], c = mv_c[m];
    s32[a] = (uint32_t)sigma[a];
    s32[c] = (uint32_t)sigma[c];
  }
}

__global__ void k_iota_i32(int32_t* a, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = (int32_t)i;
}

__global__ void k_init_singletons(int32_t* C, int64_t* sigma, int32_t* csize,
                                  const int64_t* __restrict__ degw, int64_t n, int louv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    C[v] = (int32_t)v;
    if (louv) {
      sigma[v] = degw[v];
      csize[v] = 1;
    }
  }
}

__global__ void k_init_given(const int32_t* __restrict__ C, int64_t* sigma, int32_t* csize,
                             const int64_t* __restrict__ degw, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    atomicAdd((unsigned long long*)&sigma[C[v]], (unsigned long long)degw[v]);
    atomicAdd(&csize[C[v]], 1);
  }
}

unsigned grid_cap(int64_t blocks, int64_t cap = 152 * 16) {
  if (blocks < 1) blocks = 1;
  return (unsigned)(blocks < cap ? blocks : cap);
}

// CTAs of `kernel` resident on the device at once (occupancy x SMs), cached
// per kernel. Scan grids are capped to this: a grid-stride loop over one wave
// has no partly filled second wave.
int resident_ctas(const void* kernel, int nt, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nt, smem);
  const int r = std::max(1, per) * std::max(1, sms);
  cache[kernel] = r;
  return r;
}

template <class KERN>
unsigned wave_grid(KERN kernel, int nt, size_t smem, int64_t want) {
  return grid_cap(want, resident_ctas((const void*)kernel, nt, smem));
}

// Vertices per warp batch of k_scan_warp for a bin of cnt vertices: 32, or the
// largest power of two that still gives every resident warp a batch.
template <class KERN>
int warp_batch(KERN kernel, size_t smem, int64_t cnt) {
  const int64_t warps = (int64_t)resident_ctas((const void*)kernel, 256, smem) * 8;
  int vb = 32;
  while (vb > 1 && cnt < warps * vb) vb >>= 1;
  return vb;
}

// Group-kernel configurations: (GROUP threads per vertex, CTA size, table slots).
template <class V> constexpr size_t group_smem(int gpb, int cap, int ntb) {
  return (size_t)gpb * cap * (sizeof(V) + 4) + (size_t)(ntb / 32) * 32 * 8 + (size_t)gpb * cap * 2;
}
template <class V> constexpr size_t warp_smem() { return group_smem<V>(8, WARP_CAP_SLOTS, 256); }
template <class V> constexpr size_t blk1_smem() { return group_smem<V>(4, BLK1_CAP_SLOTS, 512); }
template <class V> constexpr size_t blk4_smem() { return group_smem<V>(1, BLK4_CAP_SLOTS, 512); }
template <class V> constexpr size_t hub_smem() { return group_smem<V>(1, HUB_CAP, HUB_NT); }

template <bool LOUV, class W, class V, bool NK>
int set_smem_attrs() {
  static std::atomic<bool> done{false};  // idempotent; threads may race here
  if (done) return CD_OK;
  CD_CHECK(cudaFuncSetAttribute(k_scan_warp<LOUV, W, V, NK>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)warp_smem<V>()));
  CD_CHECK(cudaFuncSetAttribute(k_scan_group<LOUV, W, V, 512, 512, BLK4_CAP_SLOTS, B_BLK4, false, NK>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)blk4_smem<V>()));
  CD_CHECK(cudaFuncSetAttribute(k_scan_group<LOUV, W, V, 128, 512, BLK1_CAP_SLOTS, B_BLK1, false, NK>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)blk1_smem<V>()));
  CD_CHECK(cudaFuncSetAttribute(k_hub_prepare, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HUB_PREP_SMEM));
  CD_CHECK(cudaFuncSetAttribute(k_hub_build_cl<W, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hub_cl_smem<0>()));
  CD_CHECK(cudaFuncSetAttribute(k_hub_build_cl<W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hub_cl_smem<1>()));
  CD_CHECK(cudaFuncSetAttribute(k_hub_build_cl<W, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hub_cl_smem<2>()));
  CD_CHECK(cudaFuncSetAttribute(k_hub_build_cl<W, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hub_cl_smem<3>()));
  CD_CHECK(cudaFuncSetAttribute(k_hub_build_cl<W, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hub_cl_smem<4>()));
  CD_CHECK(cudaFuncSetAttribute(k_hub_build<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)hub_smem<V>()));
  done = true;
  return CD_OK;
}

// Algorithmic bytes of one scan launch (per examined vertex: offset, own
// label, flag; per arc: column, neighbour label, weight; Louvain adds deg_w,
// Sigma_tot[A], sizes per vertex and one Sigma_tot gather per candidate).
double scan_bytes(bool louv, int wbytes, int64_t act, int64_t arcs, int64_t cands) {
  double b = (double)act * (8 + 4 + 1) + (double)arcs * (4 + 4 + wbytes);
  if (louv) b += (double)act * (8 + 8 + 8) + (double)cands * 8;
  return b;
}

constexpr int64_t CONC_LOUV_BYTES = (int64_t)64 << 20;  // half of the 129 MB L2, rounded down

// Scan kernels of different bins may run concurrently when none of them
// writes what another reads: hub histograms are then only read during the
// scans (their updates go to the log, applied after the join). fork() makes
// the auxiliary streams wait for everything enqueued so far on g->stream;
// join() makes g->stream wait for them.
struct BinStreams {
  cudaStream_t s[4];
  bool on = false;
};

// The auxiliary streams and their events belong to the calling host thread
// (created on its first use), so handles cost no stream creation and the
// server's worker threads never share them.
struct AuxStreams {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
  bool ok = false;
  AuxStreams() {
    ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 3 && ok; ++i)
      ok = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
};

AuxStreams& aux_streams() {
  static thread_local AuxStreams a;
  return a;
}

BinStreams fork_bins(cd_graph* g, bool concurrent) {
  BinStreams b;
  for (auto& x : b.s) x = g->stream;
  if (!concurrent || g->ktiming) return b;  // per-kernel events need the kernels one after another
  AuxStreams& a = aux_streams();
  if (!a.ok || cudaEventRecord(a.fork, g->stream) != cudaSuccess) return b;
  for (int i = 0; i < 3; ++i) {
    if (cudaStreamWaitEvent(a.s[i], a.fork, 0) != cudaSuccess) return b;
    b.s[i + 1] = a.s[i];
  }
  b.on = true;
  return b;
}

int join_bins(cd_graph* g, const BinStreams& b) {
  if (!b.on) return CD_OK;
  AuxStreams& a = aux_streams();
  for (int i = 0; i < 3; ++i) {
    CD_CHECK(cudaEventRecord(a.join[i], a.s[i]));
    CD_CHECK(cudaStreamWaitEvent(g->stream, a.join[i], 0));
  }
  return CD_OK;
}

// Launch the first round from rows over every bin.
template <bool LOUV, class W, bool NK>
int launch_first_round(cd_graph* g, ScanCtx& s, std::vector<std::pair<size_t, int>>& marks) {
  auto cnt = [&](int b) { return g->bin_start[b + 1] - g->bin_start[b]; };
  auto lst = [&](int b) { return (const int32_t*)g->bin_list + g->bin_start[b]; };
  auto dcnt = [&](int b) { return (const unsigned long long*)g->full_cnt + b; };
  static const int kname[NBINS] = {K_SCAN_T4, K_SCAN_T8, K_SCAN_T16, K_SCAN_T32, K_SCAN_WARP,
                                   K_SCAN_BLK128, K_SCAN_BLK512, K_HUB_EVAL};
  // stream of each bin: hubs, the 512- and 128-thread groups, the warp bin, the tiles
  static const int sidx[NBINS] = {0, 0, 0, 0, 3, 2, 2, 1};
  const BinStreams bs = fork_bins(g, !s.async_mode);
  for (int b = NBINS - 1; b >= 0; --b) {
    const int64_t c = cnt(b);
    if (c == 0) continue;
    const cudaStream_t st = bs.s[sidx[b]];
    {
      KTimer t(g, kname[b], 0.0, st);
      switch (b) {
        case B_T4: CD_LAUNCH((k_first_round<LOUV, W, NK, 4><<<grid_cap((c + 63) / 64), NT, 0, st>>>(s, lst(b), dcnt(b), b))); break;
        case B_T8: CD_LAUNCH((k_first_round<LOUV, W, NK, 8><<<grid_cap((c + 31) / 32), NT, 0, st>>>(s, lst(b), dcnt(b), b))); break;
        case B_T16: CD_LAUNCH((k_first_round<LOUV, W, NK, 16><<<grid_cap((c + 15) / 16), NT, 0, st>>>(s, lst(b), dcnt(b), b))); break;
        case B_HUB:
        case B_BLK4: CD_LAUNCH((k_first_round<LOUV, W, NK, NT><<<grid_cap(c), NT, 0, st>>>(s, lst(b), dcnt(b), b))); break;
        default: CD_LAUNCH((k_first_round<LOUV, W, NK, 32><<<grid_cap((c + NW - 1) / NW), NT, 0, st>>>(s, lst(b), dcnt(b), b))); break;
      }
    }
    if (g->ktiming) marks.push_back({g->pending.size() - 1, b + FIRST_MARK});  // first-round bytes
  }
  return join_bins(g, bs);
}

template <bool LOUV, bool NK>
int dispatch_first(cd_graph* g, ScanCtx& s, std::vector<std::pair<size_t, int>>& marks) {
  if (g->wkind == W_UNIT) return launch_first_round<LOUV, WUnit, NK>(g, s, marks);
  if (g->wkind == W_I32) return launch_first_round<LOUV, WI32, NK>(g, s, marks);
  return launch_first_round<LOUV, WI64, NK>(g, s, marks);
}

template <bool LOUV, class W, class V, bool NK>
int launch_round(cd_graph* g, ScanCtx& s, const int32_t* lists, const unsigned long long* counts,
                 std::vector<std::pair<size_t, int>>& marks) {
  int rc = set_smem_attrs<LOUV, W, V, NK>();
  if (rc) return rc;
  cudaStream_t st = g->stream;
  auto cnt = [&](int b) { return g->bin_start[b + 1] - g->bin_start[b]; };
  auto lst = [&](int b) { return lists + g->bin_start[b]; };
  auto dcnt = [&](int b) { return counts + b; };
  auto mark = [&](int b) { marks.push_back({g->pending.size() - 1, b}); };
  if (cnt(B_HUB) > 0) {
    {
      KTimer t(g, K_HUB_PREP);  // compactions, and clears of the tables rebuilt below
      CD_LAUNCH(k_hub_prepare<<<grid_cap(g->nhubs, 152 * 2), NT, HUB_PREP_SMEM, st>>>(s));
      // the examined hubs' evaluate work, by the table sizes the preparation left
      CD_CHECK(cudaMemsetAsync(g->act_cnt + NBINS, 0, 2 * sizeof(unsigned long long), st));
      CD_LAUNCH(k_hub_route<<<grid_cap((g->nhubs + NT - 1) / NT), NT, 0, st>>>(s, g->act_ev, g->act_small,
                                                                             g->act_cnt + NBINS));
    }
    if (g->ktiming) marks.push_back({g->pending.size() - 1, -2});
    {
      KTimer t(g, K_HUB_INSERT);  // the builds run only for hubs queued by the preparation
      CD_LAUNCH((k_hub_build_cl<W, 0><<<152 * 6, 256, hub_cl_smem<0>(), st>>>(s)));  // 6 CTAs per SM (registers)
      CD_LAUNCH((k_hub_build_cl<W, 1><<<456, HUB_NT, hub_cl_smem<1>(), st>>>(s)));
      CD_LAUNCH((k_hub_build_cl<W, 2><<<304, HUB_NT, hub_cl_smem<2>(), st>>>(s)));
      CD_LAUNCH((k_hub_build_cl<W, 3><<<304, HUB_NT, hub_cl_smem<3>(), st>>>(s)));
      CD_LAUNCH((k_hub_build_cl<W, 4><<<304, HUB_NT, hub_cl_smem<4>(), st>>>(s)));
      CD_LAUNCH(k_hub_build<W, V><<<grid_cap(g->hub_items, 152 * 3), HUB_NT, hub_smem<V>(), st>>>(s));
    }
    if (g->ktiming) marks.push_back({g->pending.size() - 1, -1});
  }
  // the scans of the bins, concurrently when the hub histograms are only read,
  // except for Louvain on a graph whose labels and Sigma_tot copy (8 bytes per
  // vertex) exceed half of L2: there the concurrent bins' random gathers
  // evict one another (measured at R-MAT 26: Louvain 2.62 s concurrent, 2.51 s
  // one bin after another; LPA 353 vs 366 ms and R-MAT 22 Louvain 164 vs
  // 183 ms in favour of running them concurrently)
  const bool conc = !LOUV || g->n * 8 <= CONC_LOUV_BYTES;
  const BinStreams bs = fork_bins(g, conc && !s.async_mode && (g->nhubs == 0 || s.hub_log != nullptr));
  if (cnt(B_HUB) > 0) {
    const cudaStream_t sh = bs.s[1];
    {
      KTimer t(g, K_HUB_EVAL, 0.0, sh);
      CD_LAUNCH(k_hub_eval_small<LOUV, NK><<<wave_grid(k_hub_eval_small<LOUV, NK>, NT, 0, (g->nhubs + NW - 1) / NW),
                                         NT, 0, sh>>>(s));
      CD_LAUNCH(k_hub_eval<LOUV, NK><<<grid_cap(g->hub_eval_items, 152 * 8), NT, 0, sh>>>(s));
    }
    if (g->ktiming) mark(B_HUB);
  }
  if (cnt(B_BLK4) > 0) {
    {
      KTimer t(g, K_SCAN_BLK512, 0.0, bs.s[2]);
      auto kern = k_scan_group<LOUV, W, V, 512, 512, BLK4_CAP_SLOTS, B_BLK4, false, NK>;
      CD_LAUNCH((kern<<<wave_grid(kern, 512, blk4_smem<V>(), cnt(B_BLK4)), 512, blk4_smem<V>(), bs.s[2]>>>(
          s, lst(B_BLK4), dcnt(B_BLK4))));
    }
    if (g->ktiming) mark(B_BLK4);
  }
  if (cnt(B_BLK1) > 0) {
    {
      KTimer t(g, K_SCAN_BLK128, 0.0, bs.s[2]);
      auto kern = k_scan_group<LOUV, W, V, 128, 512, BLK1_CAP_SLOTS, B_BLK1, false, NK>;
      CD_LAUNCH((kern<<<wave_grid(kern, 512, blk1_smem<V>(), (cnt(B_BLK1) + 3) / 4), 512, blk1_smem<V>(), bs.s[2]>>>(
          s, lst(B_BLK1), dcnt(B_BLK1))));
    }
    if (g->ktiming) mark(B_BLK1);
  }
  if (cnt(B_WARP) > 0) {
    {
      KTimer t(g, K_SCAN_WARP, 0.0, bs.s[3]);
      auto kern = k_scan_warp<LOUV, W, V, NK>;
      const int vb = warp_batch(kern, warp_smem<V>(), cnt(B_WARP));
      CD_LAUNCH((kern<<<wave_grid(kern, 256, warp_smem<V>(), (cnt(B_WARP) + 8 * vb - 1) / (8 * vb)), 256,
                        warp_smem<V>(), bs.s[3]>>>(s, lst(B_WARP), dcnt(B_WARP), vb)));
    }
    if (g->ktiming) mark(B_WARP);
  }
  if (cnt(B_T32) > 0) {
    {
      KTimer t(g, K_SCAN_T32);
      auto kern = k_scan_tile<32, LOUV, W, NK>;
      CD_LAUNCH(kern<<<wave_grid(kern, NT, 0, (cnt(B_T32) + NW - 1) / (NW)), NT, 0, st>>>(
          s, lst(B_T32), dcnt(B_T32), B_T32));
    }
    if (g->ktiming) mark(B_T32);
  }
  if (cnt(B_T16) > 0) {
    {
      KTimer t(g, K_SCAN_T16);
      auto kern = k_scan_tile<16, LOUV, W, NK>;
      CD_LAUNCH(kern<<<wave_grid(kern, NT, 0, (cnt(B_T16) + 2 * NW - 1) / (2 * NW)), NT, 0, st>>>(
          s, lst(B_T16), dcnt(B_T16), B_T16));
    }
    if (g->ktiming) mark(B_T16);
  }
  if (cnt(B_T8) > 0) {
    {
      KTimer t(g, K_SCAN_T8);
      auto kern = k_scan_tile<8, LOUV, W, NK>;
      CD_LAUNCH(kern<<<wave_grid(kern, NT, 0, (cnt(B_T8) + 4 * NW - 1) / (4 * NW)), NT, 0, st>>>(
          s, lst(B_T8), dcnt(B_T8), B_T8));
    }
    if (g->ktiming) mark(B_T8);
  }
  if (cnt(B_T4) > 0) {
    {
      KTimer t(g, K_SCAN_T4);
      auto kern = k_scan_tile<4, LOUV, W, NK>;
      CD_LAUNCH(kern<<<wave_grid(kern, NT, 0, (cnt(B_T4) + 8 * NW - 1) / (8 * NW)), NT, 0, st>>>(
          s, lst(B_T4), dcnt(B_T4), B_T4));
    }
    if (g->ktiming) mark(B_T4);
  }
  CD_CHECK(cudaGetLastError());
  return join_bins(g, bs);
}

template <bool LOUV, bool NK>
int dispatch_round(cd_graph* g, ScanCtx& s, const int32_t* lists, const unsigned long long* counts,
                   std::vector<std::pair<size_t, int>>& marks, bool v32) {
  if (g->wkind == W_UNIT)
    return v32 ? launch_round<LOUV, WUnit, uint32_t, NK>(g, s, lists, counts, marks)
               : launch_round<LOUV, WUnit, unsigned long long, NK>(g, s, lists, counts, marks);
  if (g->wkind == W_I32)
    return v32 ? launch_round<LOUV, WI32, uint32_t, NK>(g, s, lists, counts, marks)
               : launch_round<LOUV, WI32, unsigned long long, NK>(g, s, lists, counts, marks);
  return v32 ? launch_round<LOUV, WI64, uint32_t, NK>(g, s, lists, counts, marks)
             : launch_round<LOUV, WI64, unsigned long long, NK>(g, s, lists, counts, marks);
}

// The parts of a round's context that do not change from round to round.
ScanCtx static_ctx(cd_graph* g, const RunOpts& o, bool louv, bool use_s32, bool per_graph_stop) {
  ScanCtx s;
  s.hub_act = nullptr;
  s.hub_act_cnt = nullptr;
  s.off = g->off;
  s.cols = g->cols;
  s.w = g->w;
  s.degw = g->degw;
  s.vol = g->vol;
  s.C = g->C;
  s.sigma = g->sigma;
  s.sigma32 = use_s32 ? g->sigma32 : nullptr;
  s.csize = g->csize;
  s.all_active = o.use_frontier ? 0 : 1;
  s.mark = o.use_frontier ? 1 : 0;
  s.mv_v = g->mv_v;
  s.mv_c = g->mv_c;
  s.ctr = (unsigned long long*)g->ctr;
  s.status = g->status;
  s.seed = o.sched_seed;
  s.level = o.level;
  s.tie_keep = o.tie_keep_current;
  s.singleton_rule = o.singleton_rule;
  s.mv_a = g->mv_a;
  s.hub_list = g->bin_list + g->bin_start[B_HUB];
  s.hub_pref = g->hub_pref;
  s.hub_bits = g->hub_bits;
  s.hub_tab = g->hub_tab;
  s.hub_cc = g->hub_cc;
  s.hub_live = g->hub_live;
  s.hub_slot = g->hub_slot;
  s.hub_wide = g->hub_wide;
  s.hub_item_hub = g->hub_item_hub;
  s.hub_item_arc = g->hub_item_arc;
  s.hub_ev_hub = g->hub_ev_hub;
  s.hub_ev_slot = g->hub_ev_slot;
  s.hub_ev_first = g->hub_ev_first;
  s.hub_part = g->hub_part;
  s.hub_cur = g->hub_cur;
  s.hub_hascur = g->hub_hascur;
  s.hub_done = g->hub_done;
  s.hub_mv = g->hub_mv;
  s.hub_rb = g->hub_rb;
  s.hub_used = g->hub_used;
  s.hub_item_first = g->hub_item_first;
  s.hub_blist = g->hub_blist;
  s.hub_mlist = g->hub_mlist;
  s.hub_lcnt = g->hub_lcnt;
  s.hub_cl = g->hub_cl;
  s.hub_ccnt = g->hub_ccnt;
  s.n_items = g->hub_items;
  s.nhubs = g->nhubs;
  s.n_ev_items = g->hub_eval_items;
  s.async_mode = o.async_mode;
  s.C_w = g->C;
  s.sigma_w = louv ? g->sigma : nullptr;
  s.csize_w = g->csize;
  s.gid = o.batched ? g->gid : nullptr;
  s.gbase = o.batched ? g->gbase : nullptr;
  s.gvol = o.batched ? g->gvol : nullptr;
  s.gfrozen = o.batched ? g->gfrozen : nullptr;
  s.gcnt = per_graph_stop ? (unsigned long long*)g->gcnt : nullptr;
  s.round_p = nullptr;
  s.hub_upd_p = nullptr;
  s.hub_upd = 1;
  const bool log = g->nhubs > 0 && g->hub_log && !g->hub_wide && !o.async_mode;
  s.hub_log = log ? g->hub_log : nullptr;
  s.hub_log_cnt = log ? (unsigned long long*)g->ctr + C_HUB_LOG : nullptr;  // cleared with the counters
  s.hub_log_cap = log ? g->hub_log_cap : 0;
  return s;
}

// Rounds from `r0` on as one graph launch (see the device-side round loop
// above). fcur/fnxt: the flag bitmaps as left by the host loop; the hubs
// flagged by round r0 - 1 are in list (r0 - 1) & 1 of hub_flist.
int device_rounds(cd_graph* g, const RunOpts& o, bool louv, bool use_s32, bool per_graph_stop, int32_t r0,
                  uint32_t* fcur, uint32_t* fnxt, int64_t prev_moves, int64_t& total_moves, int32_t& rounds,
                  std::vector<int32_t>* graph_rounds) {
  const cudaStream_t st = g->stream;
  const int64_t n = g->n, nh = g->nhubs;
  const size_t fbytes = (size_t)((n + 31) / 32) * 4;
  DevLoop* dl = nullptr;
  long long* trace = nullptr;
  int32_t* grounds = nullptr;
  int rc;
  if ((rc = dev_alloc_t(&dl, 1, st)) || (rc = dev_alloc_t(&trace, (int64_t)TRACE_W * o.max_iter, st)) ||
      (per_graph_stop && (rc = dev_alloc_t(&grounds, g->nb, st)))) {
    dev_free(dl, st);
    dev_free(trace, st);
    return rc;
  }
  DevLoop h0{};
  h0.round = r0;
  h0.hub_upd = 1;
  h0.max_iter = o.max_iter;
  h0.prev_moves = prev_moves;
  h0.total_moves = total_moves;
  CD_CHECK(cudaMemcpyAsync(dl, &h0, sizeof(h0), cudaMemcpyHostToDevice, st));
  if (per_graph_stop)
    CD_CHECK(cudaMemcpyAsync(grounds, graph_rounds->data(), g->nb * 4, cudaMemcpyHostToDevice, st));
  // the flagged-hub lists: the body reads list A (what the previous round
  // wrote) and writes list B, then carries B to A
  int32_t* listA = nh > 0 ? g->hub_flist + ((r0 - 1) & 1) * nh : nullptr;
  int32_t* listB = nh > 0 ? g->hub_flist + (r0 & 1) * nh : nullptr;
  unsigned long long* cntA = nh > 0 ? g->hub_fcnt + ((r0 - 1) & 1) : nullptr;
  unsigned long long* cntB = nh > 0 ? g->hub_fcnt + (r0 & 1) : nullptr;
  ScanCtx s = static_ctx(g, o, louv, use_s32, per_graph_stop);
  s.flag_cur = fcur;
  s.flag_nxt = fnxt;
  s.round = r0;
  s.round_p = &dl->round;
  s.hub_upd_p = &dl->hub_upd;
  s.hub_flist_w = listB;
  s.hub_fcnt_w = cntB;
  s.hub_flist_r = listA;
  s.hub_fcnt_r = cntA;
  const bool compact = o.use_frontier && g->bin_start[NBINS] > 0;
  const int32_t* lists = compact ? g->act_list : g->bin_list;
  const unsigned long long* counts = compact ? g->act_cnt : g->full_cnt;
  s.ev_list = g->act_ev;
  s.ev_cnt = g->act_cnt + NBINS;
  s.small_list = g->act_small;
  s.small_cnt = g->act_cnt + NBINS + 1;
  s.hub_act = compact ? g->act_list + g->bin_start[B_HUB] : nullptr;
  s.hub_act_cnt = compact ? g->act_cnt + B_HUB : nullptr;
  const bool v32 = g->max_degw < ((int64_t)1 << 32);

  cudaGraph_t graph = nullptr, body = nullptr;
  cudaGraphExec_t exec = nullptr;
  // capture happens on a stream of this thread's own (never the legacy
  // default stream, which cannot be captured); the graph runs on g->stream
  static thread_local cudaStream_t cap = nullptr;
  cudaGraphConditionalHandle handle;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  };
  cudaError_t e = cap ? cudaSuccess : cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cleanup();
    dev_free(dl, st);
    dev_free(trace, st);
    dev_free(grounds, st);
    return set_cuda_error(e);
  }
  // one round, enqueued on the capture stream (the launch helpers use g->stream)
  g->stream = cap;
  rc = [&]() -> int {
    CD_CHECK(cudaMemsetAsync(g->ctr, 0, C_COUNT * sizeof(int64_t), cap));
    if (per_graph_stop) {
      CD_CHECK(cudaMemsetAsync(g->gcnt, 0, g->nb * sizeof(int64_t), cap));
      CD_CHECK(cudaMemsetAsync(&dl->alive, 0, sizeof(unsigned long long), cap));
    }
    if (o.use_frontier && n > 0) CD_CHECK(cudaMemsetAsync(fnxt, 0, fbytes, cap));
    if (nh > 0) {
      CD_CHECK(cudaMemsetAsync(g->hub_mv, 0, 3 * nh * sizeof(int32_t), cap));
      CD_CHECK(cudaMemsetAsync(g->hub_lcnt, 0, 2 * sizeof(unsigned long long), cap));
      CD_CHECK(cudaMemsetAsync(g->hub_ccnt, 0, HUB_NCLASS * sizeof(unsigned long long), cap));
      CD_CHECK(cudaMemsetAsync(cntB, 0, sizeof(unsigned long long), cap));
    }
    CD_LAUNCH(k_loop_begin<<<1, 1, 0, cap>>>(dl, n, louv ? HUB_SKIP_DIV : HUB_SKIP_DIV_LPA, nh > 0));
    if (compact) {
      CD_CHECK(cudaMemsetAsync(g->act_cnt, 0, (NBINS + 2) * sizeof(unsigned long long), cap));
      BinBounds bb;
      for (int b = 0; b <= NBINS; ++b) bb.b[b] = g->bin_start[b];
      CD_LAUNCH(k_compact<<<wave_grid(k_compact, NT, 0, (g->bin_start[NBINS] + NT - 1) / NT), NT, 0, cap>>>(
          s, g->bin_list, bb, g->act_list, g->act_cnt));
    }
    std::vector<std::pair<size_t, int>> marks;
    int rc2;
    if (louv) {
      if (g->vol < ((int64_t)1 << 31)) rc2 = dispatch_round<true, true>(g, s, lists, counts, marks, v32);
      else rc2 = dispatch_round<true, false>(g, s, lists, counts, marks, v32);
    } else {
      rc2 = dispatch_round<false, false>(g, s, lists, counts, marks, v32);
    }
    if (rc2) return rc2;
    const unsigned ga = grid_cap(n > 0 ? (n + NT - 1) / NT : 1, 152 * 8);
    if (!o.async_mode) {  // asynchronous moves were applied when made
      if (louv) {
        CD_LAUNCH(k_apply_state<true><<<ga, NT, 0, cap>>>(s, s.ctr + C_MOVES, g->sigma, g->csize, g->C));
        if (use_s32)
          CD_LAUNCH(k_sigma32_moves<<<ga, NT, 0, cap>>>(g->mv_a, g->mv_c, s.ctr + C_MOVES, g->sigma, g->sigma32));
      } else {
        CD_LAUNCH(k_apply_state<false><<<ga, NT, 0, cap>>>(s, s.ctr + C_MOVES, g->sigma, g->csize, g->C));
      }
    }
    if (nh > 0) {
      const unsigned gh = grid_cap(g->hub_items, 152 * 8);
      if (g->wkind == W_UNIT) CD_LAUNCH(k_hub_mark<WUnit><<<gh, NT, 0, cap>>>(s));
      else if (g->wkind == W_I32) CD_LAUNCH(k_hub_mark<WI32><<<gh, NT, 0, cap>>>(s));
      else CD_LAUNCH(k_hub_mark<WI64><<<gh, NT, 0, cap>>>(s));
      if (s.hub_log) CD_LAUNCH(k_hub_apply_log<<<152 * 8, NT, 0, cap>>>(s));  // no records when not updating
      CD_LAUNCH(k_queue_all<<<grid_cap((nh + NT - 1) / NT), NT, 0, cap>>>(s, dl));
      CD_LAUNCH(k_flist_carry<<<grid_cap((nh + NT - 1) / NT), NT, 0, cap>>>(listB, cntB, listA, cntA));
    }
    if (per_graph_stop)
      CD_LAUNCH(k_loop_freeze<<<grid_cap((g->nb + NT - 1) / NT), NT, 0, cap>>>(
          (const unsigned long long*)g->gcnt, g->gfrozen, grounds, g->nb, dl, o.threshold));
    CD_LAUNCH(k_loop_end<<<1, 1, 0, cap>>>(s.ctr, dl, trace, louv ? 1 : 0, o.threshold, per_graph_stop ? 1 : 0,
                                           o.use_frontier ? 0 : g->n_isolated, handle));
    if (o.use_frontier && n > 0) CD_CHECK(cudaMemcpyAsync(fcur, fnxt, fbytes, cudaMemcpyDeviceToDevice, cap));
    CD_CHECK(cudaGetLastError());
    return CD_OK;
  }();
  g->stream = st;
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cap, &captured);
  if (!rc && e != cudaSuccess) rc = set_cuda_error(e);
  if (!rc) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) rc = set_cuda_error(e);
    else note_launch();
  }
  DevLoop hd{};
  std::vector<long long> ht;
  if (!rc) {
    ht.resize((size_t)TRACE_W * o.max_iter);
    CD_CHECK(cudaMemcpyAsync(&hd, dl, sizeof(hd), cudaMemcpyDeviceToHost, st));
    CD_CHECK(cudaMemcpyAsync(ht.data(), trace, ht.size() * 8, cudaMemcpyDeviceToHost, st));
    if (per_graph_stop)
      CD_CHECK(cudaMemcpyAsync(graph_rounds->data(), grounds, g->nb * 4, cudaMemcpyDeviceToHost, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = CD_ECUDA;
  }
  cleanup();
  dev_free(dl, st);
  dev_free(trace, st);
  dev_free(grounds, st);
  if (rc) return rc;
  for (int32_t r = r0; r < hd.round; ++r) {
    const long long* t = ht.data() + (size_t)TRACE_W * r;
    cd_round_trace tr;
    tr.level = o.level;
    tr.round = r;
    tr.active = t[0];
    tr.arcs = t[1];
    tr.moved = t[2];
    tr.deferred = t[3];
    tr.cands = t[4];
    tr.moved_arcs = t[5];
    tr.scan_ms = tr.round_ms = 0.f;
    g->trace.push_back(tr);
  }
  total_moves = hd.total_moves;
  rounds = hd.round;
  return CD_OK;
}

int run_rounds(cd_graph* g, const RunOpts& o, bool louv, int64_t* moves_out, int32_t* rounds_out,
               std::vector<int32_t>* graph_rounds = nullptr) {
  cudaStream_t st = g->stream;
  const int64_t n = g->n;
  const bool per_graph_stop = o.batched && graph_rounds != nullptr;
  std::vector<int64_t> h_gcnt;
  std::vector<uint8_t> h_frozen;
  if (per_graph_stop) {
    graph_rounds->assign(g->nb, o.max_iter);
    h_gcnt.resize(g->nb);
    h_frozen.assign(g->nb, 0);
    CD_CHECK(cudaMemsetAsync(g->gfrozen, 0, g->nb, st));
  }
  int rc = CD_OK;
  if (g->nhubs > 0) {  // every histogram is built from the starting labels in round 0
    CD_LAUNCH(k_fill_i32<<<grid_cap((g->nhubs + NT - 1) / NT), NT, 0, st>>>(g->hub_rb, g->nhubs, 1));
    CD_LAUNCH(k_iota_i32<<<grid_cap((g->nhubs + NT - 1) / NT), NT, 0, st>>>(g->hub_flist + g->nhubs, g->nhubs));
    const unsigned long long nh = (unsigned long long)g->nhubs;
    CD_CHECK(cudaMemcpyAsync(g->hub_fcnt + 1, &nh, sizeof(nh), cudaMemcpyHostToDevice, st));
    CD_CHECK(cudaStreamSynchronize(st));  // nh lives on this stack frame
  }
  uint32_t* fcur = g->flag[0];
  uint32_t* fnxt = g->flag[1];
  const size_t fbytes = (size_t)((n + 31) / 32) * 4;  // bitmap words
  if (o.use_frontier && n > 0) CD_CHECK(cudaMemsetAsync(fcur, 0xff, fbytes, st));
  const int wbytes = g->wkind == W_UNIT ? 0 : g->wkind == W_I32 ? 4 : 8;
  int64_t total_moves = 0;
  int64_t prev_moves = -1;
  // 32-bit Sigma_tot copy for the gathers (synchronous Louvain, vol(V) < 2^31)
  const bool use_s32 = louv && !o.async_mode && g->vol < ((int64_t)1 << 31) && n > 0;
  if (use_s32) {
    if (!g->sigma32) {
      int rc2 = dev_alloc_t(&g->sigma32, n, st);
      if (rc2) return rc2;
    }
    CD_LAUNCH(k_sigma32_all<<<grid_cap((n + NT - 1) / NT), NT, 0, st>>>(g->sigma, n, g->sigma32));
  }
  // round 0 from the rows when every vertex starts alone and no row repeats a
  // column (the asynchronous mode keeps the general scan)
  const bool first_rows = o.singleton_start && g->cols_distinct && !o.async_mode;
  int32_t rounds = 0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (g->timing)
    for (auto& e : ev) cudaEventCreate(&e);
  // rounds after the first as one captured graph (a device-side loop) unless
  // per-round events are wanted
  const bool dev_loop = o.device_loop && !g->timing && (o.batched || o.device_loop_all);
  for (int32_t r = 0; r < o.max_iter && rc == CD_OK; ++r) {
    if (r > 0 && dev_loop) {
      rc = device_rounds(g, o, louv, use_s32, per_graph_stop, r, fcur, fnxt, prev_moves, total_moves, rounds,
                         graph_rounds);
      break;
    }
    if (g->timing) cudaEventRecord(ev[0], st);
    CD_CHECK(cudaMemsetAsync(g->ctr, 0, C_COUNT * sizeof(int64_t), st));
    if (per_graph_stop) CD_CHECK(cudaMemsetAsync(g->gcnt, 0, g->nb * sizeof(int64_t), st));
    if (o.use_frontier && n > 0) CD_CHECK(cudaMemsetAsync(fnxt, 0, fbytes, st));
    if (g->nhubs > 0) {
      CD_CHECK(cudaMemsetAsync(g->hub_mv, 0, 3 * g->nhubs * sizeof(int32_t), st));
      CD_CHECK(cudaMemsetAsync(g->hub_lcnt, 0, 2 * sizeof(unsigned long long), st));
      CD_CHECK(cudaMemsetAsync(g->hub_ccnt, 0, HUB_NCLASS * sizeof(unsigned long long), st));
      CD_CHECK(cudaMemsetAsync(g->hub_fcnt + (r & 1), 0, sizeof(unsigned long long), st));
    }
    ScanCtx s = static_ctx(g, o, louv, use_s32, per_graph_stop);
    s.flag_cur = fcur;
    s.flag_nxt = fnxt;
    s.round = r;
    s.hub_flist_w = g->hub_flist ? g->hub_flist + (r & 1) * g->nhubs : nullptr;
    s.hub_fcnt_w = g->hub_fcnt ? g->hub_fcnt + (r & 1) : nullptr;
    s.hub_flist_r = g->hub_flist ? g->hub_flist + ((r + 1) & 1) * g->nhubs : nullptr;
    s.hub_fcnt_r = g->hub_fcnt ? g->hub_fcnt + ((r + 1) & 1) : nullptr;
    // In a round that moves many vertices (the first of a run or level, or
    // after one that moved more than 1/HUB_SKIP_DIV of them, 1/4 for LPA) the hub
    // histograms are not updated move by move: every hub is rebuilt from its
    // row at the start of the next round instead, which costs less than that
    // many scattered updates.
    const bool skip_upd =
        g->nhubs > 0 && (r == 0 || prev_moves * (louv ? HUB_SKIP_DIV : HUB_SKIP_DIV_LPA) > n);
    s.hub_upd = skip_upd ? 0 : 1;
    // the round's work lists: every listed vertex in round 0 (or without a
    // frontier), else the active ones, compacted
    const int32_t* lists = g->bin_list;
    const unsigned long long* counts = g->full_cnt;
    s.ev_list = g->act_ev;
    s.ev_cnt = g->act_cnt + NBINS;
    s.small_list = g->act_small;
    s.small_cnt = g->act_cnt + NBINS + 1;
    s.hub_act = nullptr;
    s.hub_act_cnt = nullptr;
    if (o.use_frontier && r > 0 && g->bin_start[NBINS] > 0) {
      KTimer t(g, K_FRONTIER, (double)g->bin_start[NBINS] * (4 + 1 + 4));
      CD_CHECK(cudaMemsetAsync(g->act_cnt, 0, (NBINS + 2) * sizeof(unsigned long long), st));
      BinBounds bb;
      for (int b = 0; b <= NBINS; ++b) bb.b[b] = g->bin_start[b];
      CD_LAUNCH(k_compact<<<wave_grid(k_compact, NT, 0, (g->bin_start[NBINS] + NT - 1) / NT), NT, 0, st>>>(
          s, g->bin_list, bb, g->act_list, g->act_cnt));
      lists = g->act_list;
      counts = g->act_cnt;
      s.hub_act = g->act_list + g->bin_start[B_HUB];
      s.hub_act_cnt = g->act_cnt + B_HUB;
    }
    std::vector<std::pair<size_t, int>> marks;
    const bool v32 = g->max_degw < ((int64_t)1 << 32);
    if (r == 0 && first_rows) {
      if (!louv) rc = dispatch_first<false, false>(g, s, marks);
      else if (g->vol < ((int64_t)1 << 31)) rc = dispatch_first<true, true>(g, s, marks);
      else rc = dispatch_first<true, false>(g, s, marks);
    } else if (louv) {
      // Louvain candidate keys vol(V) k - deg_w(v) Sigma_tot need 128 bits in
      // general; when vol(V) < 2^31 each product is < 2^62 and they fit in 64
      if (g->vol < ((int64_t)1 << 31)) rc = dispatch_round<true, true>(g, s, lists, counts, marks, v32);
      else rc = dispatch_round<true, false>(g, s, lists, counts, marks, v32);
    } else {
      rc = dispatch_round<false, false>(g, s, lists, counts, marks, v32);
    }
    if (rc) break;
    if (g->timing) cudaEventRecord(ev[1], st);
    CD_CHECK(cudaMemcpyAsync(g->h_ctr, g->ctr, C_COUNT * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (per_graph_stop)
      CD_CHECK(cudaMemcpyAsync(h_gcnt.data(), g->gcnt, g->nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CD_CHECK(cudaStreamSynchronize(st));
    const int64_t* h = g->h_ctr;
    const int64_t moves = h[C_MOVES], deferred = h[C_DEFERRED];
    int64_t act = 0, arcs = 0, cands = 0;
    for (int b = 0; b < NBINS; ++b) {
      act += h[C_BIN0 + 3 * b];
      arcs += h[C_BIN0 + 3 * b + 1];
      cands += h[C_BIN0 + 3 * b + 2];
    }
    for (auto& mk : marks) {
      const int b = mk.second;
      const int64_t ab = b >= 0 ? h[C_BIN0 + 3 * b] : 0;
      const int64_t rb = h[C_BIN0 + 3 * B_HUB + 1], cb = b >= 0 ? h[C_BIN0 + 3 * b + 2] : 0;
      double bytes;
      if (b >= FIRST_MARK) {  // first round from rows: no label gathers
        const int fb = b - FIRST_MARK;
        const int64_t fa = h[C_BIN0 + 3 * fb], farcs = h[C_BIN0 + 3 * fb + 1], fc = h[C_BIN0 + 3 * fb + 2];
        bytes = (double)fa * (8 + 4 + 1) + (double)farcs * (4 + wbytes) + (louv ? (double)fa * 24 + (double)fc * 8 : 0.0);
      } else if (b == -1)  // hub table builds: the arcs they read, the slots they wrote
        bytes = (double)h[C_HUB_BARCS] * (4 + 4 + wbytes) + (double)h[C_HUB_BSLOTS] * 8;
      else if (b == -2)  // hub preparation: slots cleared, or read and written by compactions; the route
        bytes = (double)h[C_HUB_PSLOTS] * 8 + (double)g->nhubs * 8;
      else if (b == B_HUB)  // hub evaluate: the candidates of every active hub
        bytes = (double)cb * (12 + 12 + (louv ? 8 : 0)) + (double)ab * (8 + 4);
      else
        bytes = scan_bytes(louv, wbytes, ab, h[C_BIN0 + 3 * b + 1], cb);
      g->pending_bytes[mk.first] = bytes;
    }
    if (moves > 0) {
      if (!o.async_mode) {  // asynchronous moves were applied when made
        KTimer t(g, K_APPLY, (double)moves * (8 + 4 + (louv ? 8 + 16 + 8 : 0)));
        const unsigned gt = grid_cap((moves + NT - 1) / NT);
        if (louv) {
          CD_LAUNCH(k_apply_state<true><<<gt, NT, 0, st>>>(s, s.ctr + C_MOVES, g->sigma, g->csize, g->C));
          if (use_s32)
            CD_LAUNCH(k_sigma32_moves<<<gt, NT, 0, st>>>(g->mv_a, g->mv_c, s.ctr + C_MOVES, g->sigma, g->sigma32));
        }
        else
          CD_LAUNCH(k_apply_state<false><<<gt, NT, 0, st>>>(s, s.ctr + C_MOVES, g->sigma, g->csize, g->C));
      }
      if (g->nhubs > 0) {
        // flags and logged updates of the moved hubs' arcs (column 4, flag 1), and every logged
        // update (record 16, two slots read and written 32)
        KTimer t(g, K_HUB_MARK, (double)h[C_HUB_MARCS] * 5 + (double)h[C_HUB_LOG] * (16 + 16 + 32));
        const unsigned gh = grid_cap(g->hub_items, 152 * 8);
        if (g->wkind == W_UNIT) CD_LAUNCH(k_hub_mark<WUnit><<<gh, NT, 0, st>>>(s));
        else if (g->wkind == W_I32) CD_LAUNCH(k_hub_mark<WI32><<<gh, NT, 0, st>>>(s));
        else CD_LAUNCH(k_hub_mark<WI64><<<gh, NT, 0, st>>>(s));
        if (s.hub_log && !skip_upd) CD_LAUNCH(k_hub_apply_log<<<152 * 8, NT, 0, st>>>(s));
      }
      CD_CHECK(cudaGetLastError());
    }
    if (skip_upd) {  // queue every hub for a rebuild at the start of the next round
      CD_LAUNCH(k_fill_i32<<<grid_cap((g->nhubs + NT - 1) / NT), NT, 0, st>>>(g->hub_rb, g->nhubs, 1));
      CD_LAUNCH(k_iota_i32<<<grid_cap((g->nhubs + NT - 1) / NT), NT, 0, st>>>(g->hub_flist + (r & 1) * g->nhubs,
                                                                           g->nhubs));
      CD_LAUNCH(k_set_u64<<<1, 1, 0, st>>>(g->hub_fcnt + (r & 1), (unsigned long long)g->nhubs));
    }
    prev_moves = moves;
    cd_round_trace tr;
    tr.level = o.level;
    tr.round = r;
    tr.active = act + ((r == 0 || !o.use_frontier) ? g->n_isolated : 0);
    tr.arcs = arcs;
    tr.moved = moves;
    tr.deferred = deferred;
    tr.cands = cands;
    tr.moved_arcs = h[C_MARCS];
    tr.scan_ms = tr.round_ms = 0.f;
    if (g->timing) {
      cudaEventRecord(ev[2], st);
      CD_CHECK(cudaEventSynchronize(ev[2]));
      cudaEventElapsedTime(&tr.scan_ms, ev[0], ev[1]);
      cudaEventElapsedTime(&tr.round_ms, ev[0], ev[2]);
    }
    g->trace.push_back(tr);
    total_moves += moves;
    rounds = r + 1;
    std::swap(fcur, fnxt);
    bool stop = louv ? (moves + deferred == 0) : (moves + deferred <= o.threshold);
    if (per_graph_stop) {  // a graph stops after its own round with dN <= threshold
      bool newly = false, all = true;
      for (int64_t b = 0; b < g->nb; ++b) {
        if (h_frozen[b]) continue;
        if (h_gcnt[b] <= o.threshold) {
          h_frozen[b] = 1;
          (*graph_rounds)[b] = r + 1;
          newly = true;
        } else {
          all = false;
        }
      }
      if (newly) CD_CHECK(cudaMemcpyAsync(g->gfrozen, h_frozen.data(), g->nb, cudaMemcpyHostToDevice, st));
      stop = all;
    }
    if (stop) break;
  }
  if (g->timing)
    for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  int32_t stw = 0;
  CD_CHECK(cudaMemcpyAsync(&stw, g->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CD_CHECK(cudaStreamSynchronize(st));
  if (stw) return stw;
  if (moves_out) *moves_out = total_moves;
  if (rounds_out) *rounds_out = rounds;
  return profile_flush(g);
}

}  // namespace

int run_lpa(cd_graph* g, const RunOpts& o, int32_t* rounds_out) {
  int rc = ensure_run_state(g);
  if (rc) return rc;
  if (g->n > 0)
    CD_LAUNCH(k_init_singletons<<<grid_cap((g->n + NT - 1) / NT), NT, 0, g->stream>>>(g->C, g->sigma, g->csize,
                                                                            g->degw, g->n, 0));
  CD_CHECK(cudaGetLastError());
  RunOpts os = o;
  os.singleton_start = true;
  return run_rounds(g, os, false, nullptr, rounds_out);
}

int run_lpa_batched(cd_graph* g, const RunOpts& o, std::vector<int32_t>& rounds) {
  int rc = ensure_run_state(g);
  if (rc) return rc;
  if (g->n > 0)
    CD_LAUNCH(k_init_singletons<<<grid_cap((g->n + NT - 1) / NT), NT, 0, g->stream>>>(g->C, g->sigma, g->csize,
                                                                                      g->degw, g->n, 0));
  CD_CHECK(cudaGetLastError());
  RunOpts ob = o;
  ob.batched = true;
  ob.singleton_start = true;
  return run_rounds(g, ob, false, nullptr, nullptr, &rounds);
}

int run_local_move(cd_graph* g, const RunOpts& o, int init_given, int64_t* moves_out,
                   int32_t* rounds_out) {
  int rc = ensure_run_state(g);
  if (rc) return rc;
  cudaStream_t st = g->stream;
  if (g->n > 0) {
    if (!init_given) {
      CD_LAUNCH(k_init_singletons<<<grid_cap((g->n + NT - 1) / NT), NT, 0, st>>>(g->C, g->sigma, g->csize,
                                                                       g->degw, g->n, 1));
    } else {
      CD_CHECK(cudaMemsetAsync(g->sigma, 0, g->n * sizeof(int64_t), st));
      CD_CHECK(cudaMemsetAsync(g->csize, 0, g->n * sizeof(int32_t), st));
      CD_LAUNCH(k_init_given<<<grid_cap((g->n + NT - 1) / NT), NT, 0, st>>>(g->C, g->sigma, g->csize, g->degw,
                                                                  g->n));
    }
  }
  CD_CHECK(cudaGetLastError());
  RunOpts os = o;
  os.singleton_start = !init_given;
  return run_rounds(g, os, true, moves_out, rounds_out);
}

RunOpts opts_from(const cd_params* p, int32_t level) {
  RunOpts o;
  o.max_iter = p->max_iter;
  o.threshold = p->threshold;
  o.tie_keep_current = p->tie_keep_current;
  o.singleton_rule = p->singleton_rule;
  o.use_frontier = p->use_frontier;
  o.sched_seed = p->sched_seed;
  o.level = level;
  o.async_mode = p->asynchronous ? 1 : 0;
  o.device_loop = p->device_loop != 0;
  o.device_loop_all = p->device_loop == 2;
  return o;
}

int begin_run(cd_graph* g, const cd_params* p) {
  if (!g || !p || p->max_iter < 0 || p->max_iter > 65535 || p->max_levels < 0 ||
      p->max_levels > 32767)
    return CD_EINVAL;
  g->timing = p->timing != 0;
  g->ktiming = p->timing == 1;
  g->trace.clear();
  profile_reset(g);
  return CD_OK;
}

}  // namespace cd

using namespace cd;

extern "C" {

int cd_lpa_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
               int32_t* rounds_out) {
  int rc = begin_run(g, p);
  if (rc) return rc;
  if (!labels_out && g->n > 0) return CD_EINVAL;
  rc = run_lpa(g, opts_from(p, 0), rounds_out);
  if (rc) return rc;
  if (g->n > 0)
    CD_CHECK(cudaMemcpyAsync(labels_out, g->C, g->n * sizeof(int32_t),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
  CD_CHECK(cudaStreamSynchronize(g->stream));
  return CD_OK;
}

int cd_louvain_local_move(cd_graph* g, const cd_params* p, int32_t* labels_io, int init_given,
                          int on_device, int64_t* moves_out, int32_t* rounds_out) {
  int rc = begin_run(g, p);
  if (rc) return rc;
  if (!labels_io && g->n > 0) return CD_EINVAL;
  if ((rc = ensure_run_state(g))) return rc;
  if (init_given && g->n > 0) {
    CD_CHECK(cudaMemcpyAsync(g->C, labels_io, g->n * sizeof(int32_t),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    if ((rc = check_labels(g, g->C))) return rc;
  }
  rc = run_local_move(g, opts_from(p, 0), init_given, moves_out, rounds_out);
  if (rc) return rc;
  if (g->n > 0)
    CD_CHECK(cudaMemcpyAsync(labels_io, g->C, g->n * sizeof(int32_t),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
  CD_CHECK(cudaStreamSynchronize(g->stream));
  return CD_OK;
}

int cd_graph_set_bins(cd_graph* g, int32_t t_warp, int32_t t_hub) {
  if (!g) return CD_EINVAL;
  return rebin(g, t_warp, t_hub);
}

int cd_autotune(cd_graph* g, const cd_params* p, int32_t rounds, int32_t* t_warp_out, int32_t* t_hub_out) {
  if (!g || !p || rounds < 1) return CD_EINVAL;
  static const int tw[] = {64, 128, 256};
  static const int th[] = {512, 1024, 2048, 4096};
  int rc = ensure_run_state(g);
  if (rc) return rc;
  cudaEvent_t a, b;
  CD_CHECK(cudaEventCreate(&a));
  CD_CHECK(cudaEventCreate(&b));
  float best = -1.f;
  int bw = g->t_warp, bh = g->t_hub;
  const bool timing = g->timing, ktiming = g->ktiming;
  g->timing = g->ktiming = false;
  for (int i = 0; i < 3 && !rc; ++i)
    for (int j = 0; j < 4 && !rc; ++j) {
      if (th[j] < tw[i]) continue;
      if ((rc = rebin(g, tw[i], th[j]))) break;
      RunOpts o = opts_from(p, 0);
      o.max_iter = rounds;
      cudaEventRecord(a, g->stream);
      rc = run_lpa(g, o, nullptr);
      if (!rc) rc = run_local_move(g, o, 0, nullptr, nullptr);
      cudaEventRecord(b, g->stream);
      if (rc) break;
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (best < 0.f || ms < best) {
        best = ms;
        bw = tw[i];
        bh = th[j];
      }
    }
  g->timing = timing;
  g->ktiming = ktiming;
  g->trace.clear();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if ((rc = rebin(g, bw, bh))) return rc;
  if (t_warp_out) *t_warp_out = bw;
  if (t_hub_out) *t_hub_out = bh;
  return CD_OK;
}

}  // extern "C"
