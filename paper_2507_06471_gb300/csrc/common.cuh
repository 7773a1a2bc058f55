// Internal declarations of libcdgpu (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cdgpu.h"

namespace cd {

typedef __int128 i128;
constexpr unsigned FULL = 0xffffffffu;
constexpr int32_t EMPTY = -1;        // empty hash slot (labels are >= 0)
constexpr int32_t NOCAND = INT32_MAX;  // "no candidate" community id

// Degree bins of the scan (degree = row length, loops included). Vertices
// above BLOCK_MAX ("hubs") keep persistent label histograms instead of being
// rescanned every round.
enum Bin { B_T4 = 0, B_T8, B_T16, B_T32, B_WARP, B_BLK1, B_BLK4, B_HUB, NBINS };
constexpr int WARP_MAX = 256;    // a warp per vertex, table <= 512 slots
constexpr int BLK1_MAX = 1024;   // 128 threads per vertex, table <= 2048 slots
constexpr int BLK4_MAX = 4096;   // a whole 512-thread CTA per vertex, table <= 8192 slots
constexpr int BLOCK_MAX = 1024;  // default hub threshold (largest degree rescanned every round)
// A coarse graph (a Louvain level after the first) of at least COARSE_HUB_ARCS
// arcs takes the lower hub threshold COARSE_T_HUB unless the thresholds were
// set on the graph it came from: such levels run many rounds that move few
// vertices, where a persistent histogram costs less than rescanning a row of
// 513..1024 arcs (measured: R-MAT 24 and 26 coarse levels 4-6% faster; R-MAT 22
// no change; a 1M-vertex LFR-style graph, whose coarse graphs are far smaller,
// 50% slower with the lower threshold, hence the size condition).
constexpr int64_t COARSE_HUB_ARCS = (int64_t)1 << 27;
constexpr int COARSE_T_HUB = 512;
// The runtime bin boundaries t_warp (warp vs 128-thread group) and t_hub
// (group vs hub histogram) may be lowered below these capacities (autotuner).
constexpr int HUB_CHUNK = 4096;  // arcs per hub build/mark item (a 512-thread CTA, 8192-slot table)
constexpr int HUB_SLICE = 32768;  // histogram slots per hub evaluate item
constexpr int HUB_SMALL = 8192;  // hubs of at most this many slots are evaluated by one warp
constexpr int COL_PAD = 4;       // column arrays carry 4 spare entries for 16-byte loads

// Weight kinds of the device CSR.
enum WKind { W_UNIT = 0, W_I32 = 1, W_I64 = 2 };

struct WUnit {
  static constexpr bool unit = true;
  __device__ __forceinline__ static int64_t get(const void*, int64_t) { return 1; }
};
struct WI32 {
  static constexpr bool unit = false;
  __device__ __forceinline__ static int64_t get(const void* w, int64_t e) {
    return (int64_t)__ldg((const int32_t*)w + e);
  }
};
struct WI64 {
  static constexpr bool unit = false;
  __device__ __forceinline__ static int64_t get(const void* w, int64_t e) {
    return (int64_t)__ldg((const long long*)w + e);
  }
};

// Counters written by the scan kernels (one int64 each).
enum Ctr {
  C_MOVES = 0,   // append cursor of the move list = vertices moved this round
  C_DEFERRED,    // vertices whose move the coin deferred
  C_BIN0,        // then per bin: active, arcs, candidates
  C_HUB_BARCS = C_BIN0 + 3 * NBINS,  // arcs read by hub table builds this round
  C_HUB_BSLOTS,                      // table slots they wrote
  C_MARCS,                           // arcs of the vertices that moved this round
  C_HUB_MARCS,                       // arcs of the hubs that moved this round
  C_HUB_LOG,                         // hub-histogram updates logged this round
  C_HUB_PSLOTS,                      // table slots cleared, or read and written by compactions
  C_COUNT
};

// Per-kernel profiling slots.
enum Kern {
  K_UPLOAD = 0, K_SCAN_T4, K_SCAN_T8, K_SCAN_T16, K_SCAN_T32, K_SCAN_WARP, K_SCAN_BLK128,
  K_HUB_INSERT, K_HUB_EVAL, K_APPLY, K_RENUMBER, K_AGG_EMIT, K_SORT, K_AGG_REDUCE, K_MODULARITY,
  K_HUB_MARK, K_FRONTIER, K_SCAN_BLK512, K_HUB_PREP, K_COUNT
};
extern const char* const kKernelNames[K_COUNT];

}  // namespace cd

// The opaque handle.
struct cd_graph {
  cudaStream_t stream = nullptr;
  int64_t n = 0, nnz = 0, vol = 0, n_isolated = 0;
  int64_t* off = nullptr;   // n+1
  int32_t* cols = nullptr;  // nnz
  void* w = nullptr;        // nnz (int32 or int64), loop arcs carry 2L; null = unit
  int wkind = cd::W_UNIT;
  int64_t* degw = nullptr;  // n

  // static degree bins
  int32_t* bin_list = nullptr;           // n vertex ids grouped by bin
  int64_t bin_start[cd::NBINS + 1] = {};  // host copy of the bin offsets
  // frontier: the active vertices of a round, bin b at act_list + bin_start[b]
  int32_t* act_list = nullptr;
  unsigned long long* act_cnt = nullptr;   // NBINS+2: active per bin (hub bin: hub numbers), then the
                                           // evaluate items and small hubs routed this round
  unsigned long long* full_cnt = nullptr;  // NBINS+2: the same for every listed vertex
  int32_t* act_ev = nullptr;               // evaluate items of the examined hubs with large tables in use
  int32_t* act_small = nullptr;            // examined hubs with small tables in use (one warp each)
  // hubs (degree > BLOCK_MAX): one persistent label histogram per hub, kept in
  // step with the labels by the moves of its neighbours: an open-addressing
  // table allocated cap_h = 1.5 deg + 64 slots in [hub_tab[h], hub_tab[h+1]),
  // of which the first hub_cc[h] are in use (a compaction shrinks it). A slot
  // is one word (label << 32 | count) when every deg_w < 2^32 ("packed"),
  // otherwise two words (label, count).
  int64_t nhubs = 0, hub_slots = 0, hub_items = 0, hub_eval_items = 0;
  int hub_wide = 0;                        // 1: two-word slots
  uint32_t* hub_pref = nullptr;        // per 32-vertex word: hubs with smaller vertex ids (hub number = rank)
  uint32_t* hub_bits = nullptr;            // (n+31)/32: bit v set iff v is a hub
  int64_t* hub_tab = nullptr;              // nhubs+1
  int64_t* hub_cc = nullptr;               // nhubs: slots in use, [0, hub_cc) of the allocation (rest empty)
  int32_t* hub_live = nullptr;             // nhubs: live entries counted by the evaluate items of a round
  unsigned long long* hub_slot = nullptr;  // hub_slots words (x2 when wide)
  int32_t* hub_item_hub = nullptr;         // per build/mark item (HUB_CHUNK arcs): hub
  int64_t* hub_item_arc = nullptr;         // per build/mark item: first arc
  int32_t* hub_ev_hub = nullptr;           // per evaluate item (HUB_SLICE entries): hub
  int64_t* hub_ev_slot = nullptr;          // per evaluate item: first slot
  int64_t* hub_ev_first = nullptr;         // nhubs+1: first evaluate item of each hub
  int64_t* hub_part = nullptr;             // per evaluate item: (key hi, key lo, community)
  int64_t* hub_cur = nullptr;              // nhubs: weight into the hub's own label
  int32_t* hub_hascur = nullptr;           // nhubs
  int32_t* hub_done = nullptr;             // nhubs: finished evaluate items this round
  int32_t* hub_mv = nullptr;               // 3 x nhubs: moved flag, old label, new label
  int32_t* hub_rb = nullptr;               // nhubs: 1 = rebuild this hub's table from its row
  int32_t* hub_flist = nullptr;            // 2 x nhubs: hubs flagged in even / odd rounds
  unsigned long long* hub_fcnt = nullptr;  // 2: their counts
  int32_t* hub_used = nullptr;             // nhubs: slots claimed since the last build
  int64_t* hub_item_first = nullptr;       // nhubs+1: first build/mark item of each hub
  int32_t* hub_blist = nullptr;            // hub_items: build items queued this round
  int32_t* hub_mlist = nullptr;            // hub_items: mark items queued this round
  unsigned long long* hub_lcnt = nullptr;  // 2: queued build and mark items
  int32_t* hub_cl = nullptr;               // 5 x nhubs: hubs rebuilt per build class
  unsigned long long* hub_ccnt = nullptr;  // 5: their counts
  unsigned long long* hub_log = nullptr;   // per round: hub-histogram updates (hub, old, new, w) to apply
  int64_t hub_log_cap = 0;
  int64_t max_degw = 0;            // largest deg_w (selects 32-bit table counters)
  bool cols_distinct = false;      // no row repeats a column (strictly increasing input rows, or coarse rows)
  int t_warp = cd::WARP_MAX;       // degrees 33..t_warp: a warp per vertex
  int t_hub = cd::BLOCK_MAX;       // degrees t_warp+1..t_hub: 128 threads (512 above 1024); above: hub
  bool bins_set = false;           // thresholds chosen by cd_graph_set_bins / cd_autotune (kept by coarse graphs)

  // run state (allocated on first use)
  int32_t* C = nullptr;
  int64_t* sigma = nullptr;
  uint32_t* sigma32 = nullptr;  // 32-bit copy for the gathers (allocated on first use)
  int32_t* csize = nullptr;
  uint32_t* flag[2] = {nullptr, nullptr};  // needCheck / tmpNeedCheck bitmaps (n bits each)

  int32_t* mv_v = nullptr;  // committed moves: vertex, new label, old label
  int32_t* mv_c = nullptr;
  int32_t* mv_a = nullptr;
  int64_t* ctr = nullptr;      // device counters
  int64_t* h_ctr = nullptr;    // pinned host copy
  int32_t* status = nullptr;   // device status word (0 = ok)

  // batched mode: independent graphs packed block-diagonally (graph b owns
  // vertices [gbase[b], gbase[b+1]) and no arc leaves its block)
  int64_t nb = 0;                  // number of graphs (0: not batched)
  int32_t* gid = nullptr;          // n: graph of each vertex
  int64_t* gbase = nullptr;        // nb+1: first vertex of each graph
  int64_t* gvol = nullptr;         // nb: vol(V) of each graph
  uint8_t* gfrozen = nullptr;      // nb: 1 = graph finished, its vertices are not examined
  int64_t* gcnt = nullptr;         // nb: vertices of the graph that moved or deferred this round
  std::vector<int64_t> h_gbase;    // host copy of gbase

  std::vector<cd_round_trace> trace;
  cd_kernel_profile prof[cd::K_COUNT] = {};
  bool timing = false;   // per-round events (trace scan_ms/round_ms)
  bool ktiming = false;  // per-kernel events (profile); the bins' kernels then run one after another
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;  // (kernel, events)
  std::vector<double> pending_bytes;
};

namespace cd {

// Every kernel launch of the library goes through CD_LAUNCH, which counts it
// (process-wide; read with cd_launch_count).
void note_launch();
#define CD_LAUNCH(...) (::cd::note_launch(), __VA_ARGS__)

// error plumbing
int set_cuda_error(cudaError_t e);
#define CD_CHECK(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return ::cd::set_cuda_error(_e); \
  } while (0)

int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
template <class T>
int dev_alloc_t(T** p, int64_t count, cudaStream_t s) {
  return dev_alloc((void**)p, (size_t)(count > 0 ? count : 1) * sizeof(T), s);
}

// profiling helpers: bracket a launch with events when per-kernel timing is on
struct KTimer {
  cd_graph* g;
  int k;
  double bytes;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st = nullptr;  // the stream the timed kernel runs on (g->stream if null)
  KTimer(cd_graph* g_, int k_, double bytes_ = 0.0, cudaStream_t st_ = nullptr);
  ~KTimer();
};
void profile_reset(cd_graph* g);
int profile_flush(cd_graph* g);  // syncs, accumulates pending events

// graph.cu
// Takes ownership of device arrays in the internal convention (loop arcs 2L).
int graph_adopt(cudaStream_t s, int64_t n, int64_t nnz, int64_t* off, int32_t* cols, void* w,
                int wkind, cd_graph** out, int64_t* degw_pre = nullptr,
                const unsigned long long* stats_pre = nullptr, const cd_graph* like = nullptr);
int ensure_run_state(cd_graph* g);
// Recompute the degree bins and hub structures for new boundaries.
int rebin(cd_graph* g, int t_warp, int t_hub);
int check_labels(cd_graph* g, const int32_t* labels_dev);  // CD_EINVAL if out of [0, n)

// scan.cu
struct RunOpts {
  bool batched = false;  // use g's graph partition (per-graph vol, ids, freezing)
  int32_t max_iter;
  int64_t threshold;  // LPA only
  int tie_keep_current, singleton_rule, use_frontier;
  uint64_t sched_seed;
  int32_t level;
  int async_mode = 0;  // committed moves take effect at once (the coin still defers half of them)
  bool singleton_start = false;  // the run starts from C[v] = v (Sigma_tot = deg_w, sizes 1)
  bool device_loop = false;      // rounds after the first run as one captured graph (batched runs)
  bool device_loop_all = false;  // ... in every run
};
// Algorithm 1 / Algorithm 2 round loops on g->C (device). Louvain: g->C holds
// the initial partition; sigma/csize are rebuilt from it.
int run_lpa(cd_graph* g, const RunOpts& o, int32_t* rounds_out);
// Batched variants (g->nb > 0): per-graph vol(V) and coin ids, frozen graphs
// skipped. run_lpa_batched freezes a graph after its first round with
// moved + deferred <= threshold and reports its round count.
int run_lpa_batched(cd_graph* g, const RunOpts& o, std::vector<int32_t>& rounds);
void release_batches(cd_graph* g);
int run_local_move(cd_graph* g, const RunOpts& o, int init_given, int64_t* moves_out,
                   int32_t* rounds_out);
RunOpts opts_from(const cd_params* p, int32_t level);
int begin_run(cd_graph* g, const cd_params* p);  // validates params, resets trace/profile

// aggregate.cu
int renumber(cd_graph* g, const int32_t* labels_dev, int32_t* newid_dev, int64_t* k_out);
int aggregate(cd_graph* g, const int32_t* labels_dev, const int32_t* newid_dev, int64_t k,
              cd_graph** coarse_out, int mode = 0);
// Aggregation by hash-combining per community (no sort of the arcs).
int aggregate_hash(cd_graph* g, const int32_t* labels_dev, const int32_t* newid_dev, int64_t k,
                   cd_graph** coarse_out);
int modularity(cd_graph* g, const int32_t* labels_dev, double* q_out);

// prims.cu: device-wide primitives on the graph's stream
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                       cudaStream_t s);
int exclusive_scan_u8_to_i32(const uint8_t* in, int32_t* out, int64_t n, int64_t* total_dev,
                             cudaStream_t s);
// out[i] = number of run starts (keys[j] != keys[j-1]) among j < i.
int exclusive_scan_head(const uint64_t* keys, int64_t* out, int64_t n, int64_t* total_dev,
                        cudaStream_t s);
int radix_sort_pairs(uint64_t* keys, int64_t* vals, uint64_t* keys_tmp, int64_t* vals_tmp,
                     int64_t n, int bits, cudaStream_t s, uint64_t** keys_out, int64_t** vals_out);

}  // namespace cd
