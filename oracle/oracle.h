/*
 * CPU oracle for community detection (Label Propagation and Louvain) on a
 * symmetric CSR graph.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct
 * restatement of the paper's definitions and algorithms that the GPU path is
 * checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never links, loads or calls
 * it, and it shares no code with the CUDA sources.
 *
 * Graph convention (paper, Sec. II-A): an undirected weighted graph given as a
 * symmetric CSR. A non-loop edge {u,v} of weight w appears as the two arcs
 * u->v and v->u, each carrying w. A loop on v of weight L appears once, as the
 * arc v->v carrying L. Weights are integers >= 1; w == NULL means unit weights.
 * Offsets are int64 (n+1 entries), column ids int32 in [0, n).
 *
 * All volumes, cuts and gains are exact integers (int64, products in
 * __int128), so every decision is exact; modularity is returned as the exact
 * fraction num/den and as its FP64 quotient.
 */
#ifndef CD_ORACLE_H
#define CD_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Sec. II-A: deg_w(v) = sum of incident edge weights + L_v (loops counted
 * twice). Writes deg_w[n]; returns vol_w(V) = sum_v deg_w(v). */
int64_t orc_degw(int64_t n, const int64_t* off, const int32_t* cols,
                 const int64_t* w, int64_t* degw_out);

/* Sec. II-C: modularity of the partition `labels` (values in [0, n)).
 * Q = sum_c [(vol(c) - cut(c)) / vol(V) - vol(c)^2 / vol(V)^2].
 * num_out[2] / den_out[2] receive the exact numerator and denominator of Q as
 * (high int64, low uint64 bits) pairs of a signed 128-bit value.
 * Returns Q as FP64 (0.0 when vol(V) == 0). Returns NaN if a label is out of
 * range. */
double orc_modularity(int64_t n, const int64_t* off, const int32_t* cols,
                      const int64_t* w, const int32_t* labels,
                      int64_t* num_out, int64_t* den_out);

/* Sec. II-C, Eq. deltaQ: the scaled gain G of moving v from its community
 * A = labels[v] to community B, with dQ_{v->B} = 2 G / vol(V)^2, where
 * G = vol(V) (cut(v,B-) - cut(v,A-)) - deg_w(v) (vol(B-) - vol(A-)).
 * Volumes are taken from `labels` directly. G is written as a signed 128-bit
 * (high, low) pair. B == A gives 0. */
void orc_move_gain(int64_t n, const int64_t* off, const int32_t* cols,
                   const int64_t* w, const int32_t* labels, int32_t v,
                   int32_t B, int64_t* g_out);

/* Scratch for the per-vertex decisions: a dense accumulator over community
 * ids plus a touched list, reset after every use. */
typedef struct orc_ws orc_ws;
orc_ws* orc_ws_create(int64_t n);
void orc_ws_free(orc_ws* ws);

/* Algorithm 1, PLPMove, for one vertex v: the neighbour label c* with the
 * largest total edge weight, ties broken per `tie_keep_current`
 * (1: keep labels[v] if it attains the maximum, else the smallest label among
 * the maxima; 0: always the smallest label among the maxima). Loops are not
 * neighbours. Returns labels[v] when v has no neighbour. */
int32_t orc_lpa_decide(int64_t n, const int64_t* off, const int32_t* cols,
                       const int64_t* w, const int32_t* labels, int32_t v,
                       int tie_keep_current, orc_ws* ws);

/* Algorithm 2, the body of the vertex loop, for one vertex v against the
 * start-of-round state (labels, sigma_tot = volCom, csize = community sizes):
 * the neighbour community with the largest positive gain (ties to the
 * smallest id), or labels[v] if there is none. With singleton_rule, a move of
 * a singleton into another singleton is only taken towards a smaller id. */
int32_t orc_louvain_decide(int64_t n, const int64_t* off, const int32_t* cols,
                           const int64_t* w, const int32_t* labels,
                           const int64_t* sigma_tot, const int32_t* csize,
                           const int64_t* degw, int64_t vol, int32_t v,
                           int singleton_rule, orc_ws* ws);

/* The pinned deferral coin: 1 if a vertex v whose decision differs from its
 * label commits the move in round `round` of level `level`, 0 if it defers.
 * Bit 63 of SplitMix64 draw number (level << 48 | round << 32 | v) from state
 * sched_seed. */
int orc_commit(uint64_t sched_seed, int32_t level, int32_t round, int32_t v);

/* Algorithm 1 (PLP) with synchronous rounds and the deferral coin.
 * active_in (n bytes, may be NULL = all of V) is the initial V_active.
 * labels_out[n] receives C. Per-round traces (moved, deferred, active
 * vertices, arcs scanned, candidate pairs = distinct neighbour labels summed
 * over the examined vertices, arcs of the moved vertices) go to the optional
 * arrays of length max_iter.
 * Stops after a round with moved + deferred <= threshold. Returns the number
 * of rounds. */
int32_t orc_lpa(int64_t n, const int64_t* off, const int32_t* cols,
                const int64_t* w, int32_t max_iter, int64_t threshold,
                int tie_keep_current, int use_frontier, uint64_t sched_seed,
                const unsigned char* active_in, int32_t* labels_out,
                int64_t* tr_moved, int64_t* tr_deferred, int64_t* tr_active,
                int64_t* tr_arcs, int64_t* tr_cands, int64_t* tr_marcs);

/* Algorithm 2 (local moving) with synchronous rounds and the deferral coin of
 * level `level`. If init_given is 0 the partition starts as singletons, else
 * from labels_io (values in [0, n)). active_in (n bytes, may be NULL = all)
 * is the initial needCheck. labels_io[n] receives comID.
 * *moves_out = total moves over all rounds. Per-round traces as for orc_lpa
 * (candidate pairs count the vertex's own community too). Stops after a round
 * in which no vertex moved or deferred. Returns the number of rounds (-1: bad
 * labels). */
int32_t orc_local_move(int64_t n, const int64_t* off, const int32_t* cols,
                       const int64_t* w, int32_t max_iter, int singleton_rule,
                       int use_frontier, uint64_t sched_seed, int32_t level,
                       int init_given, const unsigned char* active_in,
                       int32_t* labels_io, int64_t* moves_out,
                       int64_t* tr_moved, int64_t* tr_deferred,
                       int64_t* tr_active, int64_t* tr_arcs,
                       int64_t* tr_cands, int64_t* tr_marcs);

/* Algorithm 3, Aggregation: remap communities to 0..k-1 in ascending id order
 * (newid_out[c], -1 for unused ids) and build the coarse graph whose edge
 * {A,B} carries the summed weight of the edges between A and B (a loop {A,A}
 * carries the internal weight of A). Output arrays are caller-allocated:
 * coff[n+1], ccols[nnz], cw[nnz] suffice. Returns k; *cnnz_out = arcs. */
int64_t orc_aggregate(int64_t n, const int64_t* off, const int32_t* cols,
                      const int64_t* w, const int32_t* labels,
                      int32_t* newid_out, int64_t* coff, int32_t* ccols,
                      int64_t* cw, int64_t* cnnz_out);

/* Algorithm 3, Louvain: repeat local moving and aggregation until a level
 * leaves every vertex in its own community (or max_levels levels ran).
 * labels_out[n] receives the final community of every input vertex,
 * contiguous ids. *q_out = modularity of that partition on the input graph.
 * Per-level traces (optional, length max_levels): rounds, moves, vertices.
 * Returns the number of levels. */
int32_t orc_louvain(int64_t n, const int64_t* off, const int32_t* cols,
                    const int64_t* w, int32_t max_iter, int32_t max_levels,
                    int singleton_rule, int use_frontier, uint64_t sched_seed,
                    int32_t* labels_out,
                    double* q_out, int32_t* tr_rounds, int64_t* tr_moves,
                    int64_t* tr_nverts);

#ifdef __cplusplus
}
#endif
#endif
