/*
 * CPU oracle for community detection (Label Propagation and Louvain).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct restatement of
 * the paper's definitions and algorithms that the GPU path is checked
 * against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; it shares no code with the CUDA sources.
 *
 * Readings of the paper this file follows (each listed in the design notes):
 *  - Rounds are synchronous: every decision in a round reads the state at the
 *    start of the round, then all moves are applied at once. The paper's
 *    Chapel loops update shared arrays asynchronously (Sec. III-A-2, III-B-1);
 *    a pinned schedule is what makes the result reproducible.
 *  - The modularity formula of Sec. II-C is read per community c:
 *    Q = sum_c [(vol(c) - cut(c)) / vol(V) - vol(c)^2 / vol(V)^2].
 *  - In Eq. deltaQ the factor printed as deg_w(V) is read as deg_w(v).
 *  - A round budget of maxIteration means exactly maxIteration rounds at most.
 *  - Louvain ties among equal best gains go to the smallest community id; LPA
 *    keeps the current label when it attains the maximum, else takes the
 *    smallest label among the maxima.
 *  - Singleton rule: a singleton only joins another singleton with a smaller
 *    id (otherwise two singletons swap forever under synchronous rounds).
 *  - Randomised deferral: the paper relies on the random interleaving of
 *    asynchronous threads (and the original LPA on a random vertex order).
 *    Here that randomness is a pinned coin: in round r of level l a vertex
 *    whose decision differs from its label commits the move only if bit 63 of
 *    SplitMix64 draw number (l << 48 | r << 32 | v) from state `sched_seed`
 *    is set; otherwise it defers, stays active, and decides again next round.
 *    Without it, synchronous rounds lock into period-2 swaps between
 *    communities and never converge.
 *  - dN (Algorithm 1) and "a vertex changes community" (Algorithm 2) count the
 *    vertices whose decision differs from their label: moved plus deferred.
 *  - Next round's active set = moved vertices, their neighbours, and deferred
 *    vertices (Algorithm 1 and Algorithm 2 both mark v and N(v) after a move,
 *    and Algorithm 1 only drops a vertex whose best label is its own).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

static inline int64_t arc_w(const int64_t* w, int64_t e) { return w ? w[e] : 1; }

static void put_i128(i128 x, int64_t* out) {
  out[0] = (int64_t)(x >> 64);
  out[1] = (int64_t)(uint64_t)x;
}

/* ---- Sec. II-A: weighted degree and volume --------------------------- */

int64_t orc_degw(int64_t n, const int64_t* off, const int32_t* cols,
                 const int64_t* w, int64_t* degw_out) {
  int64_t vol = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t s = 0;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      /* every incident edge once, plus L_v once more for a loop */
      s += arc_w(w, e);
      if (cols[e] == v) s += arc_w(w, e);
    }
    degw_out[v] = s;
    vol += s;
  }
  return vol;
}

/* ---- Sec. II-C: modularity ------------------------------------------- */

double orc_modularity(int64_t n, const int64_t* off, const int32_t* cols,
                      const int64_t* w, const int32_t* labels,
                      int64_t* num_out, int64_t* den_out) {
  for (int64_t v = 0; v < n; ++v)
    if (labels[v] < 0 || labels[v] >= n) return NAN;
  int64_t* degw = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* volc = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* cutc = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t vol = orc_degw(n, off, cols, w, degw);
  for (int64_t v = 0; v < n; ++v) volc[labels[v]] += degw[v];
  /* cut(c) = weight of the edges with exactly one end in c: each such edge
   * shows up once as an arc leaving c. */
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      int32_t u = cols[e];
      if (u != v && labels[u] != labels[v]) cutc[labels[v]] += arc_w(w, e);
    }
  i128 num = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (volc[c] == 0 && cutc[c] == 0) continue;
    num += (i128)(volc[c] - cutc[c]) * vol - (i128)volc[c] * volc[c];
  }
  i128 den = (i128)vol * vol;
  if (num_out) put_i128(num, num_out);
  if (den_out) put_i128(den, den_out);
  free(degw);
  free(volc);
  free(cutc);
  if (vol == 0) return 0.0;
  return (double)num / (double)den;
}

/* ---- Sec. II-C, Eq. deltaQ: gain of one move, from the definitions ---- */

void orc_move_gain(int64_t n, const int64_t* off, const int32_t* cols,
                   const int64_t* w, const int32_t* labels, int32_t v,
                   int32_t B, int64_t* g_out) {
  int32_t A = labels[v];
  int64_t* degw = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t vol = orc_degw(n, off, cols, w, degw);
  /* A- and B- are A and B without v */
  int64_t volA = 0, volB = 0;
  for (int64_t x = 0; x < n; ++x) {
    if (x == v) continue;
    if (labels[x] == A) volA += degw[x];
    if (labels[x] == B) volB += degw[x];
  }
  /* cut_w(v, S) over the edges from v into S (S never contains v) */
  int64_t cutA = 0, cutB = 0;
  for (int64_t e = off[v]; e < off[v + 1]; ++e) {
    int32_t u = cols[e];
    if (u == v) continue;
    if (labels[u] == A) cutA += arc_w(w, e);
    if (labels[u] == B) cutB += arc_w(w, e);
  }
  i128 g = (i128)vol * (cutB - cutA) - (i128)degw[v] * (volB - volA);
  put_i128(g, g_out);
  free(degw);
}

/* ---- per-vertex neighbour-community accumulation ---------------------- */

struct orc_ws {
  int64_t n;
  int64_t* acc;     /* acc[c] = total weight from v into community c */
  unsigned char* seen;
  int32_t* touched; /* communities with seen[c] = 1 */
  int64_t ntouched;
};

orc_ws* orc_ws_create(int64_t n) {
  orc_ws* ws = (orc_ws*)calloc(1, sizeof(orc_ws));
  ws->n = n;
  ws->acc = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  ws->seen = (unsigned char*)calloc((size_t)n + 1, 1);
  ws->touched = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  ws->ntouched = 0;
  return ws;
}

void orc_ws_free(orc_ws* ws) {
  if (!ws) return;
  free(ws->acc);
  free(ws->seen);
  free(ws->touched);
  free(ws);
}

/* k_{v,c} = sum of w(v,u) over neighbours u != v with labels[u] = c */
static void accumulate(const int64_t* off, const int32_t* cols,
                       const int64_t* w, const int32_t* labels, int32_t v,
                       orc_ws* ws) {
  ws->ntouched = 0;
  for (int64_t e = off[v]; e < off[v + 1]; ++e) {
    int32_t u = cols[e];
    if (u == v) continue; /* a loop is not a neighbour */
    int32_t c = labels[u];
    if (!ws->seen[c]) {
      ws->seen[c] = 1;
      ws->touched[ws->ntouched++] = c;
    }
    ws->acc[c] += arc_w(w, e);
  }
}

static void reset(orc_ws* ws) {
  for (int64_t i = 0; i < ws->ntouched; ++i) {
    int32_t c = ws->touched[i];
    ws->acc[c] = 0;
    ws->seen[c] = 0;
  }
  ws->ntouched = 0;
}

/* number of distinct labels among v's neighbours (loops excluded) */
static int64_t distinct_labels(const int64_t* off, const int32_t* cols,
                               const int32_t* labels, int32_t v, orc_ws* ws) {
  accumulate(off, cols, NULL, labels, v, ws);
  int64_t k = ws->ntouched;
  reset(ws);
  return k;
}

/* ---- Algorithm 1, PLPMove: most frequent (heaviest) neighbour label --- */

int32_t orc_lpa_decide(int64_t n, const int64_t* off, const int32_t* cols,
                       const int64_t* w, const int32_t* labels, int32_t v,
                       int tie_keep_current, orc_ws* ws) {
  (void)n;
  int32_t cur = labels[v];
  accumulate(off, cols, w, labels, v, ws);
  int32_t best = -1;
  int64_t bestW = 0;
  for (int64_t i = 0; i < ws->ntouched; ++i) {
    int32_t c = ws->touched[i];
    int64_t W = ws->acc[c];
    if (best < 0 || W > bestW || (W == bestW && c < best)) {
      best = c;
      bestW = W;
    }
  }
  int32_t out = cur;
  if (best >= 0) {
    if (tie_keep_current && ws->seen[cur] && ws->acc[cur] == bestW)
      out = cur;
    else
      out = best;
  }
  reset(ws);
  return out;
}

/* ---- Algorithm 2, one vertex: argmax of dQ over neighbour communities - */

int32_t orc_louvain_decide(int64_t n, const int64_t* off, const int32_t* cols,
                           const int64_t* w, const int32_t* labels,
                           const int64_t* sigma_tot, const int32_t* csize,
                           const int64_t* degw, int64_t vol, int32_t v,
                           int singleton_rule, orc_ws* ws) {
  (void)n;
  int32_t A = labels[v];
  int64_t d = degw[v];
  accumulate(off, cols, w, labels, v, ws);
  int64_t kA = ws->seen[A] ? ws->acc[A] : 0; /* cut_w(v, A-) */
  int64_t volAminus = sigma_tot[A] - d;      /* vol_w(A-) */
  int32_t best = -1;
  i128 gbest = 0;
  for (int64_t i = 0; i < ws->ntouched; ++i) {
    int32_t c = ws->touched[i];
    if (c == A) continue;
    /* dQ_{v->c} * vol(V)^2 / 2 = vol(V) (cut(v,c) - cut(v,A-))
     *                          - deg_w(v) (vol(c) - vol(A-))            */
    i128 g = (i128)vol * (ws->acc[c] - kA) - (i128)d * (sigma_tot[c] - volAminus);
    if (best < 0 || g > gbest || (g == gbest && c < best)) {
      best = c;
      gbest = g;
    }
  }
  reset(ws);
  if (best < 0 || gbest <= 0) return A; /* only strictly positive dQ moves */
  if (singleton_rule && csize[A] == 1 && csize[best] == 1 && best > A) return A;
  return best;
}

/* ---- the pinned deferral coin ----------------------------------------- */

/* SplitMix64 (Steele, Lea, Flood 2014): draw number ctr of the stream with
 * state `seed` is mix(seed + (ctr + 1) * golden gamma). */
static uint64_t splitmix64_draw(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int orc_commit(uint64_t sched_seed, int32_t level, int32_t round, int32_t v) {
  uint64_t ctr = ((uint64_t)level << 48) | ((uint64_t)round << 32) | (uint32_t)v;
  return (int)(splitmix64_draw(sched_seed, ctr) >> 63);
}

/* ---- next round's active set: moved vertices and their neighbours ----- */

static void mark_next(int64_t n, const int64_t* off, const int32_t* cols,
                      const unsigned char* moved, const unsigned char* deferred,
                      unsigned char* active, int use_frontier) {
  if (!use_frontier) {
    memset(active, 1, (size_t)n);
    return;
  }
  memset(active, 0, (size_t)n);
  for (int64_t v = 0; v < n; ++v) {
    if (deferred[v]) active[v] = 1;
    if (!moved[v]) continue;
    active[v] = 1;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) active[cols[e]] = 1;
  }
}

/* ---- Algorithm 1, PLP ------------------------------------------------- */

int32_t orc_lpa(int64_t n, const int64_t* off, const int32_t* cols,
                const int64_t* w, int32_t max_iter, int64_t threshold,
                int tie_keep_current, int use_frontier, uint64_t sched_seed,
                const unsigned char* active_in, int32_t* labels_out,
                int64_t* tr_moved, int64_t* tr_deferred, int64_t* tr_active,
                int64_t* tr_arcs, int64_t* tr_cands, int64_t* tr_marcs) {
  int32_t* C = labels_out;
  int32_t* nxt = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  unsigned char* active = (unsigned char*)malloc((size_t)n + 1);
  unsigned char* moved = (unsigned char*)malloc((size_t)n + 1);
  unsigned char* deferred = (unsigned char*)malloc((size_t)n + 1);
  orc_ws* ws = orc_ws_create(n);
  for (int64_t v = 0; v < n; ++v) C[v] = (int32_t)v; /* singleton labels */
  if (active_in)
    memcpy(active, active_in, (size_t)n);             /* a given V_active */
  else
    memset(active, 1, (size_t)n);                     /* V_active = V */
  int32_t rounds = 0;
  for (int32_t r = 0; r < max_iter; ++r) {
    int64_t nact = 0, arcs = 0, nmoved = 0, ndef = 0, cands = 0, marcs = 0;
    memset(deferred, 0, (size_t)n);
    for (int64_t v = 0; v < n; ++v) {
      nxt[v] = C[v];
      if (!active[v]) continue;
      ++nact;
      arcs += off[v + 1] - off[v];
      if (tr_cands) cands += distinct_labels(off, cols, C, (int32_t)v, ws);
      int32_t c = orc_lpa_decide(n, off, cols, w, C, (int32_t)v, tie_keep_current, ws);
      if (c == C[v]) continue;
      if (orc_commit(sched_seed, 0, r, (int32_t)v))
        nxt[v] = c;
      else
        deferred[v] = 1;
    }
    for (int64_t v = 0; v < n; ++v) {
      moved[v] = (unsigned char)(nxt[v] != C[v]);
      nmoved += moved[v];
      ndef += deferred[v];
      if (moved[v]) marcs += off[v + 1] - off[v];
      C[v] = nxt[v];
    }
    mark_next(n, off, cols, moved, deferred, active, use_frontier);
    if (tr_cands) tr_cands[r] = cands;
    if (tr_marcs) tr_marcs[r] = marcs;
    if (tr_moved) tr_moved[r] = nmoved;
    if (tr_deferred) tr_deferred[r] = ndef;
    if (tr_active) tr_active[r] = nact;
    if (tr_arcs) tr_arcs[r] = arcs;
    rounds = r + 1;
    if (nmoved + ndef <= threshold) break; /* dN <= threshold */
  }
  orc_ws_free(ws);
  free(nxt);
  free(active);
  free(moved);
  free(deferred);
  return rounds;
}

/* ---- Algorithm 2, local moving ---------------------------------------- */

int32_t orc_local_move(int64_t n, const int64_t* off, const int32_t* cols,
                       const int64_t* w, int32_t max_iter, int singleton_rule,
                       int use_frontier, uint64_t sched_seed, int32_t level,
                       int init_given, const unsigned char* active_in,
                       int32_t* labels_io, int64_t* moves_out,
                       int64_t* tr_moved, int64_t* tr_deferred,
                       int64_t* tr_active, int64_t* tr_arcs,
                       int64_t* tr_cands, int64_t* tr_marcs) {
  int32_t* C = labels_io;
  if (init_given) {
    for (int64_t v = 0; v < n; ++v)
      if (C[v] < 0 || C[v] >= n) return -1;
  } else {
    for (int64_t v = 0; v < n; ++v) C[v] = (int32_t)v; /* comID = vertexID */
  }
  int64_t* degw = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int64_t* sigma = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t)); /* volCom */
  int32_t* csize = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t* target = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  unsigned char* flag = (unsigned char*)malloc((size_t)n + 1); /* needCheck */
  unsigned char* moved = (unsigned char*)malloc((size_t)n + 1);
  unsigned char* deferred = (unsigned char*)malloc((size_t)n + 1);
  orc_ws* ws = orc_ws_create(n);
  int64_t vol = orc_degw(n, off, cols, w, degw); /* volVertex = deg_w */
  for (int64_t v = 0; v < n; ++v) {
    sigma[C[v]] += degw[v];
    csize[C[v]] += 1;
  }
  if (active_in)
    memcpy(flag, active_in, (size_t)n); /* a given needCheck */
  else
    memset(flag, 1, (size_t)n);
  int64_t total = 0;
  int32_t rounds = 0;
  for (int32_t r = 0; r < max_iter; ++r) {
    int64_t nact = 0, arcs = 0, nm = 0, ndef = 0, cands = 0, marcs = 0;
    memset(deferred, 0, (size_t)n);
    for (int64_t v = 0; v < n; ++v) {
      target[v] = C[v];
      if (!flag[v]) continue;
      ++nact;
      arcs += off[v + 1] - off[v];
      if (tr_cands) cands += distinct_labels(off, cols, C, (int32_t)v, ws);
      int32_t b = orc_louvain_decide(n, off, cols, w, C, sigma, csize, degw, vol,
                                     (int32_t)v, singleton_rule, ws);
      if (b == C[v]) continue;
      if (orc_commit(sched_seed, level, r, (int32_t)v)) {
        target[v] = b;
      } else {
        deferred[v] = 1;
        ++ndef;
      }
    }
    for (int64_t v = 0; v < n; ++v) {
      moved[v] = (unsigned char)(target[v] != C[v]);
      if (!moved[v]) continue;
      int32_t A = C[v], B = target[v];
      sigma[A] -= degw[v];
      sigma[B] += degw[v];
      csize[A] -= 1;
      csize[B] += 1;
      C[v] = B;
      ++nm;
      marcs += off[v + 1] - off[v];
    }
    mark_next(n, off, cols, moved, deferred, flag, use_frontier);
    if (tr_cands) tr_cands[r] = cands;
    if (tr_marcs) tr_marcs[r] = marcs;
    if (tr_moved) tr_moved[r] = nm;
    if (tr_deferred) tr_deferred[r] = ndef;
    if (tr_active) tr_active[r] = nact;
    if (tr_arcs) tr_arcs[r] = arcs;
    total += nm;
    rounds = r + 1;
    if (nm + ndef == 0) break; /* no vertex changes community */
  }
  if (moves_out) *moves_out = total;
  orc_ws_free(ws);
  free(degw);
  free(sigma);
  free(csize);
  free(target);
  free(flag);
  free(moved);
  free(deferred);
  return rounds;
}

/* ---- Algorithm 3, Aggregation ----------------------------------------- */

/* new ids for the used community ids, ascending; returns k */
static int64_t renumber(int64_t n, const int32_t* labels, int32_t* newid) {
  for (int64_t c = 0; c < n; ++c) newid[c] = -1;
  for (int64_t v = 0; v < n; ++v) newid[labels[v]] = 0;
  int64_t k = 0;
  for (int64_t c = 0; c < n; ++c)
    if (newid[c] == 0) newid[c] = (int32_t)k++;
  return k;
}

typedef struct {
  int32_t a, b;
  int64_t w;
} triple;

static int cmp_triple(const void* x, const void* y) {
  const triple* p = (const triple*)x;
  const triple* q = (const triple*)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return 0;
}

int64_t orc_aggregate(int64_t n, const int64_t* off, const int32_t* cols,
                      const int64_t* w, const int32_t* labels,
                      int32_t* newid_out, int64_t* coff, int32_t* ccols,
                      int64_t* cw, int64_t* cnnz_out) {
  for (int64_t v = 0; v < n; ++v)
    if (labels[v] < 0 || labels[v] >= n) return -1;
  int64_t k = renumber(n, labels, newid_out);
  int64_t nnz = off[n];
  triple* t = (triple*)malloc(sizeof(triple) * ((size_t)nnz + 1));
  int64_t nt = 0;
  /* every edge {u,v} of G once: arcs with v < u, plus loops */
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      int32_t u = cols[e];
      if (u < v) continue;
      int32_t A = newid_out[labels[v]], B = newid_out[labels[u]];
      int64_t we = arc_w(w, e);
      if (A == B) {
        t[nt++] = (triple){A, A, we}; /* edge inside A: loop {A,A} */
      } else {
        t[nt++] = (triple){A, B, we}; /* edge {A,B}, both directions */
        t[nt++] = (triple){B, A, we};
      }
    }
  qsort(t, (size_t)nt, sizeof(triple), cmp_triple);
  int64_t m = 0;
  for (int64_t c = 0; c <= k; ++c) coff[c] = 0;
  for (int64_t i = 0; i < nt;) {
    int64_t j = i, s = 0;
    while (j < nt && t[j].a == t[i].a && t[j].b == t[i].b) s += t[j++].w;
    ccols[m] = t[i].b;
    cw[m] = s;
    coff[t[i].a + 1] += 1;
    ++m;
    i = j;
  }
  for (int64_t c = 0; c < k; ++c) coff[c + 1] += coff[c];
  *cnnz_out = m;
  free(t);
  return k;
}

/* ---- Algorithm 3, Louvain -------------------------------------------- */

int32_t orc_louvain(int64_t n, const int64_t* off, const int32_t* cols,
                    const int64_t* w, int32_t max_iter, int32_t max_levels,
                    int singleton_rule, int use_frontier, uint64_t sched_seed,
                    int32_t* labels_out,
                    double* q_out, int32_t* tr_rounds, int64_t* tr_moves,
                    int64_t* tr_nverts) {
  int64_t nnz = off[n];
  /* the current level's graph; level 0 is the input */
  int64_t gn = n;
  int64_t* goff = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* gcols = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nnz + 1));
  int64_t* gw = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nnz + 1));
  memcpy(goff, off, sizeof(int64_t) * ((size_t)n + 1));
  memcpy(gcols, cols, sizeof(int32_t) * (size_t)nnz);
  for (int64_t e = 0; e < nnz; ++e) gw[e] = arc_w(w, e);
  int64_t* noff = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* ncols = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nnz + 1));
  int64_t* nw = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nnz + 1));
  int32_t* C = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t* newid = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  for (int64_t v = 0; v < n; ++v) labels_out[v] = (int32_t)v;
  int32_t levels = 0;
  for (int32_t lvl = 0; lvl < max_levels; ++lvl) {
    int64_t moves = 0;
    int32_t rounds = orc_local_move(gn, goff, gcols, gw, max_iter, singleton_rule,
                                    use_frontier, sched_seed, lvl, 0, NULL, C,
                                    &moves, NULL, NULL, NULL, NULL, NULL, NULL);
    if (tr_rounds) tr_rounds[lvl] = rounds;
    if (tr_moves) tr_moves[lvl] = moves;
    if (tr_nverts) tr_nverts[lvl] = gn;
    int64_t k = renumber(gn, C, newid);
    for (int64_t v = 0; v < n; ++v) labels_out[v] = newid[C[labels_out[v]]];
    levels = lvl + 1;
    if (k == gn) break; /* done: every vertex is its own community */
    int64_t cnnz = 0;
    orc_aggregate(gn, goff, gcols, gw, C, newid, noff, ncols, nw, &cnnz);
    gn = k;
    memcpy(goff, noff, sizeof(int64_t) * ((size_t)k + 1));
    memcpy(gcols, ncols, sizeof(int32_t) * (size_t)cnnz);
    memcpy(gw, nw, sizeof(int64_t) * (size_t)cnnz);
  }
  if (q_out) *q_out = orc_modularity(n, off, cols, w, labels_out, NULL, NULL);
  free(goff);
  free(gcols);
  free(gw);
  free(noff);
  free(ncols);
  free(nw);
  free(C);
  free(newid);
  return levels;
}
