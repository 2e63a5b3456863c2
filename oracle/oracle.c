/*
 * oracle.c -- plain single-threaded CPU oracle for GSL-LPA.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline and reference legs may load this file.  It shares
 * no code, header or table with the CUDA library and is written for a reader
 * checking it against the paper step by step: dense arrays, plain loops, no
 * pruning where pruning is not part of the definition, exact integer sums.
 *
 * Graph: symmetric CSR, int64 offsets[n+1], int32 cols[nnz], optional int32
 * weights[nnz] (NULL means every edge weighs 1), as in Section 3 ("unweighted
 * graphs ... unit weight").  Labels are int32 vertex ids in [0, n).
 *
 * Contents
 *   oracle_sync_sweep   one Jacobi sweep of Eq. 2 (all vertices, no pruning)
 *   oracle_sync_sweep_at  the same rule for listed vertices (sampled checks)
 *   oracle_lpa_sync     lpa() of Algorithm 3 with Jacobi sweeps
 *   oracle_lpa_seq      lpa() of Algorithm 3 run by one thread, in place,
 *                       with the processed/unprocessed flags of lpaMove()
 *   oracle_split_bfs    splitDisconnectedBfs() of Algorithm 2
 *   oracle_split_lp     splitDisconnectedLp() of Algorithm 1 (SL-LP / SL-LPP)
 *   oracle_modularity   Eq. 1 (second form), exact integer parts
 *   oracle_disconnected disconnectedCommunities() of Algorithm 4
 *   oracle_*_f32 / _f64 the same with float weights and double sums
 *
 * Readings taken where the paper is silent (all also listed in the design
 * notes):
 *   - ties between equally heavy labels go to the smallest label; the
 *     vertex's own label gets no preference (Eq. 2 leaves argmax ties open);
 *   - a vertex with no neighbour other than itself keeps its label and does
 *     not count as changed (Algorithm 3 skips j == i in scanCommunities);
 *   - the stop test after sweep t is (double)dN / (double)N <= tau, and the
 *     converging sweep counts as performed (Algorithm 3, lpa());
 *   - Algorithm 2 tests "c" where it assigned c' and compares C[j] with
 *     itself; it is read as c = C[i] and f_if(j) = (C[j] == C[i]), with the
 *     start vertex of each BFS the first unvisited vertex in ascending order,
 *     so every piece is labelled with its smallest vertex id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Eq. 2 */
/* Best label for vertex i given labels C: argmax_c sum_{j in J_i, j != i,
 * C_j = c} w_ij, ties to the smallest c.  W is a zeroed int64[n] scratch
 * array and touched an int32[deg] scratch list; both are left clean.
 * Returns C[i] itself when i has no neighbour other than itself. */
static int32_t best_label(int64_t i, const int64_t* off, const int32_t* col, const int32_t* w,
                          const int32_t* C, int64_t* W, int32_t* touched) {
  int64_t nt = 0;
  for (int64_t e = off[i]; e < off[i + 1]; ++e) {
    int32_t j = col[e];
    if (j == i) continue;                       /* scanCommunities: i != j */
    int32_t c = C[j];
    if (W[c] == 0) touched[nt++] = c;           /* weights are >= 1 */
    W[c] += (w ? w[e] : 1);
  }
  if (nt == 0) return C[i];
  int32_t best = touched[0];
  int64_t bestw = W[best];
  for (int64_t k = 1; k < nt; ++k) {
    int32_t c = touched[k];
    if (W[c] > bestw || (W[c] == bestw && c < best)) { best = c; bestw = W[c]; }
  }
  for (int64_t k = 0; k < nt; ++k) W[touched[k]] = 0;
  return best;
}

static int64_t max_degree(int64_t n, const int64_t* off) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) if (off[i + 1] - off[i] > m) m = off[i + 1] - off[i];
  return m;
}

/* One synchronous (Jacobi) sweep: next[i] = best label of i under prev, for
 * every vertex.  Returns dN = #{i : next[i] != prev[i]}, or -1 if out of memory. */
int64_t oracle_sync_sweep(int64_t n, const int64_t* off, const int32_t* col, const int32_t* w,
                          const int32_t* prev, int32_t* next) {
  int64_t* W = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(max_degree(n, off) + 1));
  if (!W || !touched) { free(W); free(touched); return -1; }
  int64_t dn = 0;
  for (int64_t i = 0; i < n; ++i) {
    next[i] = best_label(i, off, col, w, prev, W, touched);
    if (next[i] != prev[i]) ++dn;
  }
  free(W); free(touched);
  return dn;
}

/* Eq. 2 for listed vertices only: out[k] = the label oracle_sync_sweep
 * would give vertex sel[k] under labels prev (the same best_label(), one
 * vertex at a time), for checking sampled vertices of large graphs.
 * Returns 0, or -1 (out of memory or a vertex outside [0, n)). */
int oracle_sync_sweep_at(int64_t n, const int64_t* off, const int32_t* col, const int32_t* w,
                         const int32_t* prev, const int64_t* sel, int64_t k, int32_t* out) {
  int64_t maxd = 0;
  for (int64_t q = 0; q < k; ++q) {
    if (sel[q] < 0 || sel[q] >= n) return -1;
    int64_t d = off[sel[q] + 1] - off[sel[q]];
    if (d > maxd) maxd = d;
  }
  int64_t* W = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(maxd + 1));
  if (!W || !touched) { free(W); free(touched); return -1; }
  for (int64_t q = 0; q < k; ++q) out[q] = best_label(sel[q], off, col, w, prev, W, touched);
  free(W); free(touched);
  return 0;
}

/* lpa() of Algorithm 3 with synchronous sweeps.  labels[] receives C after
 * the last sweep performed; dn_per_sweep (nullable, >= max_iters entries)
 * receives dN of every sweep.  labels_init (nullable) replaces the identity
 * initialisation C = [0..N).  Returns the number of sweeps performed, or -1. */
int32_t oracle_lpa_sync(int64_t n, const int64_t* off, const int32_t* col, const int32_t* w,
                        const int32_t* labels_init, double tau, int32_t max_iters,
                        int32_t* labels, int64_t* dn_per_sweep) {
  for (int64_t i = 0; i < n; ++i) labels[i] = labels_init ? labels_init[i] : (int32_t)i;
  if (n == 0) return 0;
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!next) return -1;
  int32_t t = 0;
  while (t < max_iters) {
    int64_t dn = oracle_sync_sweep(n, off, col, w, labels, next);
    if (dn < 0) { free(next); return -1; }
    memcpy(labels, next, sizeof(int32_t) * (size_t)n);
    if (dn_per_sweep) dn_per_sweep[t] = dn;
    ++t;
    if ((double)dn / (double)n <= tau) break;   /* converged? */
  }
  free(next);
  return t;
}

/* lpa() of Algorithm 3 exactly as printed, run by a single thread: labels
 * are updated in place in ascending vertex order; a processed vertex is
 * marked processed before its scan, and when it changes label all of its
 * neighbours are marked unprocessed again.  Returns sweeps performed or -1. */
int32_t oracle_lpa_seq(int64_t n, const int64_t* off, const int32_t* col, const int32_t* w,
                       const int32_t* labels_init, double tau, int32_t max_iters,
                       int32_t* C, int64_t* dn_per_sweep) {
  for (int64_t i = 0; i < n; ++i) C[i] = labels_init ? labels_init[i] : (int32_t)i;
  if (n <= 0) return 0;
  int64_t* W = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(max_degree(n, off) + 1));
  uint8_t* processed = (uint8_t*)calloc((size_t)n, 1);     /* all unprocessed */
  if (!W || !touched || !processed) { free(W); free(touched); free(processed); return -1; }
  int32_t t = 0;
  while (t < max_iters) {
    int64_t dn = 0;
    for (int64_t i = 0; i < n; ++i) {               /* lpaMove() */
      if (processed[i]) continue;
      processed[i] = 1;                             /* prune */
      int32_t c = best_label(i, off, col, w, C, W, touched);
      if (c == C[i]) continue;
      C[i] = c;
      ++dn;
      for (int64_t e = off[i]; e < off[i + 1]; ++e) processed[col[e]] = 0;
    }
    if (dn_per_sweep) dn_per_sweep[t] = dn;
    ++t;
    if ((double)dn / (double)n <= tau) break;
  }
  free(W); free(touched); free(processed);
  return t;
}

/* ---------------------------------------------------------- Algorithm 2 */
/* splitDisconnectedBfs(): C'[i] = i; every vertex not yet visited starts a
 * BFS over neighbours in its own community, and every vertex reached takes
 * the start vertex as its label.  Scanning start vertices in ascending order
 * labels each connected piece of each community with its smallest vertex id.
 * Returns 0, or -1 if out of memory. */
int oracle_split_bfs(int64_t n, const int64_t* off, const int32_t* col, const int32_t* C, int32_t* Cp) {
  uint8_t* vis = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!vis || !queue) { free(vis); free(queue); return -1; }
  for (int64_t i = 0; i < n; ++i) Cp[i] = (int32_t)i;
  for (int64_t i = 0; i < n; ++i) {
    if (vis[i]) continue;
    int32_t c = C[i];
    int64_t head = 0, tail = 0;
    vis[i] = 1;
    queue[tail++] = (int32_t)i;
    while (head < tail) {
      int32_t u = queue[head++];
      Cp[u] = (int32_t)i;                       /* f_do */
      for (int64_t e = off[u]; e < off[u + 1]; ++e) {
        int32_t j = col[e];
        if (!vis[j] && C[j] == c) {             /* f_if */
          vis[j] = 1;
          queue[tail++] = j;
        }
      }
    }
  }
  free(vis); free(queue);
  return 0;
}

/* ---------------------------------------------------------- Algorithm 1 */
/* splitDisconnectedLp(): C'[i] = i, then repeated sweeps in which every
 * (unprocessed, with pruning) vertex takes the minimum C' over itself and
 * its neighbours of the same community, until a sweep changes nothing.
 * Single thread, in place, ascending order.  pruning=1 is SL-LPP.
 * Returns the number of sweeps, or -1 if out of memory. */
int32_t oracle_split_lp(int64_t n, const int64_t* off, const int32_t* col, const int32_t* C,
                        int pruning, int32_t* Cp) {
  uint8_t* processed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!processed) return -1;
  for (int64_t i = 0; i < n; ++i) Cp[i] = (int32_t)i;
  int32_t sweeps = 0;
  for (;;) {
    int64_t dn = 0;
    ++sweeps;
    for (int64_t i = 0; i < n; ++i) {
      if (pruning && processed[i]) continue;
      if (pruning) processed[i] = 1;
      int32_t cmin = Cp[i];
      for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int32_t j = col[e];
        if (C[j] == C[i] && Cp[j] < cmin) cmin = Cp[j];
      }
      if (cmin == Cp[i]) continue;
      Cp[i] = cmin;
      ++dn;
      if (pruning)
        for (int64_t e = off[i]; e < off[i + 1]; ++e)
          if (C[col[e]] == C[i]) processed[col[e]] = 0;
    }
    if (dn == 0) break;
  }
  free(processed);
  return sweeps;
}

/* ---------------------------------------------------------------- Eq. 1 */
/* Q = sum_c [ sigma_c / 2m - (Sigma_c / 2m)^2 ].  Over the symmetric CSR,
 * 2m = sum of all entry weights, sum_c sigma_c = S1 = sum of the weights of
 * entries (i, j) with C_i == C_j, Sigma_c = sum_{i in c} K_i with K_i the
 * weighted degree, and S2 = sum_c Sigma_c^2.  The integer parts are exact
 * (S2 in 128 bits); parts[] receives {2m, S1, S2_lo, S2_hi}.  Q is formed
 * once, in double, as S1/2m - S2/(2m)^2; an empty graph (2m = 0) gives 0.
 * Returns 0, or -1 (out of memory or a label outside [0, n)). */
int oracle_modularity(int64_t n, const int64_t* off, const int32_t* col, const int32_t* w,
                      const int32_t* C, double* q, uint64_t* parts) {
  uint64_t* Sigma = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
  if (!Sigma) return -1;
  for (int64_t i = 0; i < n; ++i) if (C[i] < 0 || C[i] >= n) { free(Sigma); return -1; }
  uint64_t two_m = 0, s1 = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t K = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
      uint64_t we = (uint64_t)(w ? w[e] : 1);
      K += we;
      if (C[col[e]] == C[i]) s1 += we;
    }
    two_m += K;
    Sigma[C[i]] += K;
  }
  unsigned __int128 s2 = 0;
  for (int64_t c = 0; c < n; ++c) s2 += (unsigned __int128)Sigma[c] * Sigma[c];
  free(Sigma);
  if (parts) {
    parts[0] = two_m; parts[1] = s1;
    parts[2] = (uint64_t)s2; parts[3] = (uint64_t)(s2 >> 64);
  }
  if (two_m == 0) { *q = 0.0; return 0; }
  double dm = (double)two_m;
  *q = (double)s1 / dm - (double)s2 / (dm * dm);
  return 0;
}

/* ------------------------------------------------ fp32 weights, fp64 sums */
/* The paper's own precision (Section 4.1): 32-bit float edge weights and
 * 64-bit float hashtable values.  best_label_f is Eq. 2 with every label's
 * sum accumulated in double in row order; equal sums go to the smallest
 * label.  Weights must be finite and > 0 (a zero sum then means "not seen"). */
static int32_t best_label_f(int64_t i, const int64_t* off, const int32_t* col, const float* w, const int32_t* C,
                            double* W, int32_t* touched) {
  int64_t nt = 0;
  for (int64_t e = off[i]; e < off[i + 1]; ++e) {
    int32_t j = col[e];
    if (j == i) continue;
    int32_t c = C[j];
    if (W[c] == 0.0) touched[nt++] = c;
    W[c] += (double)w[e];
  }
  if (nt == 0) return C[i];
  int32_t best = touched[0];
  double bestw = W[best];
  for (int64_t k = 1; k < nt; ++k) {
    int32_t c = touched[k];
    if (W[c] > bestw || (W[c] == bestw && c < best)) { best = c; bestw = W[c]; }
  }
  for (int64_t k = 0; k < nt; ++k) W[touched[k]] = 0.0;
  return best;
}

/* One Jacobi sweep with float weights; returns dN, or -1 (out of memory or
 * a weight that is not finite and positive). */
int64_t oracle_sync_sweep_f32(int64_t n, const int64_t* off, const int32_t* col, const float* w,
                              const int32_t* prev, int32_t* next) {
  for (int64_t e = 0; e < (n > 0 ? off[n] : 0); ++e)
    if (!(w[e] > 0.0f) || w[e] != w[e] || w[e] > 3.4e38f) return -1;
  double* W = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(max_degree(n, off) + 1));
  if (!W || !touched) { free(W); free(touched); return -1; }
  int64_t dn = 0;
  for (int64_t i = 0; i < n; ++i) {
    next[i] = best_label_f(i, off, col, w, prev, W, touched);
    if (next[i] != prev[i]) ++dn;
  }
  free(W); free(touched);
  return dn;
}

/* lpa() of Algorithm 3 with synchronous sweeps and float weights (the stop
 * rule as in oracle_lpa_sync). */
int32_t oracle_lpa_sync_f32(int64_t n, const int64_t* off, const int32_t* col, const float* w,
                            const int32_t* labels_init, double tau, int32_t max_iters,
                            int32_t* labels, int64_t* dn_per_sweep) {
  for (int64_t i = 0; i < n; ++i) labels[i] = labels_init ? labels_init[i] : (int32_t)i;
  if (n == 0) return 0;
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!next) return -1;
  int32_t t = 0;
  while (t < max_iters) {
    int64_t dn = oracle_sync_sweep_f32(n, off, col, w, labels, next);
    if (dn < 0) { free(next); return -1; }
    memcpy(labels, next, sizeof(int32_t) * (size_t)n);
    if (dn_per_sweep) dn_per_sweep[t] = dn;
    ++t;
    if ((double)dn / (double)n <= tau) break;
  }
  free(next);
  return t;
}

/* Eq. 1 (second form) with float weights, every sum in double:
 * Q = S1/2m - S2/(2m)^2 with 2m = sum of entry weights, S1 = weight of
 * entries inside communities, S2 = sum over communities of Sigma_c^2.
 * Returns 0, or -1 (out of memory or a label outside [0, n)). */
int oracle_modularity_f64(int64_t n, const int64_t* off, const int32_t* col, const float* w, const int32_t* C,
                          double* q) {
  double* Sigma = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!Sigma) return -1;
  for (int64_t i = 0; i < n; ++i) if (C[i] < 0 || C[i] >= n) { free(Sigma); return -1; }
  double two_m = 0.0, s1 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double K = 0.0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
      double we = (double)w[e];
      K += we;
      if (C[col[e]] == C[i]) s1 += we;
    }
    two_m += K;
    Sigma[C[i]] += K;
  }
  double s2 = 0.0;
  for (int64_t c = 0; c < n; ++c) s2 += Sigma[c] * Sigma[c];
  free(Sigma);
  *q = two_m == 0.0 ? 0.0 : s1 / two_m - s2 / (two_m * two_m);
  return 0;
}

/* ---------------------------------------------------------- Algorithm 4 */
/* disconnectedCommunities(): S = community sizes; for each vertex i in
 * ascending order whose community c is still unprocessed, BFS inside c from
 * i counting the vertices reached; flag c if fewer than S[c] were reached;
 * then mark c processed.  D (nullable, n bytes) receives the flags.
 * Returns the number of flagged communities, or -1. */
int64_t oracle_disconnected(int64_t n, const int64_t* off, const int32_t* col, const int32_t* C,
                            uint8_t* D) {
  int64_t* S = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  uint8_t* vis = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!S || !vis || !queue) { free(S); free(vis); free(queue); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    if (C[i] < 0 || C[i] >= n) { free(S); free(vis); free(queue); return -1; }
    S[C[i]]++;
  }
  if (D && n > 0) memset(D, 0, (size_t)n);
  int64_t flagged = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = C[i];
    if (S[c] == 0) continue;
    int64_t reached = 0, head = 0, tail = 0;
    vis[i] = 1;
    queue[tail++] = (int32_t)i;
    while (head < tail) {
      int32_t u = queue[head++];
      ++reached;
      for (int64_t e = off[u]; e < off[u + 1]; ++e) {
        int32_t j = col[e];
        if (!vis[j] && C[j] == c) { vis[j] = 1; queue[tail++] = j; }
      }
    }
    if (reached < S[c]) { if (D) D[c] = 1; ++flagged; }
    S[c] = 0;
  }
  free(S); free(vis); free(queue);
  return flagged;
}
