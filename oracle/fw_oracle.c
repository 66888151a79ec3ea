/*
 * CPU oracle for all-pairs shortest paths.  TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the benchmark's CPU baseline call this file; the
 * product library never links, loads or calls it, and it shares no code with
 * the CUDA path.
 *
 * Everything here is a plain definition written out, in int64 for integer
 * weights and in fp64 for real weights (inputs are read as int32 / fp32 and
 * widened).  OpenMP only splits loops whose iterations are independent.
 *
 * Conventions (readings of points the paper leaves open):
 *   - A missing edge is `inf` (int path) or +infinity (real path).  A path
 *     through an unreachable vertex does not exist, so it is never compared.
 *   - D[i][i] = 0 on input (the diagonal of a distance matrix).
 *   - P[i][j] is the LAST HOP of the chosen i->j path: initialised to i when
 *     the edge i->j exists (i != j), -1 otherwise; relaxing through k with a
 *     STRICT improvement sets P[i][j] = P[k][j].
 *
 * Floyd-Warshall is Fig. 1 of the paper (Sec. 2.3): for every intermediate
 * vertex k in order, every pair (i, j) is relaxed through k.  The paper's
 * figure compares with ">=" and stores k in P; this oracle uses "<" and the
 * last hop so that the result on a unique shortest path does not depend on the
 * order in which a blocked schedule visits the intermediates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define OMP_THREADS(t) if ((t) > 0) omp_set_num_threads(t)
#else
#define OMP_THREADS(t) (void)(t)
#endif

typedef int64_t i64;

/* ---------------------------------------------------------------- FW ---- */

/* Fig. 1 (Sec. 2.3), integer weights.  W: n x n int64, row-major (int32
   inputs are widened by the caller). */
void oracle_fw_i64(const i64* W, i64 n, i64 inf, i64* D, int32_t* P, int threads) {
  OMP_THREADS(threads);
  for (i64 i = 0; i < n; ++i)
    for (i64 j = 0; j < n; ++j) {
      i64 w = W[i * n + j];
      D[i * n + j] = w;
      P[i * n + j] = (i != j && w < inf) ? (int32_t)i : -1;
    }
  for (i64 k = 0; k < n; ++k) {
    /* Row k and column k do not change while k is the intermediate
       (D[k][k] = 0 and only strict improvements are taken), so the rows
       i are independent within one k. */
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < n; ++i) {
      i64 dik = D[i * n + k];
      if (dik >= inf) continue;
      for (i64 j = 0; j < n; ++j) {
        i64 dkj = D[k * n + j];
        if (dkj >= inf) continue;
        if (dik + dkj < D[i * n + j]) {
          D[i * n + j] = dik + dkj;
          P[i * n + j] = P[k * n + j];
        }
      }
    }
  }
}

/* Fig. 1 (Sec. 2.3), real weights in fp64.  W: n x n fp64 (fp32 inputs are
   widened by the caller, which is exact). */
void oracle_fw_f64(const double* W, i64 n, double* D, int32_t* P, int threads) {
  OMP_THREADS(threads);
  for (i64 i = 0; i < n; ++i)
    for (i64 j = 0; j < n; ++j) {
      double w = W[i * n + j];
      D[i * n + j] = w;
      P[i * n + j] = (i != j && !isinf(w)) ? (int32_t)i : -1;
    }
  for (i64 k = 0; k < n; ++k) {
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < n; ++i) {
      double dik = D[i * n + k];
      if (isinf(dik)) continue;
      for (i64 j = 0; j < n; ++j) {
        double dkj = D[k * n + j];
        if (isinf(dkj)) continue;
        if (dik + dkj < D[i * n + j]) {
          D[i * n + j] = dik + dkj;
          P[i * n + j] = P[k * n + j];
        }
      }
    }
  }
}

/* Fig. 1 (Sec. 2.3) as printed in its path bookkeeping: P[i][j] receives the
   intermediate vertex k of the relaxation that last improved (i, j), -1 when
   none did (the diagonal, a shortest path that is the edge itself, an
   unreachable pair).  The comparison is the strict "<" of the functions above
   (with ">=" the relaxations through k = i and k = j, which add D[i][i] = 0 or
   D[j][j] = 0, would always tie and overwrite P).  The last improvement
   happens at the first k for which a shortest path with every intermediate
   vertex <= k exists, so K[i][j] is the smallest, over the shortest i -> j
   paths, of the largest intermediate vertex on the path: on a unique shortest
   path, its largest intermediate vertex.  D receives the distances. */
void oracle_fw_k_i64(const i64* W, i64 n, i64 inf, i64* D, int32_t* K, int threads) {
  OMP_THREADS(threads);
  for (i64 i = 0; i < n * n; ++i) {
    D[i] = W[i];
    K[i] = -1;
  }
  for (i64 k = 0; k < n; ++k) {
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < n; ++i) {
      i64 dik = D[i * n + k];
      if (dik >= inf) continue;
      for (i64 j = 0; j < n; ++j) {
        i64 dkj = D[k * n + j];
        if (dkj >= inf) continue;
        if (dik + dkj < D[i * n + j]) {
          D[i * n + j] = dik + dkj;
          K[i * n + j] = (int32_t)k;
        }
      }
    }
  }
}

void oracle_fw_k_f64(const double* W, i64 n, double* D, int32_t* K, int threads) {
  OMP_THREADS(threads);
  for (i64 i = 0; i < n * n; ++i) {
    D[i] = W[i];
    K[i] = -1;
  }
  for (i64 k = 0; k < n; ++k) {
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < n; ++i) {
      double dik = D[i * n + k];
      if (isinf(dik)) continue;
      for (i64 j = 0; j < n; ++j) {
        double dkj = D[k * n + j];
        if (isinf(dkj)) continue;
        if (dik + dkj < D[i * n + j]) {
          D[i * n + j] = dik + dkj;
          K[i * n + j] = (int32_t)k;
        }
      }
    }
  }
}

/* ---------------------------------------------------------- Dijkstra ---- */

/* Dense Dijkstra from each source in src[0..nsrc): textbook O(n^2) version.
   Output rows are written in source order: D[s*n + v], P[s*n + v]. */
void oracle_dijkstra_i64(const int32_t* W, i64 n, i64 inf, const i64* src, i64 nsrc,
                         i64* D, int32_t* P, int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 s = 0; s < nsrc; ++s) {
    i64* d = D + s * n;
    int32_t* p = P + s * n;
    unsigned char* done = (unsigned char*)calloc((size_t)n, 1);
    for (i64 v = 0; v < n; ++v) { d[v] = inf; p[v] = -1; }
    d[src[s]] = 0;
    for (i64 it = 0; it < n; ++it) {
      i64 u = -1, best = inf;
      for (i64 v = 0; v < n; ++v)
        if (!done[v] && d[v] < best) { best = d[v]; u = v; }
      if (u < 0) break;
      done[u] = 1;
      const int32_t* row = W + u * n;
      for (i64 v = 0; v < n; ++v) {
        i64 w = row[v];
        if (v == u || w >= inf || done[v]) continue;
        if (best + w < d[v]) { d[v] = best + w; p[v] = (int32_t)u; }
      }
    }
    free(done);
  }
}

void oracle_dijkstra_f64(const float* W, i64 n, const i64* src, i64 nsrc, double* D,
                         int32_t* P, int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 s = 0; s < nsrc; ++s) {
    double* d = D + s * n;
    int32_t* p = P + s * n;
    unsigned char* done = (unsigned char*)calloc((size_t)n, 1);
    for (i64 v = 0; v < n; ++v) { d[v] = INFINITY; p[v] = -1; }
    d[src[s]] = 0.0;
    for (i64 it = 0; it < n; ++it) {
      i64 u = -1;
      double best = INFINITY;
      for (i64 v = 0; v < n; ++v)
        if (!done[v] && d[v] < best) { best = d[v]; u = v; }
      if (u < 0) break;
      done[u] = 1;
      const float* row = W + u * n;
      for (i64 v = 0; v < n; ++v) {
        double w = (double)row[v];
        if (v == u || isinf(w) || done[v]) continue;
        if (best + w < d[v]) { d[v] = best + w; p[v] = (int32_t)u; }
      }
    }
    free(done);
  }
}

/* ------------------------------------------------------- certificate ---- */

/* LP-duality certificate of exact shortest distances for the rows listed in
   rows[0..nrows) (all rows when rows == NULL).  D and P hold those rows in the
   listed order (row r of D/P belongs to source rows[r]).  W is the full graph.
   bad[0]: D[s][s] != 0
   bad[1]: a finite D[s][v] (v != s) whose P is not a tight last hop
           (P out of range, no edge P->v, or D[s][P] + W[P][v] != D[s][v])
   bad[2]: an edge u->v with D[s][v] > D[s][u] + W[u][v] (not feasible)
   bad[3]: following P from v does not reach s within n steps, or P is set on
           an unreachable / diagonal entry, or a reachable v has P = -1. */
void oracle_certificate_i64(const int32_t* W, const int32_t* Drows, const int32_t* Prows, i64 n,
                            i64 inf, const i64* rows, i64 nrows, i64* bad, int threads) {
  OMP_THREADS(threads);
  i64 b0 = 0, b1 = 0, b2 = 0, b3 = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : b0, b1, b2, b3)
  for (i64 r = 0; r < nrows; ++r) {
    i64 s = rows ? rows[r] : r;
    const int32_t* d = Drows + r * n;
    const int32_t* p = Prows + r * n;
    if (d[s] != 0) b0++;
    for (i64 v = 0; v < n; ++v) {
      i64 dv = d[v];
      if (v == s) { if (p[v] != -1) b3++; continue; }
      if (dv >= inf) { if (p[v] != -1) b3++; continue; }
      i64 u = p[v];
      if (u < 0 || u >= n || u == v) { b1++; continue; }
      i64 w = W[u * n + v];
      if (w >= inf || d[u] >= inf || (i64)d[u] + w != dv) b1++;
      /* walk back along P: must reach s within n steps */
      i64 x = v, steps = 0;
      while (x != s && x >= 0 && steps <= n) { x = p[x]; steps++; }
      if (x != s) b3++;
    }
    for (i64 u = 0; u < n; ++u) {
      i64 du = d[u];
      if (du >= inf) continue;
      const int32_t* row = W + u * n;
      for (i64 v = 0; v < n; ++v) {
        i64 w = row[v];
        if (w >= inf || v == u) continue;
        if ((i64)d[v] > du + w) b2++;
      }
    }
  }
  bad[0] = b0; bad[1] = b1; bad[2] = b2; bad[3] = b3;
}

/* ----------------------------------------------- unique shortest paths ---- */

/* Number of distinct shortest s->v paths, capped at 2, for each listed source
   row (positive weights).  D holds exact distances for those rows.  A vertex's
   count is the sum of the counts of its tight in-neighbours u (D[s][u] +
   W[u][v] == D[s][v]); vertices are taken in increasing distance, which is a
   topological order of the tight edges when every weight is positive. */
static int cmp_pair(const void* a, const void* b) {
  const i64* x = (const i64*)a;
  const i64* y = (const i64*)b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  return x[1] < y[1] ? -1 : (x[1] > y[1]);
}

void oracle_path_count_i64(const int32_t* W, const i64* Drows, i64 n, i64 inf, const i64* rows,
                           i64 nrows, uint8_t* cnt, int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 r = 0; r < nrows; ++r) {
    i64 s = rows ? rows[r] : r;
    const i64* d = Drows + r * n;
    uint8_t* c = cnt + r * n;
    i64* order = (i64*)malloc((size_t)n * 2 * sizeof(i64));
    i64 m = 0;
    for (i64 v = 0; v < n; ++v) {
      c[v] = 0;
      if (d[v] < inf) { order[2 * m] = d[v]; order[2 * m + 1] = v; m++; }
    }
    qsort(order, (size_t)m, 2 * sizeof(i64), cmp_pair);
    c[s] = 1;
    for (i64 t = 0; t < m; ++t) {
      i64 v = order[2 * t + 1];
      if (v == s) continue;
      int total = 0;
      for (i64 u = 0; u < n && total < 2; ++u) {
        if (u == v || d[u] >= inf) continue;
        i64 w = W[u * n + v];
        if (w >= inf) continue;
        if (d[u] + w == d[v]) total += c[u];
      }
      c[v] = (uint8_t)(total > 2 ? 2 : total);
    }
    free(order);
  }
}

/* --------------------------------------------------- fp64 last-hop margin ---- */

/* For each listed source row and each v: the gap between the best path that
   ends with an edge u->v, u != P[s][v], and the shortest distance D[s][v]:
       margin = min_{u != P[s][v], u != v, W[u][v] < inf} (D[s][u] + W[u][v]) - D[s][v].
   +inf when no alternative last hop exists; -1 for unreachable v or v == s.
   A path whose last hop differs from P costs at least D + margin. */
void oracle_lasthop_margin_f64(const float* W, const double* Drows, const int32_t* Prows, i64 n,
                               const i64* rows, i64 nrows, double* margin, int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 r = 0; r < nrows; ++r) {
    i64 s = rows ? rows[r] : r;
    const double* d = Drows + r * n;
    const int32_t* p = Prows + r * n;
    double* mg = margin + r * n;
    for (i64 v = 0; v < n; ++v) {
      if (v == s || isinf(d[v])) { mg[v] = -1.0; continue; }
      double best = INFINITY;
      for (i64 u = 0; u < n; ++u) {
        if (u == v || u == p[v] || isinf(d[u])) continue;
        double w = (double)W[u * n + v];
        if (isinf(w)) continue;
        double alt = d[u] + w;
        if (alt < best) best = alt;
      }
      mg[v] = best - d[v];
    }
  }
}

/* Same quantity for integer weights (exact): 0 means a tie at the last hop. */
void oracle_lasthop_margin_i64(const int32_t* W, const i64* Drows, const int32_t* Prows, i64 n,
                               i64 inf, const i64* rows, i64 nrows, i64* margin, int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 r = 0; r < nrows; ++r) {
    i64 s = rows ? rows[r] : r;
    const i64* d = Drows + r * n;
    const int32_t* p = Prows + r * n;
    i64* mg = margin + r * n;
    for (i64 v = 0; v < n; ++v) {
      if (v == s || d[v] >= inf) { mg[v] = -1; continue; }
      i64 best = INT64_MAX;
      for (i64 u = 0; u < n; ++u) {
        if (u == v || u == p[v] || d[u] >= inf) continue;
        i64 w = W[u * n + v];
        if (w >= inf) continue;
        if (d[u] + w < best) best = d[u] + w;
      }
      mg[v] = best == INT64_MAX ? INT64_MAX : best - d[v];
    }
  }
}

/* --------------------------------------------------------------- hops ---- */

/* Number of edges on the path recorded by P from source s to v (row r of P
   belongs to source rows[r]); -1 when unreachable or when P does not lead back
   to s within n steps. */
void oracle_hops(const int32_t* Prows, i64 n, const i64* rows, i64 nrows, int32_t* hops,
                 int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 r = 0; r < nrows; ++r) {
    i64 s = rows ? rows[r] : r;
    const int32_t* p = Prows + r * n;
    for (i64 v = 0; v < n; ++v) {
      if (v == s) { hops[r * n + v] = 0; continue; }
      i64 x = v, h = 0;
      while (x != s && x >= 0 && h <= n) { x = p[x]; h++; }
      hops[r * n + v] = (x == s) ? (int32_t)h : -1;
    }
  }
}

/* Largest intermediate vertex on the path that a last-hop matrix records:
   walk from v back to the source s (row r of P belongs to source rows[r]) and
   take the largest vertex met strictly between them.  -1 on the diagonal, for
   a path that is a single edge, an unreachable v (P = -1) and a P that does
   not lead back to s within n steps. */
void oracle_max_intermediate(const int32_t* Prows, i64 n, const i64* rows, i64 nrows,
                             int32_t* out, int threads) {
  OMP_THREADS(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 r = 0; r < nrows; ++r) {
    i64 s = rows ? rows[r] : r;
    const int32_t* p = Prows + r * n;
    for (i64 v = 0; v < n; ++v) {
      i64 best = -1, x = v, h = 0;
      if (v != s) {
        x = p[v];
        while (x != s && x >= 0 && x < n && h <= n) {
          if (x > best) best = x;
          x = p[x];
          h++;
        }
      }
      out[r * n + v] = (x == s) ? (int32_t)best : -1;
    }
  }
}

/* ------------------------------------------------------------ gradient ---- */

/* Gradient of L = sum_{i,j} G[i][j] * D[i][j] with respect to the edge
   weights, through the shortest-path trees given by P (fp64).  For source i
   the tree has the edges P[i][v] -> v.  D[i][v] is the sum of the weights on
   the tree path i -> v, so dL/dW[u][v] collects G[i][j] over every pair (i, j)
   whose tree path uses the edge u -> v:
       E[i][v]  = G[i][v] + sum over tree children c of v of E[i][c]
       dL/dW[u][v] = sum over sources i with P[i][v] == u of E[i][v].
   Vertices are visited in decreasing hop depth so every child is complete
   before its parent reads it.  GW must be zeroed by the caller. */
void oracle_grad_f64(const double* G, const int32_t* P, i64 n, double* GW) {
  i64* depth = (i64*)malloc((size_t)n * sizeof(i64));
  i64* order = (i64*)malloc((size_t)n * 2 * sizeof(i64));
  double* E = (double*)malloc((size_t)n * sizeof(double));
  for (i64 i = 0; i < n; ++i) {
    const int32_t* p = P + i * n;
    i64 m = 0;
    for (i64 v = 0; v < n; ++v) {
      E[v] = G[i * n + v];
      depth[v] = -1;
      if (v == i) { depth[v] = 0; continue; }
      if (p[v] < 0) continue;
      i64 x = v, h = 0;
      while (x != i && x >= 0 && h <= n) { x = p[x]; h++; }
      if (x == i) depth[v] = h;
    }
    for (i64 v = 0; v < n; ++v)
      if (v != i && depth[v] > 0) { order[2 * m] = -depth[v]; order[2 * m + 1] = v; m++; }
    qsort(order, (size_t)m, 2 * sizeof(i64), cmp_pair);
    for (i64 t = 0; t < m; ++t) {
      i64 v = order[2 * t + 1];
      i64 u = p[v];
      E[u] += E[v];
      GW[u * n + v] += E[v];
    }
  }
  free(depth);
  free(order);
  free(E);
}
