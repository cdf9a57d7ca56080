/*
 * graphgen.c -- seeded synthetic input graphs shared by the CPU oracle and the GPU path.
 *
 * This module holds input generation only: no step of the partitioning method lives here.
 * Every graph is undirected, stored as a symmetric CSR (int64 row offsets, int32 column ids,
 * rows sorted ascending, no self-loops, no duplicate entries) with optional int32 edge weights
 * that are equal in both directions.
 *
 * Random numbers come from a counter-based generator: the SplitMix64 output function
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
 * (seed XOR counter). A uniform double in [0,1) is the top 53 bits of such a word times 2^-53.
 *
 * Workload families (stand-ins for the paper's benchmark classes, Section VI, Table I, whose files
 * are not available):
 *   grid  -- a x b 4-neighbour grid, id = row*b + col (mesh-like)
 *   rgg   -- random geometric graph in the unit square (the paper's rgg family, Section VI)
 *   rmat  -- R-MAT power-law graph (complex-network stand-in), symmetrised and deduplicated
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct gg_graph {
  int64_t n;
  int64_t m_dir;
  int64_t *off;   /* n+1 */
  int32_t *adj;   /* m_dir */
  int32_t *ew;    /* m_dir or NULL (unit) */
} gg_graph;

static uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

uint64_t gg_word(uint64_t seed, uint64_t ctr) { return gg_mix(seed ^ ctr); }

double gg_unif(uint64_t seed, uint64_t ctr) {
  return (double)(gg_word(seed, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

/* Three-argument keyed word used for per-edge weights and per-graph seeds in a batch. */
uint64_t gg_key3(uint64_t a, uint64_t b, uint64_t c) { return gg_mix(gg_mix(gg_mix(a) ^ b) ^ c); }

void gg_free(gg_graph *g) {
  if (!g) return;
  free(g->off);
  free(g->adj);
  free(g->ew);
  free(g);
}

int64_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_m(const gg_graph *g) { return g->m_dir; }
int gg_weighted(const gg_graph *g) { return g->ew != NULL; }

void gg_copy(const gg_graph *g, int64_t *off, int32_t *adj, int32_t *ew) {
  memcpy(off, g->off, sizeof(int64_t) * (size_t)(g->n + 1));
  memcpy(adj, g->adj, sizeof(int32_t) * (size_t)g->m_dir);
  if (ew && g->ew) memcpy(ew, g->ew, sizeof(int32_t) * (size_t)g->m_dir);
}

static gg_graph *gg_alloc(int64_t n) {
  gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
  g->n = n;
  g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  return g;
}

/* ---------------------------------------------------------------- grid */
gg_graph *gg_grid(int64_t a, int64_t b) {
  int64_t n = a * b;
  gg_graph *g = gg_alloc(n);
  for (int64_t r = 0; r < a; r++)
    for (int64_t c = 0; c < b; c++) {
      int64_t v = r * b + c;
      int d = (r > 0) + (r + 1 < a) + (c > 0) + (c + 1 < b);
      g->off[v + 1] = d;
    }
  for (int64_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
  g->m_dir = g->off[n];
  g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m_dir ? g->m_dir : 1));
  for (int64_t r = 0; r < a; r++)
    for (int64_t c = 0; c < b; c++) {
      int64_t v = r * b + c, p = g->off[v];
      /* ascending id order: up, left, right, down */
      if (r > 0) g->adj[p++] = (int32_t)(v - b);
      if (c > 0) g->adj[p++] = (int32_t)(v - 1);
      if (c + 1 < b) g->adj[p++] = (int32_t)(v + 1);
      if (r + 1 < a) g->adj[p++] = (int32_t)(v + b);
    }
  return g;
}

/* ---------------------------------------------------------------- helpers */
static int cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

static void sort_i32(int32_t *p, int64_t len) {
  /* insertion sort for short rows, qsort otherwise */
  if (len < 32) {
    for (int64_t i = 1; i < len; i++) {
      int32_t x = p[i];
      int64_t j = i - 1;
      while (j >= 0 && p[j] > x) {
        p[j + 1] = p[j];
        j--;
      }
      p[j + 1] = x;
    }
  } else {
    qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/* ---------------------------------------------------------------- rgg */
/* n points: x_i = U(seed, 2i), y_i = U(seed, 2i+1). Edge {i,j} iff squared distance < r^2,
 * r = sqrt(avg_deg / (pi * n)). Ids are in point-generation order. */
gg_graph *gg_rgg(int64_t n, double avg_deg, uint64_t seed) {
  double r = sqrt(avg_deg / (3.14159265358979323846 * (double)n));
  double r2 = r * r;
  double *x = (double *)malloc(sizeof(double) * (size_t)n);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; i++) {
    x[i] = gg_unif(seed, (uint64_t)(2 * i));
    y[i] = gg_unif(seed, (uint64_t)(2 * i + 1));
  }
  int64_t gcell = (int64_t)floor(1.0 / r);
  if (gcell < 1) gcell = 1;
  if (gcell > 65536) gcell = 65536;
  int64_t ncell = gcell * gcell;
  int64_t *cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) {
    int64_t cx = (int64_t)(x[i] * (double)gcell), cy = (int64_t)(y[i] * (double)gcell);
    if (cx >= gcell) cx = gcell - 1;
    if (cy >= gcell) cy = gcell - 1;
    cell[i] = cy * gcell + cx;
    cstart[cell[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; c++) cstart[c + 1] += cstart[c];
  int64_t *cfill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
  memcpy(cfill, cstart, sizeof(int64_t) * (size_t)ncell);
  int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) members[cfill[cell[i]]++] = (int32_t)i;
  free(cfill);

  gg_graph *g = gg_alloc(n);
  /* pass 1: degrees; pass 2: fill */
  for (int pass = 0; pass < 2; pass++) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
      int64_t ci = cell[i], cx = ci % gcell, cy = ci / gcell;
      int64_t cnt = 0, p = pass ? g->off[i] : 0;
      for (int64_t dy = -1; dy <= 1; dy++)
        for (int64_t dx = -1; dx <= 1; dx++) {
          int64_t nx = cx + dx, ny = cy + dy;
          if (nx < 0 || ny < 0 || nx >= gcell || ny >= gcell) continue;
          int64_t c = ny * gcell + nx;
          for (int64_t t = cstart[c]; t < cstart[c + 1]; t++) {
            int32_t j = members[t];
            if (j == i) continue;
            double ddx = x[i] - x[j], ddy = y[i] - y[j];
            if (ddx * ddx + ddy * ddy < r2) {
              if (pass) g->adj[p++] = j;
              else cnt++;
            }
          }
        }
      if (!pass) g->off[i + 1] = cnt;
      else sort_i32(g->adj + g->off[i], g->off[i + 1] - g->off[i]);
    }
    if (!pass) {
      for (int64_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
      g->m_dir = g->off[n];
      g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m_dir ? g->m_dir : 1));
    }
  }
  free(x);
  free(y);
  free(cstart);
  free(cell);
  free(members);
  return g;
}

/* ---------------------------------------------------------------- rmat */
/* R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004) with quadrant probabilities (a,b,c,1-a-b-c),
 * no noise, no id permutation. Sample i draws its quadrant at recursion level l from the 16-bit
 * field (l mod 4) of the word gg_word(seed, 8*i + l/4), compared with the probabilities scaled to
 * 2^16 and rounded. The samples are symmetrised; self-loops and duplicates are dropped.
 * When weighted, omega(u,v) = 1 + (gg_key3(seed, min(u,v), max(u,v)) & 7), so both directions
 * and all duplicates of one pair carry the same weight. */
gg_graph *gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                  int weighted) {
  int64_t n = (int64_t)1 << scale;
  int64_t ns = edge_factor * n;
  uint32_t ta = (uint32_t)floor(a * 65536.0 + 0.5);
  uint32_t tb = ta + (uint32_t)floor(b * 65536.0 + 0.5);
  uint32_t tc = tb + (uint32_t)floor(c * 65536.0 + 0.5);
  uint32_t *su = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ns);
  uint32_t *sv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ns);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < ns; i++) {
    uint32_t u = 0, v = 0;
    uint64_t w = 0;
    for (int l = 0; l < scale; l++) {
      if ((l & 3) == 0) w = gg_word(seed, (uint64_t)(8 * i + (l >> 2)));
      uint32_t p = (uint32_t)((w >> (16 * (l & 3))) & 0xFFFF);
      uint32_t bu, bv;
      if (p < ta) { bu = 0; bv = 0; }
      else if (p < tb) { bu = 0; bv = 1; }
      else if (p < tc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    su[i] = u;
    sv[i] = v;
  }
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < ns; i++) {
    if (su[i] == sv[i]) continue;
    deg[su[i] + 1]++;
    deg[sv[i] + 1]++;
  }
  for (int64_t v = 0; v < n; v++) deg[v + 1] += deg[v];
  int64_t tot = deg[n];
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot ? tot : 1));
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(pos, deg, sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < ns; i++) {
    if (su[i] == sv[i]) continue;
    tmp[pos[su[i]]++] = (int32_t)sv[i];
    tmp[pos[sv[i]]++] = (int32_t)su[i];
  }
  free(pos);
  free(su);
  free(sv);
  gg_graph *g = gg_alloc(n);
  int64_t *cnt = g->off; /* reuse: cnt[v+1] = unique count of row v */
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; v++) {
    int32_t *row = tmp + deg[v];
    int64_t len = deg[v + 1] - deg[v];
    sort_i32(row, len);
    int64_t u = 0;
    for (int64_t t = 0; t < len; t++)
      if (t == 0 || row[t] != row[t - 1]) row[u++] = row[t];
    cnt[v + 1] = u;
  }
  for (int64_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
  g->m_dir = g->off[n];
  g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m_dir ? g->m_dir : 1));
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; v++)
    memcpy(g->adj + g->off[v], tmp + deg[v], sizeof(int32_t) * (size_t)(g->off[v + 1] - g->off[v]));
  free(tmp);
  free(deg);
  if (weighted) {
    g->ew = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m_dir ? g->m_dir : 1));
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; v++)
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
        uint64_t u = (uint64_t)g->adj[e];
        uint64_t lo = (uint64_t)v < u ? (uint64_t)v : u, hi = (uint64_t)v < u ? u : (uint64_t)v;
        g->ew[e] = 1 + (int32_t)(gg_key3(seed, lo, hi) & 7);
      }
  }
  return g;
}

/* ---------------------------------------------------------------- validation */
/* 0 = valid symmetric CSR; otherwise a code for the first violated rule. */
int gg_validate(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *ew) {
  if (off[0] != 0) return 1;
  for (int64_t v = 0; v < n; v++)
    if (off[v + 1] < off[v]) return 2;
  for (int64_t v = 0; v < n; v++)
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      int32_t u = adj[e];
      if (u < 0 || u >= n) return 3;
      if (u == v) return 4;
      if (e > off[v] && adj[e - 1] >= u) return 5;
      if (ew && ew[e] <= 0) return 6;
      /* reverse entry by binary search */
      int64_t lo = off[u], hi = off[u + 1];
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (adj[mid] < v) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= off[u + 1] || adj[lo] != v) return 7;
      if (ew && ew[lo] != ew[e]) return 8;
    }
  return 0;
}
