// mlp.cpp -- oracle: per-edge features and the 8->32->1 edge-scoring network in FP64.
//
// TEST INFRASTRUCTURE ONLY (CPU oracle; shares no code with the GPU library).
//
// The paper has no learned component; this scorer guides the label-propagation tie-break and
// admission order during coarsening (the coarsening step of Section III-A / Section IV-A). Features
// of CSR entry (v,u), symmetric in v and u:
//   0 log2(1 + min(d(v), d(u)))        1 log2(1 + max(d(v), d(u)))
//   2 log2(1 + omega(v,u))             3 log2(1 + min(c(v), c(u)))
//   4 log2(1 + max(c(v), c(u)))
//   5 |first64(N(v)) intersect first64(N(u))| / 64   (first 64 entries of each sorted row)
//   6 omega(v,u) / max(wdeg(v), wdeg(u)), wdeg = sum of incident edge weights
//   7 level / 16
// Network: h = relu(W1 x + b1) with W1 row-major [32][8]; s = sigmoid(w2 . h + b2).
// Loss: mean binary cross-entropy over the rows, written through the logit z:
//   softplus(z) - y z = max(z, 0) - y z + log(1 + exp(-|z|)); dLoss/dz = (sigmoid(z) - y) / m.
#include <cmath>
#include <vector>

#include "oracle.h"

namespace {
constexpr int kIn = 8, kHid = 32;

int64_t shared_first64(const or_graph *g, int32_t v, int32_t u) {
  int64_t a = g->off[v], ae = std::min(g->off[v + 1], g->off[v] + 64);
  int64_t b = g->off[u], be = std::min(g->off[u + 1], g->off[u] + 64);
  int64_t cnt = 0;
  while (a < ae && b < be) {
    if (g->adj[a] < g->adj[b]) a++;
    else if (g->adj[a] > g->adj[b]) b++;
    else {
      cnt++;
      a++;
      b++;
    }
  }
  return cnt;
}

double logit(const double *x, const double *w1, const double *b1, const double *w2, double b2,
             double *pre) {
  double z = b2;
  for (int j = 0; j < kHid; j++) {
    double a = b1[j];
    for (int i = 0; i < kIn; i++) a += w1[j * kIn + i] * x[i];
    pre[j] = a;
    z += w2[j] * (a > 0.0 ? a : 0.0);
  }
  return z;
}
}  // namespace

extern "C" void or_edge_features(const or_graph *g, int64_t level, double *feat) {
  std::vector<double> wdeg(g->n, 0.0);
  for (int64_t v = 0; v < g->n; v++)
    for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) wdeg[v] += g->ew ? (double)g->ew[e] : 1.0;
  for (int64_t v = 0; v < g->n; v++) {
    const double dv = (double)(g->off[v + 1] - g->off[v]);
    const double cv = g->vw ? (double)g->vw[v] : 1.0;
    for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
      const int32_t u = g->adj[e];
      const double du = (double)(g->off[u + 1] - g->off[u]);
      const double cu = g->vw ? (double)g->vw[u] : 1.0;
      const double w = g->ew ? (double)g->ew[e] : 1.0;
      double *f = feat + e * kIn;
      f[0] = std::log2(1.0 + std::min(dv, du));
      f[1] = std::log2(1.0 + std::max(dv, du));
      f[2] = std::log2(1.0 + w);
      f[3] = std::log2(1.0 + std::min(cv, cu));
      f[4] = std::log2(1.0 + std::max(cv, cu));
      f[5] = (double)shared_first64(g, (int32_t)v, u) / 64.0;
      f[6] = w / std::max(wdeg[v], wdeg[u]);
      f[7] = (double)level / 16.0;
    }
  }
}

extern "C" void or_mlp_forward(int64_t m, const double *x, const double *w1, const double *b1,
                               const double *w2, double b2, double *s_out) {
  double pre[kHid];
  for (int64_t r = 0; r < m; r++) {
    const double z = logit(x + r * kIn, w1, b1, w2, b2, pre);
    s_out[r] = 1.0 / (1.0 + std::exp(-z));
  }
}

extern "C" double or_mlp_loss_grad(int64_t m, const double *x, const double *y, const double *w1,
                                   const double *b1, const double *w2, double b2, double *gw1,
                                   double *gb1, double *gw2, double *gb2) {
  for (int j = 0; j < kHid * kIn; j++) gw1[j] = 0.0;
  for (int j = 0; j < kHid; j++) gb1[j] = gw2[j] = 0.0;
  *gb2 = 0.0;
  double loss = 0.0, pre[kHid];
  for (int64_t r = 0; r < m; r++) {
    const double *xr = x + r * kIn;
    const double z = logit(xr, w1, b1, w2, b2, pre);
    loss += std::max(z, 0.0) - y[r] * z + std::log1p(std::exp(-std::fabs(z)));
    const double dz = (1.0 / (1.0 + std::exp(-z)) - y[r]) / (double)m;
    *gb2 += dz;
    for (int j = 0; j < kHid; j++) {
      const double h = pre[j] > 0.0 ? pre[j] : 0.0;
      gw2[j] += dz * h;
      if (pre[j] > 0.0) {
        const double dh = dz * w2[j];
        gb1[j] += dh;
        for (int i = 0; i < kIn; i++) gw1[j * kIn + i] += dh * xr[i];
      }
    }
  }
  return loss / (double)m;
}
