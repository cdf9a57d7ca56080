// match.cu -- matching-based clustering for the coarsening phase.
//
// The paper's clustering step (Section III-A) names matching algorithms (clusters of size two) as the
// alternative to size-constrained label propagation, and its conclusion (Section VII) plans a parallel
// matching for mesh-like graphs. This file implements the library's reading of it: deterministic
// handshake matching with the edge rating omega(u,v)^2 / (c(u) c(v)).
//
//   * Round r: every unmatched vertex v proposes to its best unmatched neighbour u with
//     c(v) + c(u) <= U -- largest rating (compared exactly as omega1^2 c(u2) vs omega2^2 c(u1) in
//     128-bit integers), then larger H(seed, min(u,v), max(u,v)), then smaller u. Proposals read the
//     matching of the round's start (a Jacobi step).
//   * v and u are matched when they propose to each other.
//   * Rounds repeat until one matches nothing or `rounds` have run; every kernel of a round reads the
//     previous round's pair count on the device and returns at once when it is zero, so the host
//     issues all rounds without waiting.
//   * label(v) = min(v, mate(v)) for matched v, else v; the clustering contracts like any other.
//
// Kernels: proposals of vertices of degree <= kSmallDeg by groups of 8 lanes (several vertices per
// warp, neighbour loads strided over the group, a shuffle reduction of the best candidate); larger
// degrees by one CTA each (a list built once per call). Acceptance and the final labels are one thread
// per vertex. Everything is integer work bound by memory traffic: per unmatched vertex its row offsets,
// its mate and weight, and per scanned entry the neighbour id, its mate, its weight and the edge weight.
#include <algorithm>
#include <vector>

#include "gp_internal.cuh"
#include "match.cuh"

namespace gp {
namespace {

constexpr int kGroup = 8;
constexpr int kSmallDeg = 256;
constexpr int kBigThreads = 256;

struct Cand {
  long long w;
  long long c;
  unsigned long long h;
  int u;  // -1: none
};

__device__ __forceinline__ Cand no_cand() {
  Cand x;
  x.w = 0;
  x.c = 1;
  x.h = 0;
  x.u = -1;
  return x;
}

// a better than b: larger w^2 / c, then larger h, then smaller u
__device__ __forceinline__ bool cand_better(const Cand &a, const Cand &b) {
  if (a.u < 0) return false;
  if (b.u < 0) return true;
  const unsigned __int128 x = (unsigned __int128)(unsigned long long)a.w * (unsigned long long)a.w *
                              (unsigned long long)b.c;
  const unsigned __int128 y = (unsigned __int128)(unsigned long long)b.w * (unsigned long long)b.w *
                              (unsigned long long)a.c;
  if (x != y) return x > y;
  if (a.h != b.h) return a.h > b.h;
  return a.u < b.u;
}

__device__ __forceinline__ Cand shfl_cand(const Cand &a, int o) {
  Cand r;
  r.w = __shfl_xor_sync(kFull, a.w, o);
  r.c = __shfl_xor_sync(kFull, a.c, o);
  r.h = __shfl_xor_sync(kFull, a.h, o);
  r.u = __shfl_xor_sync(kFull, a.u, o);
  return r;
}

// Candidate neighbour u over entry e of vertex v (weight cv), or none.
template <int EW>
__device__ __forceinline__ Cand cand_of(const DGraph &g, const int32_t *mate, int64_t U, uint64_t smix, int v,
                                        long long cv, int64_t e) {
  const int u = __ldg(g.adj + e);
  if (mate[u] >= 0) return no_cand();
  const long long cu = g.vweight(u);
  if (cv + cu > U) return no_cand();
  Cand x;
  x.w = load_ew<EW>(g.ew, e);
  x.c = cu;
  const int lo = min(u, v), hi = max(u, v);
  x.h = mix64(mix64(smix ^ (uint64_t)(uint32_t)lo) ^ (uint64_t)(uint32_t)hi);
  x.u = u;
  return x;
}

__device__ __forceinline__ bool round_live(const unsigned long long *pairs, int r) {
  return r == 0 || pairs[r - 1] != 0;
}

// stats[0] visits, stats[1] scanned entries, summed over the warp (at most 32 * kSmallDeg entries)
__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned vis, unsigned ent) {
  vis = __reduce_add_sync(kFull, vis);
  ent = __reduce_add_sync(kFull, ent);
  if ((threadIdx.x & 31) == 0) {
    if (vis) atomicAdd(&stats[0], (unsigned long long)vis);
    if (ent) atomicAdd(&stats[1], (unsigned long long)ent);
  }
}

template <int EW>
__global__ void k_propose_small(DGraph g, const int32_t *mate, int32_t *prop, int64_t U, uint64_t smix,
                                const unsigned long long *pairs, int r, unsigned long long *stats) {
  if (!round_live(pairs, r)) return;
  const int lane_g = threadIdx.x & (kGroup - 1);
  const int64_t groups = (int64_t)gridDim.x * blockDim.x / kGroup;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
  // every lane of a warp runs the same number of iterations (the shuffles need all 32)
  const int64_t iters = (g.n + groups - 1) / groups;
  for (int64_t it = 0; it < iters; it++) {
    const int64_t v = g0 + it * groups;
    bool live = v < g.n;
    int64_t rb = 0, re = 0;
    if (live) {
      rb = g.row_begin(v);
      re = g.row_begin(v + 1);
      live = mate[v] < 0 && re - rb <= kSmallDeg;
    }
    Cand best = no_cand();
    long long cv = 0;
    if (live) {
      cv = g.vweight(v);
      for (int64_t e = rb + lane_g; e < re; e += kGroup) {
        const Cand x = cand_of<EW>(g, mate, U, smix, (int)v, cv, e);
        if (cand_better(x, best)) best = x;
      }
    }
#pragma unroll
    for (int o = kGroup / 2; o > 0; o >>= 1) {
      const Cand x = shfl_cand(best, o);
      if (cand_better(x, best)) best = x;
    }
    if (live && lane_g == 0) prop[v] = best.u;
    else if (v < g.n && lane_g == 0 && re - rb <= kSmallDeg) prop[v] = -1;
    add_stats(stats, (live && lane_g == 0) ? 1u : 0u, (live && lane_g == 0) ? (unsigned)(re - rb) : 0u);
  }
}

// vertices of degree > kSmallDeg, one CTA each
template <int EW>
__global__ void k_propose_big(DGraph g, const int32_t *mate, int32_t *prop, int64_t U, uint64_t smix,
                              const unsigned long long *pairs, int r, const int32_t *big, const unsigned *nbig,
                              unsigned long long *stats) {
  if (!round_live(pairs, r)) return;
  __shared__ Cand sb[kBigThreads / 32];
  const unsigned cnt = *nbig;
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int v = big[i];
    const bool live = mate[v] < 0;  // (uniform over the block)
    if (!live) {
      if (threadIdx.x == 0) prop[v] = -1;
      continue;
    }
    const int64_t rb = g.row_begin(v), re = g.row_begin(v + 1);
    const long long cv = g.vweight(v);
    Cand best = no_cand();
    for (int64_t e = rb + threadIdx.x; e < re; e += kBigThreads) {
      const Cand x = cand_of<EW>(g, mate, U, smix, v, cv, e);
      if (cand_better(x, best)) best = x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Cand x = shfl_cand(best, o);
      if (cand_better(x, best)) best = x;
    }
    if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      Cand b = sb[0];
      for (int w = 1; w < kBigThreads / 32; w++)
        if (cand_better(sb[w], b)) b = sb[w];
      prop[v] = b.u;
      atomicAdd(&stats[0], 1ull);
      atomicAdd(&stats[1], (unsigned long long)(re - rb));
    }
    __syncthreads();
  }
}

__global__ void k_list_big(DGraph g, int32_t *big, unsigned *nbig) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    if (g.row_begin(v + 1) - g.row_begin(v) > kSmallDeg) big[atomicAdd(nbig, 1u)] = (int32_t)v;
  }
}

__global__ void k_accept(int64_t n, int32_t *mate, const int32_t *prop, unsigned long long *pairs, int r) {
  if (!round_live(pairs, r)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (n + stride - 1) / stride;
  for (int64_t it = 0; it < iters; it++) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + it * stride;
    bool pair = false;
    if (v < n && mate[v] < 0) {
      const int u = prop[v];
      if (u >= 0 && prop[u] == (int32_t)v) {
        mate[v] = u;
        pair = v < u;
      }
    }
    const unsigned c = __popc(__ballot_sync(kFull, pair));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&pairs[r], (unsigned long long)c);
  }
}

__global__ void k_match_labels(int64_t n, const int32_t *mate, int32_t *labels) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int m = mate[v];
    labels[v] = (m >= 0 && m < v) ? m : (int32_t)v;
  }
}

__global__ void k_fill(int32_t *a, int64_t n, int32_t x) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) a[v] = x;
}

int grid_for(int64_t items, int per_block) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + per_block - 1) / per_block, (int64_t)num_sms() * 8));
}

}  // namespace

int run_match(const DGraph &g, int64_t U, int rounds, uint64_t seed, int32_t *labels, MatchStats *out,
              cudaStream_t s, bool read_stats) {
  if (out) *out = MatchStats();
  if (g.n <= 0) return GP_OK;
  Workspace ws(s);
  int32_t *mate, *prop, *big;
  unsigned *nbig;
  unsigned long long *pairs, *stats;
  const int R = std::max(rounds, 0);
  GP_TRY(ws.get(&mate, (size_t)g.n));
  GP_TRY(ws.get(&prop, (size_t)g.n));
  GP_TRY(ws.get(&big, (size_t)g.n));
  GP_TRY(ws.zeros(&nbig, 1));
  GP_TRY(ws.zeros(&pairs, (size_t)R + 1));
  GP_TRY(ws.zeros(&stats, 2));
  const uint64_t smix = mix64(seed);
  const int gn = grid_for(g.n, 256);
  (count_launch(), k_fill<<<gn, 256, 0, s>>>(mate, g.n, -1));
  (count_launch(), k_list_big<<<gn, 256, 0, s>>>(g, big, nbig));
  GP_LAUNCH_CHECK();
  const int gsmall = grid_for(g.n * kGroup, 256);
  const int gbig = num_sms() * 4;
  const int ew = g.ew_mode();
  for (int r = 0; r < R; r++) {
    ProfScope ps("match_round", s);
    if (ew == 0) {
      (count_launch(), k_propose_small<0><<<gsmall, 256, 0, s>>>(g, mate, prop, U, smix, pairs, r, stats));
      (count_launch(), k_propose_big<0><<<gbig, kBigThreads, 0, s>>>(g, mate, prop, U, smix, pairs, r, big, nbig, stats));
    } else if (ew == 1) {
      (count_launch(), k_propose_small<1><<<gsmall, 256, 0, s>>>(g, mate, prop, U, smix, pairs, r, stats));
      (count_launch(), k_propose_big<1><<<gbig, kBigThreads, 0, s>>>(g, mate, prop, U, smix, pairs, r, big, nbig, stats));
    } else {
      (count_launch(), k_propose_small<2><<<gsmall, 256, 0, s>>>(g, mate, prop, U, smix, pairs, r, stats));
      (count_launch(), k_propose_big<2><<<gbig, kBigThreads, 0, s>>>(g, mate, prop, U, smix, pairs, r, big, nbig, stats));
    }
    (count_launch(), k_accept<<<gn, 256, 0, s>>>(g.n, mate, prop, pairs, r));
    GP_LAUNCH_CHECK();
  }
  (count_launch(), k_match_labels<<<gn, 256, 0, s>>>(g.n, mate, labels));
  GP_LAUNCH_CHECK();
  if (!read_stats && !profiling()) return GP_OK;
  std::vector<unsigned long long> hp((size_t)R + 1), hs(2);
  GP_CUDA(cudaMemcpyAsync(hp.data(), pairs, sizeof(unsigned long long) * (R + 1), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaMemcpyAsync(hs.data(), stats, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  MatchStats m;
  for (int r = 0; r < R; r++) {
    m.rounds = r + 1;
    m.pairs += (int64_t)hp[r];
    if (hp[r] == 0) break;
  }
  m.visits = (int64_t)hs[0];
  m.edges = (int64_t)hs[1];
  // algorithmic bytes: per visit two offsets, own mate, own weight, proposal write; per scanned entry
  // the neighbour id, its mate, its weight and the edge weight
  const int64_t vb = 2 * g.offset_bytes() + 4 + g.vw_bytes() + 4;
  const int64_t eb = 4 + 4 + g.vw_bytes() + g.ew_bytes();
  prof_add_counts("match_round", m.visits, m.edges, m.visits * vb + m.edges * eb);
  if (out) *out = m;
  return GP_OK;
}

}  // namespace gp
