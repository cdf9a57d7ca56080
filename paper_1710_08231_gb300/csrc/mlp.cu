// mlp.cu -- learned edge scorer: per-edge features, BF16 tensor-core inference, training kernels.
//
// The paper has no learned component. This scorer guides label propagation during coarsening: its
// quantised score q = round-half-even(s * 2^15) of each CSR entry breaks ties between equally
// connected labels (larger score sum first) and orders admission after the gain.
//
// Features of entry (v,u), symmetric in v and u (rows of degree above 512 are spread over a CTA):
//   0 log2(1 + min(d(v), d(u)))        1 log2(1 + max(d(v), d(u)))
//   2 log2(1 + omega(v,u))             3 log2(1 + min(c(v), c(u)))
//   4 log2(1 + max(c(v), c(u)))
//   5 |first64(N(v)) intersect first64(N(u))| / 64
//   6 omega(v,u) / max(wdeg(v), wdeg(u))
//   7 level / 16
// Network: h = relu(W1 x + b1) (32 hidden), s = sigmoid(w2 . h + b2). Inference multiplies BF16
// features by BF16 W1 on the tensor cores (mma.sync m16n8k16, FP32 accumulation), rounds the hidden
// activations to BF16 and finishes the second layer in FP32. Training runs full-batch Adam on FP32
// master weights; its forward pass uses the BF16-rounded weights that inference uses.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mlp.cuh"

namespace gp {

namespace {

constexpr int kIn = 8, kHid = 32, kParams = kHid * kIn + kHid + kHid + 1;  // 321

__device__ __forceinline__ int64_t gp_min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ float bf16_to_float(uint16_t b) {
  return __uint_as_float(((unsigned)b) << 16);
}

__device__ __forceinline__ uint16_t float_to_bf16(float f) {
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t *>(&h);
}

__device__ __forceinline__ unsigned pack2(uint16_t lo, uint16_t hi) { return (unsigned)lo | ((unsigned)hi << 16); }

__global__ void k_wdeg(DGraph g, float *wdeg) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = gw; v < g.n; v += nw) {
    const int64_t b = g.row_begin(v), e = g.row_begin(v + 1);
    double s = 0;
    for (int64_t x = b + lane; x < e; x += 32) s += (double)g.eweight(x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) wdeg[v] = (float)s;
  }
}

// Features of entry e = (v,u) of v's row (called by one lane per entry; `has` false for the lanes past
// the row's end). The shared-neighbour count: the lane takes the first 64 neighbours of u and looks
// each up in `tab`, the set of v's first 64 neighbours (an open-addressing table of kTab slots in shared
// memory, slot mix32(x) mod kTab, linear probing).
constexpr int kTab = 128;  // set slots (at most 64 keys)
constexpr int64_t kFeatSmall = 512;  // rows up to this degree: a half-warp per vertex; longer: a CTA

template <bool BF16>
__device__ __forceinline__ void feature_entry(const DGraph &g, const float *wdeg, int64_t e, bool has, int64_t dv,
                                              float cv, float wv, const int *tab, float flevel, float *fout,
                                              unsigned *bout) {
  const int u = has ? g.adj[e] : 0;
  const int64_t bu = has ? g.row_begin(u) : 0;
  const int64_t eu = has ? g.row_begin(u + 1) : 0;
  const int lenu = (int)gp_min64(eu - bu, 64);
  // u's weight, its weighted degree and the entry's weight are loaded before the search
  const float cu = has ? (float)g.vweight(u) : 0.0f;
  const float wu = has ? wdeg[u] : 0.0f;
  const float w = has ? (float)g.eweight(e) : 0.0f;
  int mine = 0;
  // eight of u's neighbours are loaded before any is searched (independent loads in flight)
  constexpr int kBatch = 8;
  for (int k0 = 0; k0 < lenu; k0 += kBatch) {
    int xs[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; q++) xs[q] = k0 + q < lenu ? __ldg(g.adj + bu + k0 + q) : 0;
#pragma unroll
    for (int q = 0; q < kBatch; q++) {
      if (k0 + q >= lenu) break;
      const int x = xs[q];
      unsigned sl = mix32((unsigned)x) & (kTab - 1);
      while (true) {
        const int k = tab[sl];
        if (k == x) {
          mine++;
          break;
        }
        if (k == -1) break;
        sl = (sl + 1) & (kTab - 1);
      }
    }
  }
  if (!has) return;
  const float du = (float)(eu - bu);
  const float dvf = (float)dv;
  float f[kIn];
  f[0] = log2f(1.0f + fminf(dvf, du));
  f[1] = log2f(1.0f + fmaxf(dvf, du));
  f[2] = log2f(1.0f + w);
  f[3] = log2f(1.0f + fminf(cv, cu));
  f[4] = log2f(1.0f + fmaxf(cv, cu));
  f[5] = (float)mine / 64.0f;
  f[6] = w / fmaxf(wv, wu);
  f[7] = flevel;
  if (BF16) {
#pragma unroll
    for (int i = 0; i < 4; i++) bout[e * 4 + i] = pack2(float_to_bf16(f[2 * i]), float_to_bf16(f[2 * i + 1]));
  } else {
#pragma unroll
    for (int i = 0; i < kIn; i++) fout[e * kIn + i] = f[i];
  }
}

// Rows of degree <= kFeatSmall: one half-warp (16 lanes) per vertex, each lane one entry of a 16-entry
// step; the set of v's first 64 neighbours is the half-warp's own table.
template <bool BF16>
__global__ void __launch_bounds__(256, 6) k_features(DGraph g, int level, const float *wdeg, float *fout, unsigned *bout) {
  constexpr int kH = 16;  // lanes per vertex
  __shared__ int tab_s[8][2][kTab];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane / kH, hl = lane % kH;
  const unsigned hmask = 0xFFFFu << (kH * half);
  int *tab = tab_s[wid][half];
  const int64_t gh = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kH;
  const int64_t nh = ((int64_t)gridDim.x * blockDim.x) / kH;
  const float flevel = (float)level / 16.0f;
  for (int64_t v = gh; v < g.n; v += nh) {
    const int64_t beg = g.row_begin(v), end = g.row_begin(v + 1);
    const int64_t dv = end - beg;
    if (dv == 0 || dv > kFeatSmall) continue;  // (uniform over the half-warp)
    const int lenv = (int)gp_min64(dv, 64);
    __syncwarp(hmask);
    for (int t = hl; t < kTab; t += kH) tab[t] = -1;
    __syncwarp(hmask);
    for (int t = hl; t < lenv; t += kH) {
      const int x = g.adj[beg + t];
      unsigned sl = mix32((unsigned)x) & (kTab - 1);
      while (atomicCAS(&tab[sl], -1, x) != -1) sl = (sl + 1) & (kTab - 1);  // ids in a row are distinct
    }
    __syncwarp(hmask);
    const float cv = (float)g.vweight(v);
    const float wv = wdeg[v];
    for (int64_t e0 = beg; e0 < end; e0 += kH) {
      const int64_t e = e0 + hl;
      feature_entry<BF16>(g, wdeg, e, e < end, dv, cv, wv, tab, flevel, fout, bout);
    }
  }
}

// Rows of degree > kFeatSmall (hubs of power-law graphs): one CTA per vertex, its 16 half-warps taking
// 16-entry steps of the row in turn, one shared set of v's first 64 neighbours. A row is thus spread
// over 256 lanes instead of 16, which keeps the longest rows from deciding the kernel's duration.
__global__ void k_list_feat_big(DGraph g, int32_t *big, unsigned *nbig) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
    if (g.row_begin(v + 1) - g.row_begin(v) > kFeatSmall) big[atomicAdd(nbig, 1u)] = (int32_t)v;
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_features_big(DGraph g, int level, const float *wdeg, float *fout,
                                                      unsigned *bout, const int32_t *big, const unsigned *nbig) {
  __shared__ int tab[kTab];
  const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15;
  const float flevel = (float)level / 16.0f;
  const unsigned cnt = *nbig;
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int v = big[i];
    const int64_t beg = g.row_begin(v), end = g.row_begin(v + 1);
    const int64_t dv = end - beg;
    for (int t = threadIdx.x; t < kTab; t += blockDim.x) tab[t] = -1;
    __syncthreads();
    if (threadIdx.x < 64) {
      const int x = g.adj[beg + threadIdx.x];  // (dv > 64)
      unsigned sl = mix32((unsigned)x) & (kTab - 1);
      while (atomicCAS(&tab[sl], -1, x) != -1) sl = (sl + 1) & (kTab - 1);
    }
    __syncthreads();
    const float cv = (float)g.vweight(v);
    const float wv = wdeg[v];
    for (int64_t e0 = beg + hw * 16; e0 < end; e0 += 256) {
      const int64_t e = e0 + hl;
      feature_entry<BF16>(g, wdeg, e, e < end, dv, cv, wv, tab, flevel, fout, bout);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void mma_16816(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp scores 16 entries per step: A = 16 entries x 16 features (8 used, 8 zero), B = W1^T in
// four 16x8 slices (32 hidden units). Thread (g = lane/4, t = lane%4) holds features 2t, 2t+1 of
// rows g and g+8, and C elements (rows g, g+8; hidden units 8nb + 2t, 8nb + 2t + 1).
__global__ void __launch_bounds__(256) k_mlp_score(const unsigned *fb, int64_t m, const gp_mlp *mlp, float *s_out,
                                                   int32_t *q_out) {
  const int lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  unsigned bfrag[4][2];
  float bias[4][2], w2v[4][2];
#pragma unroll
  for (int nb = 0; nb < 4; nb++) {
    const int j = nb * 8 + gq;
    bfrag[nb][0] = pack2(mlp->w1[j * kIn + 2 * t], mlp->w1[j * kIn + 2 * t + 1]);
    bfrag[nb][1] = 0;  // features 8..15 are zero
    bias[nb][0] = mlp->b1[nb * 8 + 2 * t];
    bias[nb][1] = mlp->b1[nb * 8 + 2 * t + 1];
    w2v[nb][0] = bf16_to_float(mlp->w2[nb * 8 + 2 * t]);
    w2v[nb][1] = bf16_to_float(mlp->w2[nb * 8 + 2 * t + 1]);
  }
  const float b2 = mlp->b2;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tiles = (m + 15) / 16;
  for (int64_t tile = gw; tile < tiles; tile += nw) {
    const int64_t r0 = tile * 16 + gq, r1 = r0 + 8;
    unsigned a[4];
    a[0] = r0 < m ? fb[r0 * 4 + t] : 0u;
    a[1] = r1 < m ? fb[r1 * 4 + t] : 0u;
    a[2] = 0u;
    a[3] = 0u;
    float z0 = 0.f, z1 = 0.f;
#pragma unroll
    for (int nb = 0; nb < 4; nb++) {
      float c[4] = {bias[nb][0], bias[nb][1], bias[nb][0], bias[nb][1]};
      mma_16816(c, a, bfrag[nb]);
      // hidden activations are rounded to BF16 before the second layer
      const float h0 = bf16_to_float(float_to_bf16(fmaxf(c[0], 0.f)));
      const float h1 = bf16_to_float(float_to_bf16(fmaxf(c[1], 0.f)));
      const float h2 = bf16_to_float(float_to_bf16(fmaxf(c[2], 0.f)));
      const float h3 = bf16_to_float(float_to_bf16(fmaxf(c[3], 0.f)));
      z0 = fmaf(h0, w2v[nb][0], fmaf(h1, w2v[nb][1], z0));
      z1 = fmaf(h2, w2v[nb][0], fmaf(h3, w2v[nb][1], z1));
    }
    z0 += __shfl_xor_sync(kFull, z0, 1);
    z0 += __shfl_xor_sync(kFull, z0, 2);
    z1 += __shfl_xor_sync(kFull, z1, 1);
    z1 += __shfl_xor_sync(kFull, z1, 2);
    if (t == 0) {
      if (r0 < m) {
        const float s = 1.0f / (1.0f + expf(-(z0 + b2)));
        if (s_out) s_out[r0] = s;
        if (q_out) q_out[r0] = __float2int_rn(s * 32768.0f);
      }
      if (r1 < m) {
        const float s = 1.0f / (1.0f + expf(-(z1 + b2)));
        if (s_out) s_out[r1] = s;
        if (q_out) q_out[r1] = __float2int_rn(s * 32768.0f);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------ training
struct TrainWeights {
  float w1[kHid * kIn];
  float b1[kHid];
  float w2[kHid];
  float b2;
};

// Loss and gradient partial sums of one block (FP32), forward with the given weights.
__global__ void __launch_bounds__(256) k_grad(const float *x, const float *y, int64_t m, const TrainWeights *W,
                                              float *partials) {
  __shared__ float acc[kParams + 1];
  __shared__ TrainWeights sw;
  for (int p = threadIdx.x; p < kParams + 1; p += blockDim.x) acc[p] = 0.f;
  for (int p = threadIdx.x; p < (int)(sizeof(TrainWeights) / 4); p += blockDim.x)
    reinterpret_cast<float *>(&sw)[p] = reinterpret_cast<const float *>(W)[p];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float inv_m = 1.0f / (float)m;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = base + threadIdx.x;
    const bool valid = e < m;
    float xi[kIn];
#pragma unroll
    for (int i = 0; i < kIn; i++) xi[i] = valid ? x[e * kIn + i] : 0.f;
    const float ye = valid ? y[e] : 0.f;
    float pre[kHid];
    float z = sw.b2;
#pragma unroll
    for (int j = 0; j < kHid; j++) {
      float a = sw.b1[j];
#pragma unroll
      for (int i = 0; i < kIn; i++) a = fmaf(sw.w1[j * kIn + i], xi[i], a);
      pre[j] = a;
      z = fmaf(sw.w2[j], fmaxf(a, 0.f), z);
    }
    const float s = 1.0f / (1.0f + expf(-z));
    const float loss = valid ? (fmaxf(z, 0.f) - ye * z + log1pf(expf(-fabsf(z)))) : 0.f;
    const float dz = valid ? (s - ye) * inv_m : 0.f;
    // gradients of this entry, reduced over the warp one parameter at a time
    auto red = [&](float val, int p) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
      if (lane == 0) atomicAdd(&acc[p], val);
    };
#pragma unroll
    for (int j = 0; j < kHid; j++) {
      const float h = fmaxf(pre[j], 0.f);
      const float dh = pre[j] > 0.f ? dz * sw.w2[j] : 0.f;
#pragma unroll
      for (int i = 0; i < kIn; i++) red(dh * xi[i], j * kIn + i);
      red(dh, kHid * kIn + j);
      red(dz * h, kHid * kIn + kHid + j);
    }
    red(dz, kHid * kIn + 2 * kHid);
    red(loss * inv_m, kParams);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kParams + 1; p += blockDim.x) partials[(size_t)blockIdx.x * (kParams + 1) + p] = acc[p];
}

__global__ void k_grad_sum(const float *partials, int nblocks, float *out) {
  for (int p = threadIdx.x; p < kParams + 1; p += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nblocks; b++) s += partials[(size_t)b * (kParams + 1) + p];
    out[p] = (float)s;
  }
}

// Adam step on the FP32 master weights; writes the BF16 weights used by inference and the next
// forward pass.
__global__ void k_adam(const float *grad, TrainWeights *master, TrainWeights *fwd, float *mom, float *vel, int step,
                       float lr, gp_mlp *mlp, float *loss_log) {
  const float beta1 = 0.9f, beta2 = 0.999f, epsv = 1e-8f;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  float *wm = reinterpret_cast<float *>(master);
  float *wf = reinterpret_cast<float *>(fwd);
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    const float g = grad[p];
    mom[p] = beta1 * mom[p] + (1.f - beta1) * g;
    vel[p] = beta2 * vel[p] + (1.f - beta2) * g * g;
    wm[p] -= lr * (mom[p] / c1) / (sqrtf(vel[p] / c2) + epsv);
    if (p < kHid * kIn) {
      const uint16_t b = float_to_bf16(wm[p]);
      mlp->w1[p] = b;
      wf[p] = bf16_to_float(b);
    } else if (p < kHid * kIn + kHid) {
      mlp->b1[p - kHid * kIn] = wm[p];
      wf[p] = wm[p];
    } else if (p < kHid * kIn + 2 * kHid) {
      const uint16_t b = float_to_bf16(wm[p]);
      mlp->w2[p - kHid * kIn - kHid] = b;
      wf[p] = bf16_to_float(b);
    } else {
      mlp->b2 = wm[p];
      wf[p] = wm[p];
    }
  }
  if (threadIdx.x == 0 && loss_log) loss_log[step - 1] = grad[kParams];
}

// Master/forward weights from the gp_mlp (BF16 weights become exact FP32 values).
__global__ void k_weights_from(const gp_mlp *mlp, TrainWeights *master, TrainWeights *fwd) {
  float *wm = reinterpret_cast<float *>(master);
  float *wf = reinterpret_cast<float *>(fwd);
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    float v;
    if (p < kHid * kIn) v = bf16_to_float(mlp->w1[p]);
    else if (p < kHid * kIn + kHid) v = mlp->b1[p - kHid * kIn];
    else if (p < kHid * kIn + 2 * kHid) v = bf16_to_float(mlp->w2[p - kHid * kIn - kHid]);
    else v = mlp->b2;
    wm[p] = v;
    wf[p] = v;
  }
}

int grid_for(int64_t items, int per_block, int limit) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + per_block - 1) / per_block, limit));
}

int features(const DGraph &g, int level, float *fout, unsigned *bout, cudaStream_t s) {
  if (g.m == 0) return GP_OK;
  Workspace ws(s);
  float *wdeg;
  GP_TRY(ws.get(&wdeg, (size_t)g.n));
  const int nsm = num_sms();
  int32_t *big;
  unsigned *nbig;
  GP_TRY(ws.get(&big, (size_t)g.n));
  GP_TRY(ws.zeros(&nbig, 1));
  (::gp::count_launch(), k_wdeg<<<grid_for(g.n * 32, 256, nsm * 8), 256, 0, s>>>(g, wdeg));
  (::gp::count_launch(), k_list_feat_big<<<grid_for(g.n, 256, nsm * 8), 256, 0, s>>>(g, big, nbig));
  {
    ProfScope ps("mlp_features", s);
    if (bout) {
      (::gp::count_launch(), k_features<true><<<grid_for(g.n * 16, 256, nsm * 6), 256, 0, s>>>(g, level, wdeg, nullptr, bout));
      (::gp::count_launch(), k_features_big<true><<<nsm * 8, 256, 0, s>>>(g, level, wdeg, nullptr, bout, big, nbig));
    } else {
      (::gp::count_launch(), k_features<false><<<grid_for(g.n * 16, 256, nsm * 6), 256, 0, s>>>(g, level, wdeg, fout, nullptr));
      (::gp::count_launch(), k_features_big<false><<<nsm * 8, 256, 0, s>>>(g, level, wdeg, fout, nullptr, big, nbig));
    }
  }
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace

int mlp_score(const DGraph &g, int level, const gp_mlp *mlp, float *s_out, int32_t *q_out, cudaStream_t s) {
  if (g.m == 0) return GP_OK;
  Workspace ws(s);
  unsigned *fb;
  GP_TRY(ws.get(&fb, (size_t)g.m * 4));
  GP_TRY(features(g, level, nullptr, fb, s));
  {
    ProfScope ps("mlp_score_mma", s);
    (::gp::count_launch(), k_mlp_score<<<grid_for((g.m + 15) / 16, 8, num_sms() * 8), 256, 0, s>>>(fb, g.m, mlp, s_out, q_out));
  }
  GP_LAUNCH_CHECK();
  prof_add_counts("mlp_score_mma", g.m, g.m, g.m * (16 + 4 + (s_out ? 4 : 0)));
  return GP_OK;
}

int mlp_train(const float *x, const float *y, int64_t m, gp_mlp *mlp, int steps, float lr, float *loss_host,
              float *grad_host, cudaStream_t s) {
  Workspace ws(s);
  TrainWeights *master, *fwd;
  float *mom, *vel, *partials, *grad, *losses;
  GP_TRY(ws.get(&master, 1));
  GP_TRY(ws.get(&fwd, 1));
  GP_TRY(ws.zeros(&mom, kParams));
  GP_TRY(ws.zeros(&vel, kParams));
  const int nb = grid_for(m, 256, num_sms() * 4);
  GP_TRY(ws.get(&partials, (size_t)nb * (kParams + 1)));
  GP_TRY(ws.get(&grad, kParams + 1));
  GP_TRY(ws.get(&losses, (size_t)std::max(steps, 1)));
  (::gp::count_launch(), k_weights_from<<<1, 352, 0, s>>>(mlp, master, fwd));
  if (steps <= 0) {
    // gradient only
    (::gp::count_launch(), k_grad<<<nb, 256, 0, s>>>(x, y, m, fwd, partials));
    (::gp::count_launch(), k_grad_sum<<<1, 352, 0, s>>>(partials, nb, grad));
    GP_LAUNCH_CHECK();
    if (grad_host) GP_CUDA(cudaMemcpyAsync(grad_host, grad, sizeof(float) * (kParams + 1), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
  }
  for (int st = 1; st <= steps; st++) {
    (::gp::count_launch(), k_grad<<<nb, 256, 0, s>>>(x, y, m, fwd, partials));
    (::gp::count_launch(), k_grad_sum<<<1, 352, 0, s>>>(partials, nb, grad));
    (::gp::count_launch(), k_adam<<<1, 352, 0, s>>>(grad, master, fwd, mom, vel, st, lr, mlp, losses));
  }
  GP_LAUNCH_CHECK();
  if (loss_host) GP_CUDA(cudaMemcpyAsync(loss_host, losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" {

int gp_mlp_score(const gp_graph *g, int32_t level, const gp_mlp *mlp, float *s_out, int32_t *q_out, gp_stream stream) {
  if (!g || !mlp || g->n < 0 || g->m_dir < 0) {
    set_error("gp_mlp_score: graph and mlp are required");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GP_TRY(mlp_score(make_dgraph(g), level, mlp, s_out, q_out, s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_edge_features(const gp_graph *g, int32_t level, float *feat_out, gp_stream stream) {
  if (!g || !feat_out || g->n < 0 || g->m_dir < 0) {
    set_error("gp_edge_features: graph and output are required");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GP_TRY(features(make_dgraph(g), level, feat_out, nullptr, s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_mlp_train(const float *feat, const float *y, int64_t m, gp_mlp *mlp, int32_t steps, float lr, float *loss_out,
                 gp_stream stream) {
  if (!feat || !y || m <= 0 || !mlp || steps < 1) {
    set_error("gp_mlp_train: feat, y, m > 0, mlp and steps >= 1 are required");
    return GP_ERR_INVALID_ARG;
  }
  return mlp_train(feat, y, m, mlp, steps, lr, loss_out, nullptr, (cudaStream_t)stream);
}

int gp_mlp_grad(const float *feat, const float *y, int64_t m, const gp_mlp *mlp, float *loss_out, float *grad_out,
                gp_stream stream) {
  if (!feat || !y || m <= 0 || !mlp) {
    set_error("gp_mlp_grad: feat, y, m > 0 and mlp are required");
    return GP_ERR_INVALID_ARG;
  }
  std::vector<float> g(kParams + 1);
  GP_TRY(mlp_train(feat, y, m, const_cast<gp_mlp *>(mlp), 0, 0.f, nullptr, g.data(), (cudaStream_t)stream));
  if (grad_out) std::memcpy(grad_out, g.data(), sizeof(float) * kParams);
  if (loss_out) *loss_out = g[kParams];
  return GP_OK;
}

}  // extern "C"
