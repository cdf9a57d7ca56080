// block_sort.cuh -- single-CTA primitives over global-memory arrays: stable LSD radix sort of
// (uint64 key, int32 value) pairs, stable compaction and segmented exclusive scans.
// All functions must be called by every thread of the block (blockDim.x = 1024, 32 warps).
#pragma once

#include "gp_internal.cuh"

namespace gp {

struct BlockSortSmem {
  unsigned hist[256];
  unsigned base[256];
  unsigned wcnt[32][256];
  long long tmp[32];
  long long tot;
  long long carry;
  int carry_seg;
  int flag;
};

// Stable LSD radix sort by the low `bits` bits of the keys. Returns true when the sorted result is
// in (kb, vb), false when it is in (ka, va).
__device__ inline bool block_radix_sort(unsigned long long *ka, int *va, unsigned long long *kb, int *vb, int P,
                                        int bits, BlockSortSmem &sm) {
  unsigned long long *ks = ka, *kd = kb;
  int *vs = va, *vd = vb;
  bool in_b = false;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int shift = 0; shift < bits; shift += 8) {
    for (int t = threadIdx.x; t < 256; t += blockDim.x) sm.hist[t] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < P; t += blockDim.x) atomicAdd(&sm.hist[(ks[t] >> shift) & 255], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned acc = 0;
      for (int t = 0; t < 256; t++) {
        sm.base[t] = acc;
        acc += sm.hist[t];
      }
    }
    __syncthreads();
    for (int t0 = 0; t0 < P; t0 += blockDim.x) {
      const int p = t0 + threadIdx.x;
      const bool valid = p < P;
      const unsigned long long key = valid ? ks[p] : 0;
      const int val = valid ? vs[p] : 0;
      const int dg = valid ? (int)((key >> shift) & 255) : 256;
      for (int k = threadIdx.x; k < nw * 256; k += blockDim.x) sm.wcnt[k >> 8][k & 255] = 0;
      __syncthreads();
      const unsigned peers = __match_any_sync(kFull, dg);
      const int rank = __popc(peers & lanemask_lt());
      if (valid && rank == 0) sm.wcnt[wid][dg] = __popc(peers);
      __syncthreads();
      if (valid) {
        unsigned pre = 0;
        for (int w = 0; w < wid; w++) pre += sm.wcnt[w][dg];
        const unsigned pos = sm.base[dg] + pre + rank;
        kd[pos] = key;
        vd[pos] = val;
      }
      __syncthreads();
      if (threadIdx.x < 256) {
        unsigned s = 0;
        for (int w = 0; w < nw; w++) s += sm.wcnt[w][threadIdx.x];
        sm.base[threadIdx.x] += s;
      }
      __syncthreads();
    }
    unsigned long long *tk = ks;
    ks = kd;
    kd = tk;
    int *tv = vs;
    vs = vd;
    vd = tv;
    in_b = !in_b;
  }
  return in_b;
}

// Stable compaction: out[0..count) = the indices i in [0, n) with pred(i), ascending. Returns count.
template <class Pred>
__device__ inline int block_compact(int n, Pred pred, int *out, BlockSortSmem &sm) {
  if (threadIdx.x == 0) sm.carry = 0;
  __syncthreads();
  for (int t0 = 0; t0 < n; t0 += blockDim.x) {
    const int i = t0 + threadIdx.x;
    const bool keep = i < n && pred(i);
    const long long ex = block_excl_scan64((long long)(keep ? 1 : 0), sm.tmp, &sm.tot);
    if (keep) out[sm.carry + ex] = i;
    __syncthreads();
    if (threadIdx.x == 0) sm.carry += sm.tot;
    __syncthreads();
  }
  const int r = (int)sm.carry;
  __syncthreads();
  return r;
}

// Segmented exclusive scan over positions [0, P): seg(p) names the segment (segments are
// contiguous), val(p) the addend; fn(p, excl, incl) is called once per position with the sums of the
// earlier positions of its segment (excl) and including it (incl).
template <class SegF, class ValF, class Fn>
__device__ inline void block_seg_scan(int P, SegF seg, ValF val, Fn fn, BlockSortSmem &sm) {
  if (threadIdx.x == 0) {
    sm.carry = 0;
    sm.carry_seg = -1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t0 = 0; t0 < P; t0 += blockDim.x) {
    const int p = t0 + threadIdx.x;
    const bool valid = p < P;
    const int sg = valid ? seg(p) : -2;
    const int sprev = valid ? (p == 0 ? -1 : (p == t0 ? sm.carry_seg : seg(p - 1))) : -2;
    const long long v = valid ? val(p) : 0;
    int f = (valid && sg != sprev) ? 1 : 0;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, x, o);
      const int fy = __shfl_up_sync(kFull, f, o);
      if (lane >= o) {
        if (!f) x += y;
        f |= fy;
      }
    }
    __shared__ long long wsum[32];
    __shared__ int wflag[32];
    if (lane == 31) {
      wsum[wid] = x;
      wflag[wid] = f;
    }
    __syncthreads();
    if (wid == 0) {
      long long s = lane < nw ? wsum[lane] : 0;
      int fl = lane < nw ? wflag[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, s, o);
        const int fy = __shfl_up_sync(kFull, fl, o);
        if (lane >= o) {
          if (!fl) s += y;
          fl |= fy;
        }
      }
      long long ps = __shfl_up_sync(kFull, s, 1);
      int pf = __shfl_up_sync(kFull, fl, 1);
      if (lane == 0) {
        ps = 0;
        pf = 0;
      }
      if (lane < nw) wsum[lane] = pf ? ps : ps + sm.carry;
    }
    __syncthreads();
    const long long incl = f ? x : x + wsum[wid];
    if (valid) fn(p, incl - v, incl);
    __syncthreads();
    const int last = min(P, t0 + (int)blockDim.x) - 1;
    if (p == last) {
      sm.carry = incl;
      sm.carry_seg = sg;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bits_of(unsigned long long x) { return x ? 64 - __clzll(x) : 0; }

}  // namespace gp
