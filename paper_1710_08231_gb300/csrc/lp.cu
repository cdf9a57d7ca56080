// lp.cu -- size-constrained label propagation on the GPU: one persistent cooperative kernel per call.
//
// Method: Section III-A ("Clustering") and Section IV-A ("Parallel Size-Constraint Label
// Propagation") of "High-Quality Shared-Memory Graph Partitioning"; as refinement with U = Lmax in
// Section III-C / IV-C. A vertex moves to the eligible cluster of strongest connection; a cluster is
// eligible when it stays within U after the move; neighbours of moved vertices are visited in the
// next iteration.
//
// GPU design (what replaces the paper's degree sort, TBB work packets and CAS on cluster sizes):
//   * each round has two Jacobi sub-rounds split by the hash bit H(seed, r, v) >> 63; all decisions of
//     a sub-round read the labels and label weights of its start, so the result does not depend on
//     the schedule;
//   * one cooperative launch runs every round of an LP call. The blocks of a "problem" (one LP run;
//     several independent runs can share a launch) meet at bounded barriers between the phases of a
//     sub-round: classify -> aggregate+choose -> admission with apply (-> contest when a target's
//     proposals do not all fit);
//   * active vertices are binned by degree: groups of 4/8/16/32 lanes (labels aggregated with
//     __match_any_sync), one warp with a shared-memory hash table, one CTA with a shared-memory hash
//     table, or several CTAs with a global-memory hash table for hubs;
//   * connection sums are exact integers and the choice is a total order (connection, score sum,
//     H(seed, v, L), -L), so the aggregation order never matters;
//   * admission is deterministic instead of CAS: proposals to one target are ordered by (gain desc,
//     score sum desc, id asc) and the longest prefix fitting under U is taken. When all proposals to a
//     target fit, no order is needed; otherwise the contested proposals are sorted (one CTA in shared
//     memory up to 4096, else a cooperative LSD radix sort) and admitted by a segmented prefix sum.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <vector>

#include "lp.cuh"

namespace gp {

namespace {

constexpr int kBins = 7;     // G4, G8, G16, G32, WARP, CTA, HUB
constexpr int kBinZero = 7;  // degree-0 visits (statistics only)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Shared-memory tables come in three classes TB, one kernel instance each:
//   TB = 0  runs with scores: 16-byte slots (8-byte sum, 4-byte label, 4-byte score sum), 256 per warp,
//           2048 per CTA, hub chunks of 1024 entries, 32 KB of dynamic shared memory;
//   TB = 1  plain runs on graphs without a vertex of degree above 1024: the same capacities, 32 KB;
//   TB = 2  plain runs on graphs with such vertices: 12-byte slots, 512 per warp, 4096 per CTA (the CTA
//           bin reaches degree 2048), hub chunks of 2048 entries, 48 KB.
// The smaller class leaves more of the SM's unified L1/shared memory to L1, which the label gathers of
// low-degree graphs use; the larger one pre-aggregates more hub entries per global table claim.
template <int TB>
constexpr int kWarpCapT = TB == 2 ? 512 : 256;
template <int TB>
constexpr int kCtaCapT = TB == 2 ? 4096 : 2048;
template <int TB>
constexpr int kHubChunkT = 1024;  // hub row entries per accumulation chunk
template <int TB>
constexpr size_t kDynSmemT = TB == 2 ? 48 * 1024 : 32 * 1024;
constexpr int kWarpCap = kWarpCapT<2>;  // the larger capacities (bounds of the schedule)
constexpr int kCtaCap = kCtaCapT<2>;
constexpr int kHubChunk = 1024;         // (bound of the work items)
// Hub accumulation: a 2048-slot shared table (a 1024-entry chunk fills at most half of it). With the
// larger class (TB = 2) the rest of the 48 KB holds two staging buffers, each the 16-byte-aligned part
// of one chunk's adjacency (4 KB) and edge weights (up to 8 KB), filled by bulk copies (cp.async.bulk
// with an mbarrier) one chunk ahead of the one being aggregated.
constexpr int kHubCap = 2048;
constexpr int kStageOff = kHubCap * 12, kStageAdj = 4096, kStageBuf = 4096 + 8192;
static_assert(kStageOff + 2 * kStageBuf <= (int)kDynSmemT<2>, "staging buffers fit the larger class");
static_assert(kHubCap * 16 <= (int)kDynSmemT<0> && kHubCap * 12 <= (int)kDynSmemT<1>, "hub tables fit every class");
constexpr int kWideDeg = 1024;          // degrees above this need the larger tables
constexpr int kSlotChunk = 8192;                      // hub table slots per choice work item
constexpr int kContestSmall = 4096;
// Hub table slots per batch and the fewest vertices per block come from LpConfig (tile sizes picked by
// gp_autotune): a problem gets at most one block per verts_per_block vertices, since small problems are
// bound by the dependent latency of each phase and more warps (fewer vertices per warp) shorten every
// sub-round.
constexpr int64_t kBigDeg = 2048;    // movers above this degree mark their neighbours with every block
// With kept hub tables (whose updates make each entry dearer) movers above degree 32 are listed in items
// of at most 256 entries, which the warps of all blocks take in turn.
constexpr int64_t kBigDegKept = 32;
constexpr int64_t kBigChunkKept = 256;
constexpr int64_t kBigChunk = 4096;  // entries per marking item of such a mover
constexpr size_t kDynSmem = kDynSmemT<0>;  // the smallest class (bound for the contest workspaces)
static_assert(kWarps * kWarpCapT<2> * 12 <= (int)kDynSmemT<2> && kWarps * kWarpCapT<0> * 16 <= (int)kDynSmemT<0>,
              "warp tables fit the dynamic shared memory");
static_assert(kCtaCapT<2> * 12 <= (int)kDynSmemT<2> && kCtaCapT<0> * 16 <= (int)kDynSmemT<0>,
              "CTA tables fit the dynamic shared memory");
static_assert(kContestSmall * 8 <= (int)kDynSmem, "contest keys must fit the dynamic shared memory");
static_assert(sizeof(DGraph) % 4 == 0, "graph view is copied word by word");

struct __align__(8) SubCounters {
  unsigned int bin_count[8];  // (the running counts live in LpProblem::binres; views copy them here)
  unsigned int n_movers;
  unsigned int n_contested;
  unsigned int hub_chunks;
  unsigned int n_big;  // marking items of admitted movers of degree > kBigDeg (done by all blocks)
  unsigned int hub_batches;
  unsigned int n_inval;  // kept hub tables that went stale in the sub-round (listed in hub_inval)
  unsigned long long max_gain, max_q;
};

static_assert(sizeof(SubCounters) % 4 == 0 && sizeof(SubCounters) / 4 <= 256, "counters are read word by word");

struct LpCounters {
  SubCounters sc[3];                  // by sub-round index mod 3 (current, next, previous)
  unsigned long long moves_round[2];  // by round parity
  unsigned long long moves, rounds, movers;
  unsigned long long bin_visits[8], bin_edges[8];
  unsigned long long phase_ns[8];  // classify, choose, hub accumulation, admit, contest, final, hub choice,
                                   // hub prefix (block 0's view)
  unsigned long long contest_small, contest_packed, contest_large;
  unsigned long long contest_large_items, hub_entries, hub_slots;
  unsigned long long hub_built_entries, hub_stale;  // entries of hubs (re)accumulated; kept tables gone stale
  int err;
  int pad;
};

// One LP run. Vertex ids of bins, slots and hashes are local (0..g.n-1); adjacency entries, labels
// and the label/activity arrays use global ids (local + vbase, labels from lbase on), so several graphs
// stored as one disjoint union can run as independent problems of one launch.
struct LpProblem {
  DGraph g;  // g.n local vertices; offsets/vertex weights indexed by local id, adjacency by global entry
  int64_t vbase, lbase;
  int64_t nl, U;
  int64_t hub_batch_slots;     // hub table slots per batch (tile size of the hub path)
  int64_t hub_chunk;           // hub row entries per accumulation work item (kHubChunkT<TB>)
  int hub_chunk_shift;         // log2(hub_chunk)
  int pad_chunk;
  unsigned wait_us;            // limit of every barrier wait (microseconds)
  unsigned pad_wait;
  uint64_t smix;  // mix64(seed)
  int rounds;
  int singletons;  // labels start as singletons (the first sub-round needs no aggregation)
  int has_hubs;
  int hub_dense;  // hub tables indexed by label directly (few labels: refinement with small k)
  int hub_keep;   // hub tables kept across sub-rounds and updated by the moves (else one batch pass each)
  int sub_t;      // the current sub-round 2 r + s (each block's shared copy)
  int hub_n;      // vertices above deg_cta (kept tables: hub indices 0..hub_n-1)
  int hub_keep_pct;  // a kept table goes stale when its key bound would pass this share of its slots
  int64_t hub_table_slots;  // slots allocated for one batch of hub tables (kept: for all hubs)
  int deg_warp, deg_cta;
  int block_begin, block_count;
  int32_t *labels;
  int64_t *lw;
  const int32_t *q;
  uint8_t *act[2];
  int32_t *bin[kBins];
  // lane-group bins 0-3 (d <= 32): beside each vertex its row, (row_begin << 6) | d, so that the
  // choice loads the row and the vertex's own data in one step
  unsigned long long *binx[4];
  int64_t bin_base[kBins];  // proposal slot of bin position i is bin_base[b] + i
  int32_t *mv_v, *mv_t;
  int32_t *mv_from;  // label an admitted mover left (its weight is moved in the next sub-round)
  int64_t *mv_gain, *mv_q;
  uint8_t *mv_adm;
  int32_t *mv_of_v;  // vertex -> its proposal index in the current sub-round
  int64_t *demand;
  uint32_t *ct, *ct2;
  unsigned long long *ck, *ck2;  // packed contest keys (large contests)
  unsigned long long *big;       // marking items of the sub-round's admitted movers of degree > kBigDeg:
                                 // (vertex << 32) | item, one item per kBigChunk entries of its row
  // hubs (bin 6), per position i of the sub-round's hub list: own-label connection, prefixes of
  // chunks, table slots and choice items, table base inside its batch; first position of each batch
  long long *hub_c0;
  unsigned int *hub_prefix;
  long long *hub_capx;
  unsigned int *hub_scx;
  long long *hub_tb;
  unsigned int *hub_bstart;
  long long *hub_bbase;
  // one batch's tables (reused by every batch; cleared by the choice scan) and partial choices
  int32_t *hub_keys;
  unsigned long long *hub_vals;
  unsigned long long *hub_qv;  // score sums (runs with scores; 64-bit: a hub row can hold 2^17+ scores)
  unsigned char *hub_part;
  unsigned int *hist;        // block_count * 256
  unsigned long long *hoff;  // block_count * 256 + 256
  unsigned int *bar;         // barrier_words(block_count)
  // bin reservation counters by sub-round index mod 3: bin b of set k at binres[k * 256 + b * 32], one
  // 128-byte line per counter so that the blocks' reservations on different bins do not queue on one
  // line
  unsigned int *binres;
  // kept hub tables (hub_keep): per vertex (global id) its hub index or -1; per hub index its table
  // base and slots, an upper bound of the keys in its table and whether the table is current; the hubs
  // whose tables went stale in a sub-round (cleared in the next one, rebuilt at their next activation)
  int32_t *hub_id;
  int64_t *hub_pbase, *hub_pcap;
  unsigned long long *hub_keycnt;
  int *hub_valid;
  int *hub_inval;
  LpCounters *ctr;
};

__device__ __forceinline__ int bin_of(int64_t d, int deg_warp, int deg_cta) {
  if (d <= 4) return 0;
  if (d <= 8) return 1;
  if (d <= 16) return 2;
  if (d <= 32) return 3;
  if (d <= deg_warp) return 4;
  if (d <= deg_cta) return 5;
  return 6;
}

__device__ __forceinline__ unsigned warp_append(unsigned int *counter, bool pred) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (!m) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  return base + __popc(m & lanemask_lt());
}

// Warp-aggregated arr[key] += val for the lanes with `on` (all lanes of the warp must call).
__device__ __forceinline__ void warp_add_by_key(int64_t *arr, bool on, int key, long long val) {
  if (!__any_sync(kFull, on)) return;
  const int k = on ? key : -1;
  const unsigned peers = __match_any_sync(kFull, k);
  if (on) {
    long long s = 0;
    for (unsigned m = peers; m; m &= m - 1) s += __shfl_sync(peers, val, __ffs(m) - 1);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
      atomicAdd(reinterpret_cast<unsigned long long *>(&arr[key]), (unsigned long long)s);
  }
}

// ------------------------------------------------------------------------------------ candidates
struct Best {
  long long conn;
  long long qs;
  unsigned long long h;
  int L;  // -1: none
};

__device__ __forceinline__ Best no_best() {
  Best b;
  b.conn = 0;
  b.qs = 0;
  b.h = 0;
  b.L = -1;
  return b;
}

__device__ __forceinline__ bool better(const Best &a, const Best &b) {
  if (a.L < 0) return false;
  if (b.L < 0) return true;
  if (a.conn != b.conn) return a.conn > b.conn;
  if (a.qs != b.qs) return a.qs > b.qs;
  if (a.h != b.h) return a.h > b.h;
  return a.L < b.L;
}

template <bool LQ>
__device__ __forceinline__ Best shfl_best(const Best &b, int o, int width) {
  Best r;
  r.conn = __shfl_xor_sync(kFull, b.conn, o, width);
  r.qs = LQ ? __shfl_xor_sync(kFull, b.qs, o, width) : 0;
  r.h = __shfl_xor_sync(kFull, b.h, o, width);
  r.L = __shfl_xor_sync(kFull, b.L, o, width);
  return r;
}

template <bool LQ, int W>
__device__ __forceinline__ Best group_best(Best b) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    Best x = shfl_best<LQ>(b, o, W);
    if (better(x, b)) b = x;
  }
  return b;
}

// Candidate L of vertex v (connection conn, score sum qs) against the own-label connection c0.
__device__ __forceinline__ Best make_cand(const LpProblem &P, int v, int L, int L0, long long conn, long long qs,
                                          long long c0, long long cv) {
  if (L < 0 || L == L0 || conn <= c0) return no_best();  // the own label wins ties
  if (P.lw[L] + cv > P.U) return no_best();             // not eligible
  Best b;
  b.L = L;
  b.conn = conn;
  b.qs = qs;
  b.h = mix64(mix64(P.smix ^ (uint64_t)(uint32_t)v) ^ (uint64_t)(L - P.lbase));
  return b;
}

// The same with the candidate's label weight lwL = lw[L] already loaded.
__device__ __forceinline__ Best make_cand_lw(const LpProblem &P, int v, int L, int L0, long long conn, long long qs,
                                             long long c0, long long cv, long long lwL) {
  if (L < 0 || L == L0 || conn <= c0) return no_best();  // the own label wins ties
  if (lwL + cv > P.U) return no_best();                 // not eligible
  Best b;
  b.L = L;
  b.conn = conn;
  b.qs = qs;
  b.h = mix64(mix64(P.smix ^ (uint64_t)(uint32_t)v) ^ (uint64_t)(L - P.lbase));
  return b;
}

// Records the proposal of the active vertex in slot idx (target -1: no proposal). Score sums are
// stored only when scores are given (LQ).
template <bool LQ>
__device__ __forceinline__ void write_slot(const LpProblem &P, int64_t idx, int v, const Best &b, long long c0) {
  P.mv_t[idx] = b.L;
  if (b.L >= 0) {
    P.mv_v[idx] = v;
    P.mv_gain[idx] = b.conn - c0;
    if (LQ) P.mv_q[idx] = b.qs;
    P.mv_adm[idx] = 0;
    P.mv_of_v[v] = (int32_t)idx;
  }
}

__device__ __forceinline__ unsigned slot_hash(int L) { return mix32((unsigned)L); }

// Hub tables: round_up(2 x, 64) slots for x = min(d, number of labels) (a hub row has at most that many
// distinct labels, so the load stays at or below 1/2), indexed by a multiply-shift range reduction of
// the mixed label.
__host__ __device__ __forceinline__ int64_t hub_cap(int64_t d) { return ((2 * d + 63) / 64) * 64; }
__device__ __forceinline__ uint64_t hub_slot(int L, uint64_t cap) {
  return ((uint64_t)slot_hash(L) * cap) >> 32;
}

struct Smem {
  Best best[kWarps];
  long long sum[kWarps];
  long long tmp[32];
  long long tot;
  unsigned long long vis[8], edg[8];
  unsigned wflag[kWarps];
  unsigned long long moves;   // admitted moves of the block in the current admission phase
  unsigned long long movers;  // proposals of the block over the whole call (statistics)
  long long carry;
  int carry_t;
};

template <bool LQ>
__device__ __forceinline__ Best block_best_of(Best b, Smem &sm) {
  b = group_best<LQ, 32>(b);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sm.best[wid] = b;
  __syncthreads();
  Best r = sm.best[0];
  for (int w = 1; w < kWarps; w++)
    if (better(sm.best[w], r)) r = sm.best[w];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned warp_sum_u32(unsigned x) {
  return __reduce_add_sync(kFull, x);
}

__device__ __forceinline__ long long block_sum_of(long long x, Smem &sm) {
  x = warp_sum64(x);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sm.sum[wid] = x;
  __syncthreads();
  long long r = 0;
  for (int w = 0; w < kWarps; w++) r += sm.sum[w];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------------------------ kept hub tables
// With hub_keep, each hub's table persists over the LP call: it is accumulated from the hub's row when
// the hub is first active (or after it went stale), and every admitted move of a neighbour u from
// label A to label B then moves w(u, hub) from A's slot to B's. The table stays equal to the hub's
// connection per label at the start of every sub-round, so the choice reads the same sums as a fresh
// accumulation would (integer sums: the order of the updates does not matter). A table's key count
// starts at min(d, labels) after an accumulation (an upper bound of its distinct labels) and grows by
// one per claimed slot; a table that would pass hub_keep_pct % of its slots (default 75) goes stale: it
// takes no more updates, is cleared in the next sub-round and accumulated again at the hub's next
// activation.
__device__ __forceinline__ bool hub_deltas_on(const LpProblem &P) { return P.hub_keep && P.sub_t + 1 < 2 * P.rounds; }

__device__ void hub_stale(const LpProblem &P, SubCounters &C, int h) {
  if (atomicExch(&P.hub_valid[h], 0) == 1) {
    const unsigned pos = atomicAdd(&C.n_inval, 1u);
    if (pos < (unsigned)P.hub_n) P.hub_inval[pos] = h;  // (each hub goes stale at most once per sub-round)
    atomicAdd(&P.ctr->hub_stale, 1ull);
  }
}

// w (and, with scores, the entry's score q: scores are symmetric, q(u, h) = q(h, u)) moves from label A
// to label B in hub h's table (h's neighbour moved). The hub's words and the first probes of both labels
// are loaded together.
__device__ __noinline__ void hub_delta(const LpProblem &P, SubCounters &C, int h, int A, int B, long long w,
                                       long long q) {
  const int valid = *(volatile int *)&P.hub_valid[h];
  const int64_t tb = P.hub_pbase[h];
  const uint64_t cap = (uint64_t)P.hub_pcap[h];
  if (!valid) return;
  if (P.hub_dense) {
    atomicAdd(&P.hub_vals[tb + (A - P.lbase)], (unsigned long long)(-w));
    atomicAdd(&P.hub_vals[tb + (B - P.lbase)], (unsigned long long)w);
    return;
  }
  uint64_t sa = hub_slot(A, cap), sb = hub_slot(B, cap);
  int ka = *(volatile int *)&P.hub_keys[tb + sa];
  int kb = *(volatile int *)&P.hub_keys[tb + sb];
  // A has a slot (the neighbour's weight is in it); slots are only ever claimed, never freed, so the
  // probe sequence up to A's slot is occupied
  for (uint64_t pr = 0;; pr++) {
    if (ka == A) {
      atomicAdd(&P.hub_vals[tb + sa], (unsigned long long)(-w));
      if (P.hub_qv) atomicAdd(&P.hub_qv[tb + sa], (unsigned long long)(-q));
      break;
    }
    if (ka == -1 || pr >= cap) {  // (not reachable for a current table)
      hub_stale(P, C, h);
      return;
    }
    sa = sa + 1 == cap ? 0 : sa + 1;
    ka = *(volatile int *)&P.hub_keys[tb + sa];
  }
  for (uint64_t pr = 0;; pr++) {
    if (kb == -1) {
      if (atomicAdd(&P.hub_keycnt[h], 1ull) >= (cap * (uint64_t)P.hub_keep_pct) / 100) {
        hub_stale(P, C, h);
        return;
      }
      kb = atomicCAS(&P.hub_keys[tb + sb], -1, B);
      if (kb == -1) kb = B;
    }
    if (kb == B) {
      atomicAdd(&P.hub_vals[tb + sb], (unsigned long long)w);
      if (P.hub_qv) atomicAdd(&P.hub_qv[tb + sb], (unsigned long long)q);
      return;
    }
    if (pr >= cap) {
      hub_stale(P, C, h);
      return;
    }
    sb = sb + 1 == cap ? 0 : sb + 1;
    kb = *(volatile int *)&P.hub_keys[tb + sb];
  }
}

// The neighbour walk of a warp's admitted movers (rows concatenated, two entries per lane per step, loads
// first) with kept hub tables: every neighbour is marked (act_next non-NULL) and every hub neighbour's
// table follows the move (lane j's mover leaves label A for label B). Movers of degree above
// kBigDegKept are left to mark_big, so a warp walks at most 32 kBigDegKept entries.
__device__ __forceinline__ void walk_movers_kept(const LpProblem &P, SubCounters &C, uint8_t *act_next, int64_t rb,
                                                 int64_t excl, int64_t total, int A, int B) {
  const int lane = threadIdx.x & 31;
  for (int64_t t0 = 0; t0 < total; t0 += 64) {
    int a[2], Ax[2], Bx[2], h[2];
    int64_t e[2];
#pragma unroll
    for (int x = 0; x < 2; x++) {
      const int64_t t = t0 + 32 * x + lane;
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t ex = __shfl_sync(kFull, excl, j + step);
        if (j + step < 32 && ex <= t) j += step;
      }
      const int64_t rbj = __shfl_sync(kFull, rb, j), exj = __shfl_sync(kFull, excl, j);
      Ax[x] = __shfl_sync(kFull, A, j);
      Bx[x] = __shfl_sync(kFull, B, j);
      e[x] = rbj + (t - exj);
      a[x] = t < total ? __ldg(P.g.adj + e[x]) : -1;
    }
#pragma unroll
    for (int x = 0; x < 2; x++) h[x] = a[x] >= 0 ? P.hub_id[a[x]] : -1;
#pragma unroll
    for (int x = 0; x < 2; x++) {
      if (a[x] >= 0 && act_next) act_next[a[x]] = 1;
      if (h[x] >= 0) hub_delta(P, C, h[x], Ax[x], Bx[x], P.g.eweight(e[x]), P.q ? (long long)P.q[e[x]] : 0);
    }
  }
}

// Stale kept tables of the previous sub-round are cleared (a block per hub) before any is rebuilt.
__device__ void hub_clear_stale(const LpProblem &P, unsigned ninv, int lb, int nb) {
  ninv = min(ninv, (unsigned)P.hub_n);
  for (unsigned j = lb; j < ninv; j += nb) {
    const int h = P.hub_inval[j];
    const int64_t tb = P.hub_pbase[h], cap = P.hub_pcap[h];
    for (int64_t x = threadIdx.x; x < cap; x += kThreads) {
      P.hub_keys[tb + x] = -1;
      P.hub_vals[tb + x] = 0;
      if (P.hub_qv) P.hub_qv[tb + x] = 0;
    }
  }
}

// Connection of label L in a hub's table (0 when absent).
__device__ long long hub_lookup(const LpProblem &P, int64_t tb, uint64_t cap, int L) {
  if (P.hub_dense) return (long long)P.hub_vals[tb + (L - P.lbase)];
  uint64_t sl = hub_slot(L, cap);
  for (uint64_t pr = 0; pr < cap; pr++) {
    const int k = P.hub_keys[tb + sl];
    if (k == L) return (long long)P.hub_vals[tb + sl];
    if (k == -1) return 0;
    sl = sl + 1 == cap ? 0 : sl + 1;
  }
  return 0;
}

// ------------------------------------------------------------------------------------ moves
// Applies the admitted movers of a warp (all lanes call; `adm` marks the lanes whose proposal idx of
// vertex v to target T was admitted): new label, the left label recorded for the weight update of the
// next sub-round, neighbours marked active for the next round. Movers of degree above kBigDeg are
// listed in P.big instead (counter C.n_big); every block marks their neighbours after the phase.
// act_next NULL (the last round: no round reads the marks) skips the marking. Returns the warp's
// admitted count.
// This form takes the mover's current label L0 and its row (rb, deg) already loaded.
__device__ __forceinline__ unsigned apply_movers_pre(const LpProblem &P, SubCounters &C, uint8_t *act_next, bool adm,
                                                     int64_t idx, int v, int T, int L0, int64_t rb, int64_t deg) {
  const int lane = threadIdx.x & 31;
  if (adm) {
    P.labels[P.vbase + v] = T;
    P.mv_from[idx] = L0;
  } else {
    rb = 0;
    deg = 0;
  }
  const unsigned am = __ballot_sync(kFull, adm);
  if (!am) return 0;
  const bool dl = hub_deltas_on(P);
  if (!act_next && !dl) return (unsigned)__popc(am);
  const bool big = adm && deg > (dl ? kBigDegKept : kBigDeg);
  if (__any_sync(kFull, big)) {
    // one marking item per kBigChunk (kept tables: kBigChunkKept) entries; the warp reserves all of its
    // items with one atomic
    const int64_t chunk = dl ? kBigChunkKept : kBigChunk;
    const unsigned nit = big ? (unsigned)((deg + chunk - 1) / chunk) : 0u;
    unsigned ex = nit;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, ex, o);
      if (lane >= o) ex += y;
    }
    const unsigned tot = __shfl_sync(kFull, ex, 31);
    ex -= nit;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&C.n_big, tot);
    base = __shfl_sync(kFull, base, 0);
    for (unsigned x = 0; x < nit; x++) P.big[base + ex + x] = ((unsigned long long)(unsigned)v << 32) | x;
    if (big) deg = 0;
  }
  // mark the neighbours of the other admitted movers: the warp walks the concatenation of their rows
  int64_t incl = deg;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const int64_t excl = incl - deg;
  const int64_t total = __shfl_sync(kFull, incl, 31);
  if (dl) {
    walk_movers_kept(P, C, act_next, rb, excl, total, L0, T);
    return (unsigned)__popc(am);
  }
  // four entries per lane per step: all adjacency loads are issued before any mark is stored
  constexpr int kMarkUnroll = 4;
  for (int64_t t0 = 0; t0 < total; t0 += 32 * kMarkUnroll) {
    int32_t a[kMarkUnroll];
#pragma unroll
    for (int x = 0; x < kMarkUnroll; x++) {
      const int64_t t = t0 + x * 32 + lane;
      // owner: the largest lane j with excl_j <= t
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t ex = __shfl_sync(kFull, excl, j + step);
        if (j + step < 32 && ex <= t) j += step;
      }
      const int64_t rbj = __shfl_sync(kFull, rb, j), exj = __shfl_sync(kFull, excl, j);
      a[x] = t < total ? __ldg(P.g.adj + rbj + (t - exj)) : -1;
    }
#pragma unroll
    for (int x = 0; x < kMarkUnroll; x++)
      if (a[x] >= 0) act_next[a[x]] = 1;
  }
  return (unsigned)__popc(am);
}

__device__ __forceinline__ unsigned apply_movers(const LpProblem &P, SubCounters &C, uint8_t *act_next, bool adm,
                                                 int64_t idx, int v, int T) {
  int L0 = 0;
  int64_t rb = 0, deg = 0;
  if (adm) {
    L0 = P.labels[P.vbase + v];
    rb = P.g.row_begin(v);
    deg = P.g.row_begin(v + 1) - rb;
  }
  return apply_movers_pre(P, C, act_next, adm, idx, v, T, L0, rb, deg);
}

// Neighbours of the high-degree movers: every block takes marking items (kBigChunk entries of one
// mover's row) in turn. With kept hub tables the items hold kBigChunkKept entries and every warp takes
// items in turn (four entries per lane in flight); the hub neighbours' tables follow the move.
__device__ void mark_big(const LpProblem &P, SubCounters &C, unsigned nitems, int r, int lb, int nb) {
  uint8_t *act_next = r + 1 < P.rounds ? P.act[(r + 1) & 1] : nullptr;  // (no marks in the last round)
  if (!hub_deltas_on(P)) {
    for (unsigned i = lb; i < nitems; i += nb) {
      const unsigned long long it = P.big[i];
      const int v = (int)(it >> 32);
      const int64_t rb = P.g.row_begin(v), re = P.g.row_begin(v + 1);
      const int64_t beg = rb + (int64_t)(unsigned)(it & 0xffffffffu) * kBigChunk, end = min(re, beg + kBigChunk);
      for (int64_t e = beg + threadIdx.x; e < end; e += kThreads) act_next[__ldg(P.g.adj + e)] = 1;
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const unsigned nw = (unsigned)nb * kWarps;
  for (unsigned i = (unsigned)lb * kWarps + (threadIdx.x >> 5); i < nitems; i += nw) {
    const unsigned long long it = P.big[i];
    const int v = (int)(it >> 32);
    const int64_t rb = P.g.row_begin(v), re = P.g.row_begin(v + 1);
    const int64_t beg = rb + (int64_t)(unsigned)(it & 0xffffffffu) * kBigChunkKept, end = min(re, beg + kBigChunkKept);
    const int B = P.labels[P.vbase + v];
    const int A = P.mv_from[P.mv_of_v[v]];
    for (int64_t e0 = beg; e0 < end; e0 += 128) {
      int a[4], h[4];
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int64_t e = e0 + 32 * x + lane;
        a[x] = e < end ? __ldg(P.g.adj + e) : -1;
      }
#pragma unroll
      for (int x = 0; x < 4; x++) h[x] = a[x] >= 0 ? P.hub_id[a[x]] : -1;
#pragma unroll
      for (int x = 0; x < 4; x++) {
        if (a[x] >= 0 && act_next) act_next[a[x]] = 1;
        if (h[x] >= 0) {
          const int64_t e = e0 + 32 * x + lane;
          hub_delta(P, C, h[x], A, B, P.g.eweight(e), P.q ? (long long)P.q[e] : 0);
        }
      }
    }
  }
}

// Weight side of the moves of a finished sub-round (Vp: the block's copy of its counters): every
// proposed target's demand is cleared, and each admitted mover's weight moves from the label it left
// to its target.
__device__ void settle_moves(const LpProblem &P, const SubCounters &Vp, int lb, int nb) {
  unsigned start[kBins + 1];
  start[0] = 0;
#pragma unroll
  for (int b = 0; b < kBins; b++) start[b + 1] = start[b] + Vp.bin_count[b];
  const unsigned na = start[kBins];
  for (unsigned base = (unsigned)lb * kThreads; base < na; base += (unsigned)nb * kThreads) {
    const unsigned k = base + threadIdx.x;
    int64_t i = 0;
    if (k < na) {
      int b = 0;
#pragma unroll
      for (int x = 1; x < kBins; x++)
        if (k >= start[x]) b = x;
      i = P.bin_base[b] + (k - start[b]);
    }
    // the slot's fields are loaded together (those of a slot without a proposal are not used)
    int T = -1, vv = 0, L0 = -1;
    uint8_t a = 0;
    if (k < na) {
      T = P.mv_t[i];
      a = P.mv_adm[i];
      vv = P.mv_v[i];
      L0 = P.mv_from[i];
    }
    const bool adm = T >= 0 && a;
    if (T >= 0) P.demand[T] = 0;
    const long long c = adm ? P.g.vweight(vv) : 0;
    if (!adm) L0 = -1;
    warp_add_by_key(P.lw, adm, T, c);
    warp_add_by_key(P.lw, adm, L0, -c);
  }
}

// ------------------------------------------------------------------------------------ phases
// Classify the active vertices of sub-round (r, s) into degree bins. Each block takes a contiguous
// chunk of vertices, counts them per bin, reserves space with one atomic per bin and then fills it.
// Visits and scanned entries per bin (statistics) add up in the block's shared memory over the whole
// call and reach the counters once, at its end.
__device__ __forceinline__ int active_bin(const LpProblem &P, int64_t v, const uint8_t *act, int r, int s,
                                          uint64_t rmix, int64_t *deg) {
  if (!((r == 0 || act[P.vbase + v]) && (int)(mix64(rmix ^ (uint64_t)v) >> 63) == s)) return -1;
  const int64_t d = P.g.row_begin(v + 1) - P.g.row_begin(v);
  *deg = d;
  return d == 0 ? kBinZero : bin_of(d, P.deg_warp, P.deg_cta);
}

__device__ void phase_classify(const LpProblem &P, SubCounters &C, const SubCounters *Vp, int r, int s, uint64_t rmix,
                               int lb, int nb, Smem &sm) {
  __shared__ unsigned s_cnt[8], s_base[8];
  const unsigned bres = (unsigned)((2 * r + s) % 3) * 256;
  if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0;
  const uint8_t *act = P.act[r & 1];
  uint8_t *act_next = P.act[(r + 1) & 1];
  const int64_t n = P.g.n;
  const int64_t chunk = (n + nb - 1) / nb;
  const int64_t lo = min(n, (int64_t)lb * chunk), hi = min(n, lo + chunk);
  const int lane = threadIdx.x & 31;
  constexpr int kCls = 8;
  if (hi - lo <= (int64_t)kCls * kThreads) {
    // chunks of up to kCls vertices per thread: all flag loads first, then the offsets of the active
    // ones, then the per-bin aggregation; the bins stay in a register (4 bits per vertex) for pass 2
    const int niter = (int)((hi - lo + kThreads - 1) / kThreads);
    unsigned flag = 0;
#pragma unroll
    for (int it = 0; it < kCls; it++) {
      const int64_t v = lo + (int64_t)it * kThreads + threadIdx.x;
      if (it < niter && v < hi && (r == 0 || act[P.vbase + v])) flag |= 1u << it;
    }
    if (s == 0) {
#pragma unroll
      for (int it = 0; it < kCls; it++) {
        const int64_t v = lo + (int64_t)it * kThreads + threadIdx.x;
        if (it < niter && v < hi) act_next[P.vbase + v] = 0;  // the marks of round r go there
      }
    }
    int dd[kCls];
#pragma unroll
    for (int it = 0; it < kCls; it++) {
      const int64_t v = lo + (int64_t)it * kThreads + threadIdx.x;
      dd[it] = 0;
      if ((flag >> it & 1) && (int)(mix64(rmix ^ (uint64_t)v) >> 63) == s) {
        dd[it] = (int)(P.g.row_begin(v + 1) - P.g.row_begin(v));
      } else {
        flag &= ~(1u << it);
      }
    }
    // the previous sub-round's moves settle while the loads above are in flight
    if (Vp) settle_moves(P, *Vp, lb, nb);
    __syncthreads();
    unsigned codes = 0xffffffffu;
#pragma unroll
    for (int it = 0; it < kCls; it++) {
      if (it >= niter) break;
      int b = -1;
      if (flag >> it & 1) b = dd[it] == 0 ? kBinZero : bin_of(dd[it], P.deg_warp, P.deg_cta);
      if (b >= 0) codes = (codes & ~(15u << (4 * it))) | ((unsigned)b << (4 * it));
      const unsigned peers = __match_any_sync(kFull, b);
      // entries of the lanes in the same bin summed in the warp (at most 2^31 in all): one shared
      // atomic per bin and warp
      const unsigned esum = __reduce_add_sync(peers, (unsigned)dd[it]);
      if (b >= 0 && lane == __ffs(peers) - 1) {
        atomicAdd(&sm.vis[b], (unsigned long long)__popc(peers));
        if (b < kBins) atomicAdd(&s_cnt[b], (unsigned)__popc(peers));
        if (esum) atomicAdd(&sm.edg[b], (unsigned long long)esum);
      }
    }
    __syncthreads();
    if (threadIdx.x < kBins) {
      s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&P.binres[bres + threadIdx.x * 32], s_cnt[threadIdx.x]) : 0;
      s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kCls; it++) {
      if (it >= niter) break;
      const int64_t v = lo + (int64_t)it * kThreads + threadIdx.x;
      const int c = (int)(codes >> (4 * it) & 15u);
      const int b = c == 15 ? -1 : c;
      const bool put = b >= 0 && b < kBins;
      const unsigned peers = __match_any_sync(kFull, put ? b : -1);
      const int leader = __ffs(peers) - 1;
      unsigned pos = 0;
      if (put && lane == leader) pos = atomicAdd(&s_cnt[b], (unsigned)__popc(peers));
      pos = __shfl_sync(kFull, pos, leader);
      if (put) {
        const unsigned at = s_base[b] + pos + __popc(peers & lanemask_lt());
        P.bin[b][at] = (int32_t)v;
        // (the row begin was loaded above; this load hits L1)
        if (b < 4) P.binx[b][at] = ((unsigned long long)P.g.row_begin(v) << 6) | (unsigned long long)dd[it];
      }
    }
    return;
  }
  if (Vp) settle_moves(P, *Vp, lb, nb);
  __syncthreads();
  // pass 1: counts
  for (int64_t v0 = lo; v0 < hi; v0 += kThreads) {
    const int64_t v = v0 + threadIdx.x;
    int b = -1;
    int64_t d = 0;
    if (v < hi) {
      if (s == 0) act_next[P.vbase + v] = 0;  // the marks of round r go there
      b = active_bin(P, v, act, r, s, rmix, &d);
    }
    const unsigned peers = __match_any_sync(kFull, b);
    const unsigned esum = __reduce_add_sync(peers, (unsigned)d);
    if (b >= 0 && lane == __ffs(peers) - 1) {
      atomicAdd(&sm.vis[b], (unsigned long long)__popc(peers));
      if (b < kBins) atomicAdd(&s_cnt[b], (unsigned)__popc(peers));
      if (esum) atomicAdd(&sm.edg[b], (unsigned long long)esum);
    }
  }
  __syncthreads();
  if (threadIdx.x < kBins) {
    s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&P.binres[bres + threadIdx.x * 32], s_cnt[threadIdx.x]) : 0;
    s_cnt[threadIdx.x] = 0;
  }
  __syncthreads();
  // pass 2: fill the reserved ranges
  for (int64_t v0 = lo; v0 < hi; v0 += kThreads) {
    const int64_t v = v0 + threadIdx.x;
    int b = -1;
    int64_t d = 0;
    if (v < hi) b = active_bin(P, v, act, r, s, rmix, &d);
    const bool put = b >= 0 && b < kBins;
    const unsigned peers = __match_any_sync(kFull, put ? b : -1);
    const int leader = __ffs(peers) - 1;
    unsigned pos = 0;
    if (put && lane == leader) pos = atomicAdd(&s_cnt[b], (unsigned)__popc(peers));
    pos = __shfl_sync(kFull, pos, leader);
    if (put) {
      const unsigned at = s_base[b] + pos + __popc(peers & lanemask_lt());
      P.bin[b][at] = (int32_t)v;
      if (b < 4) P.binx[b][at] = ((unsigned long long)P.g.row_begin(v) << 6) | (unsigned long long)d;
    }
  }
}

// Groups of G lanes (G = 4, 8, 16 or 32 for bins 0-3), one vertex per group, d <= G. The four bins
// share one work loop: warp-iteration j of the concatenated bins takes U * 32/G consecutive vertices
// of one bin, so small bins overlap instead of running one after another. G is a runtime value (one
// copy of the code serves every width). Equal neighbour labels within a group are found with
// __match_any_sync and their weights summed over the matching lanes; each group issues the loads of
// its U vertices before using any (memory-level parallelism).
template <bool LQ>
__device__ __forceinline__ Best group_best_rt(Best b, int W) {
  for (int o = W / 2; o > 0; o >>= 1) {
    Best x = shfl_best<LQ>(b, o, W);
    if (better(x, b)) b = x;
  }
  return b;
}

// Unit edge weights without scores: connections are counts (at most 32 in a lane group), so a
// candidate's rank (conn, then h) is the single 64-bit key conn << 58 | h >> 6, where h = H(seed, v, L)
// = mix64(hv ^ (L - lbase)) with hv = mix64(smix ^ v). Equal keys (equal counts and equal top 58 bits
// of h) fall back to the full order (h desc, then L asc) with h recomputed for both labels. Key 0
// means no candidate (a candidate has conn >= 1). Returns the group's winning label (-1: none) and
// its key in *Kout.
__device__ __forceinline__ int group_best_unit(unsigned long long K, int L, int W, uint64_t hv, int64_t lbase,
                                               unsigned long long *Kout) {
  for (int o = W / 2; o > 0; o >>= 1) {
    const unsigned long long K2 = __shfl_xor_sync(kFull, K, o, W);
    const int L2 = __shfl_xor_sync(kFull, L, o, W);
    bool take = K2 > K;
    if (K2 == K && K2 != 0 && L2 != L) {
      const uint64_t h2 = mix64(hv ^ (uint64_t)(L2 - lbase)), h1 = mix64(hv ^ (uint64_t)(L - lbase));
      take = h2 > h1 || (h2 == h1 && L2 < L);
    }
    if (take) {
      K = K2;
      L = L2;
    }
  }
  *Kout = K;
  return L;
}

template <int EW, bool LQ>
__device__ void choose_groups(const LpProblem &P, const SubCounters &V, int lb, int nb) {
  constexpr int U = 2;
  unsigned pre[5];
  pre[0] = 0;
#pragma unroll
  for (int b = 0; b < 4; b++) {
    const unsigned per = (32u >> (2 + b)) * U;
    pre[b + 1] = pre[b] + (V.bin_count[b] + per - 1) / per;
  }
  const unsigned total = pre[4];
  if (total == 0) return;
  const int lane = threadIdx.x & 31;
  const unsigned gw = (unsigned)lb * kWarps + (threadIdx.x >> 5), nw = (unsigned)nb * kWarps;
  for (unsigned j = gw; j < total; j += nw) {
    const int bin = (j >= pre[1]) + (j >= pre[2]) + (j >= pre[3]);
    const int G = 4 << bin;
    const unsigned gpw = 32u >> (2 + bin);
    const unsigned cnt = V.bin_count[bin];
    const int32_t *list = P.bin[bin];
    const unsigned long long *listx = P.binx[bin];
    const int gl = lane & (G - 1);
    const unsigned sub = (unsigned)lane / (unsigned)G;
    const unsigned base = (j - pre[bin]) * gpw * U;
    int v[U], Lu[U], L0[U], qq[U];
    long long w[U], cv[U];
    int64_t beg[U], d[U];
    bool valid[U];
    // the vertex and its row together, then its label and weight together with the adjacency
#pragma unroll
    for (int u = 0; u < U; u++) {
      const unsigned i = base + u * gpw + sub;
      valid[u] = i < cnt;
      v[u] = 0;
      beg[u] = 0;
      d[u] = 0;
      if (valid[u]) {
        v[u] = list[i];
        const unsigned long long x = listx[i];
        beg[u] = (int64_t)(x >> 6);
        d[u] = (int64_t)(x & 63);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      L0[u] = -2;
      cv[u] = 0;
      if (valid[u]) {
        L0[u] = P.labels[P.vbase + v[u]];
        cv[u] = P.g.vweight(v[u]);
      }
    }
    int nbr[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      nbr[u] = gl < d[u] ? __ldg(P.g.adj + beg[u] + gl) : -1;
      w[u] = 0;
      qq[u] = 0;
      if (gl < d[u]) {
        w[u] = load_ew<EW>(P.g.ew, beg[u] + gl);
        if (LQ) qq[u] = __ldg(P.q + beg[u] + gl);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) Lu[u] = nbr[u] >= 0 ? P.labels[nbr[u]] : -1;
    // connections of every vertex first, then the label weights of all their candidates in one
    // round of loads, then the choices and the stores
    long long c0[U], conn[U], qs[U], lwL[U];
    bool cand[U];
    const unsigned gmask = G == 32 ? kFull : ((1u << G) - 1u) << (sub * (unsigned)G);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const bool has = gl < d[u];
      const unsigned peers = __match_any_sync(kFull, (unsigned)Lu[u]) & gmask;
      if constexpr (EW == 0) {
        conn[u] = __popc(peers);
      } else {
        if (!__any_sync(kFull, w[u] >= (1ll << 26))) {
          conn[u] = (long long)__reduce_add_sync(peers, (unsigned)w[u]);
        } else {
          conn[u] = 0;
          for (unsigned m = peers; m; m &= m - 1) conn[u] += __shfl_sync(peers, w[u], __ffs(m) - 1);
        }
      }
      qs[u] = 0;
      if constexpr (LQ) qs[u] = (long long)__reduce_add_sync(peers, (unsigned)qq[u]);
      // the own-label connection is the connection of the group's lanes that carry the own label
      const unsigned own = __ballot_sync(kFull, has && Lu[u] == L0[u]) & gmask;
      if constexpr (EW == 0) {
        c0[u] = __popc(own);
      } else {
        const long long cown = __shfl_sync(kFull, conn[u], own ? __ffs(own) - 1 : lane);
        c0[u] = own ? cown : 0;
      }
      cand[u] = has && lane == __ffs(peers) - 1 && Lu[u] != L0[u] && conn[u] > c0[u];
      lwL[u] = cand[u] ? P.lw[Lu[u]] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      Best b = no_best();
      if (!__any_sync(kFull, cand[u])) {
        // no lane of the warp has a candidate (every vertex keeps its label, the common case once
        // clusters or blocks settle): only the empty proposals are recorded
        if (valid[u] && gl == 0) P.mv_t[P.bin_base[bin] + base + u * gpw + sub] = -1;
        continue;
      }
      if constexpr (EW == 0 && !LQ) {
        // first the 32-bit key conn << 26 | h >> 38 (maximum over the group with one shuffle per
        // level); a unique maximum is the exact winner. Equal keys in some group (equal counts and
        // equal top 26 bits of h) send the whole warp through the exact 64-bit comparison.
        const uint64_t hv = mix64(P.smix ^ (uint64_t)(uint32_t)v[u]);
        const bool elig = cand[u] && lwL[u] + cv[u] <= P.U;
        const uint64_t h = elig ? mix64(hv ^ (uint64_t)(Lu[u] - P.lbase)) : 0;
        const unsigned K = elig ? ((unsigned)conn[u] << 26) | (unsigned)(h >> 38) : 0u;
        unsigned Km = K;
        for (int o = G / 2; o > 0; o >>= 1) Km = max(Km, __shfl_xor_sync(kFull, Km, o, G));
        const unsigned top = __ballot_sync(kFull, Km != 0 && K == Km) & gmask;
        if (__any_sync(kFull, __popc(top) > 1)) {
          unsigned long long K64 = elig ? ((unsigned long long)conn[u] << 58) | (h >> 6) : 0ull;
          b.L = group_best_unit(K64, elig ? Lu[u] : -1, G, hv, P.lbase, &K64);
          b.conn = (long long)(K64 >> 58);
        } else {
          const int Lw = __shfl_sync(kFull, Lu[u], top ? __ffs(top) - 1 : lane);
          b.L = top ? Lw : -1;
          b.conn = (long long)(Km >> 26);
        }
      } else {
        if (cand[u]) b = make_cand_lw(P, v[u], Lu[u], L0[u], conn[u], qs[u], c0[u], cv[u], lwL[u]);
        b = group_best_rt<LQ>(b, G);
      }
      const bool mover = valid[u] && gl == 0 && b.L >= 0;
      if (valid[u] && gl == 0) write_slot<LQ>(P, P.bin_base[bin] + base + u * gpw + sub, v[u], b, c0[u]);
      // (at most one mover per group: equal targets within a warp are rare, so no aggregation)
      if (mover) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)cv[u]);
    }
  }
}

// Warp-cooperative insert of (label L, weight w, score q) into an open-addressing table in shared
// memory (slots keys/vals/qv, `mask` = slots - 1). Lanes are grouped by label first, so each distinct
// label of the warp costs one insert however many neighbours carry it. All lanes call; lanes with
// `on` false contribute nothing.
// A table that is full (an invariant of the sizing broken) ends the probe after one pass over the table,
// records GP_ERR_INTERNAL with the site in the problem's counters, and drops the label.
__device__ __forceinline__ void table_full(LpCounters *ctr, int site) {
  atomicExch(&ctr->err, GP_ERR_INTERNAL);
  atomicExch(&ctr->pad, site);
}

template <int EW, bool LQ>
__device__ __forceinline__ void warp_insert(int *keys, unsigned long long *vals, unsigned *qv, unsigned mask, bool on,
                                            int L, long long w, unsigned q, LpCounters *ctr, int site) {
  const unsigned peers = __match_any_sync(kFull, on ? L : -1);
  // weights below 2^26 sum exactly in 32 bits over at most 32 lanes: one warp reduction
  const bool wide = EW != 0 && __any_sync(kFull, on && (w >= (1ll << 26) || w < 0));
  if (!on) return;
  long long sum;
  if constexpr (EW == 0) {
    sum = __popc(peers);
  } else if (!wide) {
    sum = (long long)__reduce_add_sync(peers, (unsigned)w);
  } else {
    sum = 0;
    for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, w, __ffs(m) - 1);
  }
  unsigned qs = 0;
  if constexpr (LQ) qs = __reduce_add_sync(peers, q);
  if ((int)(threadIdx.x & 31) != __ffs(peers) - 1) return;
  unsigned sl = slot_hash(L) & mask;
  for (unsigned probe = 0; probe <= mask; probe++) {
    const int k = atomicCAS(&keys[sl], -1, L);
    if (k == -1 || k == L) {
      atomicAdd(&vals[sl], (unsigned long long)sum);
      if (LQ) atomicAdd(&qv[sl], qs);
      return;
    }
    sl = (sl + 1) & mask;
  }
  table_full(ctr, site);
}

// One warp per vertex (32 < d <= deg_warp), open-addressing table in shared memory.
template <int EW, int TB>
__device__ void choose_warp(const LpProblem &P, const SubCounters &V, int lb, int nb, unsigned char *dsm, bool direct) {
  constexpr bool LQ = TB == 0;
  const unsigned cnt = V.bin_count[4];
  if (cnt == 0) return;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kCap = kWarpCapT<TB>;
  unsigned long long *vals = reinterpret_cast<unsigned long long *>(dsm) + wid * kCap;
  int *keys = reinterpret_cast<int *>(dsm + kWarps * kCap * 8) + wid * kCap;
  unsigned *qv = reinterpret_cast<unsigned *>(dsm + kWarps * kCap * 12) + wid * kCap;
  for (int s = lane; s < kCap; s += 32) {
    keys[s] = -1;
    vals[s] = 0;
    if (LQ) qv[s] = 0;
  }
  __syncwarp();
  const int32_t *list = P.bin[4];
  const unsigned gw = (unsigned)lb * kWarps + wid, nw = (unsigned)nb * kWarps;
  if (direct) {
    // distinct singleton labels: the connection to a label is the weight of its one entry
    for (unsigned i = gw; i < cnt; i += nw) {
      const int v = list[i];
      const int64_t beg = P.g.row_begin(v), end = P.g.row_begin(v + 1);
      const int L0 = P.labels[P.vbase + v];
      const long long cv = P.g.vweight(v);
      Best b = no_best();
      for (int64_t e = beg + lane; e < end; e += 32) {
        const Best x = make_cand(P, v, P.labels[__ldg(P.g.adj + e)], L0, load_ew<EW>(P.g.ew, e),
                                 LQ ? (long long)__ldg(P.q + e) : 0, 0, cv);
        if (better(x, b)) b = x;
      }
      b = group_best<LQ, 32>(b);
      if (lane == 0) {
        write_slot<LQ>(P, P.bin_base[4] + i, v, b, 0);
        if (b.L >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)cv);
      }
    }
    return;
  }
  for (unsigned i = gw; i < cnt; i += nw) {
    const int v = list[i];
    const int64_t beg = P.g.row_begin(v), end = P.g.row_begin(v + 1);
    const int d = (int)(end - beg);
    int cap = 64;
    while (cap < 2 * d) cap <<= 1;
    const unsigned mask = (unsigned)cap - 1;
    const int L0 = P.labels[P.vbase + v];
    long long c0 = 0;
    bool other = false;  // some neighbour carries another label
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool in = e < end;
      const int L = in ? P.labels[__ldg(P.g.adj + e)] : -1;
      const long long w = in ? load_ew<EW>(P.g.ew, e) : 0;
      if (in && L == L0) c0 += w;
      other |= in && L != L0;
      warp_insert<EW, LQ>(keys, vals, qv, mask, in && L != L0, L, w, (LQ && in) ? (unsigned)__ldg(P.q + e) : 0u,
                          P.ctr, 1);
    }
    if (!__any_sync(kFull, other)) {
      // every neighbour carries the own label: no candidate, the table is still empty
      if (lane == 0) P.mv_t[P.bin_base[4] + i] = -1;
      continue;
    }
    c0 = warp_sum64(c0);
    __syncwarp();
    const long long cv = P.g.vweight(v);
    Best b = no_best();
    for (int s = lane; s < cap; s += 32) {
      const int L = keys[s];
      if (L >= 0) {
        const Best x = make_cand(P, v, L, L0, (long long)vals[s], LQ ? (long long)qv[s] : 0, c0, cv);
        if (better(x, b)) b = x;
        keys[s] = -1;
        vals[s] = 0;
        if (LQ) qv[s] = 0;
      }
    }
    __syncwarp();
    b = group_best<LQ, 32>(b);
    if (lane == 0) {
      write_slot<LQ>(P, P.bin_base[4] + i, v, b, c0);
      if (b.L >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)cv);
    }
  }
}

// One CTA per vertex (deg_warp < d <= deg_cta), table in shared memory.
template <int EW, int TB>
__device__ void choose_cta(const LpProblem &P, const SubCounters &V, int lb, int nb, unsigned char *dsm, Smem &sm,
                           bool direct) {
  const unsigned cnt = V.bin_count[5];
  if (cnt == 0) return;
  constexpr bool LQ = TB == 0;
  constexpr int kCap = kCtaCapT<TB>;
  unsigned long long *vals = reinterpret_cast<unsigned long long *>(dsm);
  int *keys = reinterpret_cast<int *>(dsm + kCap * 8);
  unsigned *qv = reinterpret_cast<unsigned *>(dsm + kCap * 12);
  __syncthreads();
  for (int s = threadIdx.x; s < kCap; s += kThreads) {
    keys[s] = -1;
    vals[s] = 0;
    if (LQ) qv[s] = 0;
  }
  __syncthreads();
  const int32_t *list = P.bin[5];
  if (direct) {
    for (unsigned i = lb; i < cnt; i += nb) {
      const int v = list[i];
      const int64_t beg = P.g.row_begin(v), end = P.g.row_begin(v + 1);
      const int L0 = P.labels[P.vbase + v];
      const long long cv = P.g.vweight(v);
      Best b = no_best();
      for (int64_t e = beg + threadIdx.x; e < end; e += kThreads) {
        const Best x = make_cand(P, v, P.labels[__ldg(P.g.adj + e)], L0, load_ew<EW>(P.g.ew, e),
                                 LQ ? (long long)__ldg(P.q + e) : 0, 0, cv);
        if (better(x, b)) b = x;
      }
      b = block_best_of<LQ>(b, sm);
      if (threadIdx.x == 0) {
        write_slot<LQ>(P, P.bin_base[5] + i, v, b, 0);
        if (b.L >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)cv);
      }
    }
    __syncthreads();
    return;
  }
  for (unsigned i = lb; i < cnt; i += nb) {
    const int v = list[i];
    const int64_t beg = P.g.row_begin(v), end = P.g.row_begin(v + 1);
    const int d = (int)(end - beg);
    int cap = 64;
    while (cap < 2 * d) cap <<= 1;
    const unsigned mask = (unsigned)cap - 1;
    const int L0 = P.labels[P.vbase + v];
    long long c0 = 0;
    for (int64_t e0 = beg + (threadIdx.x & ~31); e0 < end; e0 += kThreads) {
      const int64_t e = e0 + (threadIdx.x & 31);
      const bool in = e < end;
      const int L = in ? P.labels[__ldg(P.g.adj + e)] : -1;
      const long long w = in ? load_ew<EW>(P.g.ew, e) : 0;
      if (in && L == L0) c0 += w;
      warp_insert<EW, LQ>(keys, vals, qv, mask, in && L != L0, L, w, (LQ && in) ? (unsigned)__ldg(P.q + e) : 0u,
                          P.ctr, 2);
    }
    c0 = block_sum_of(c0, sm);  // also completes the table
    const long long cv = P.g.vweight(v);
    Best b = no_best();
    for (int s = threadIdx.x; s < cap; s += kThreads) {
      const int L = keys[s];
      if (L >= 0) {
        const Best x = make_cand(P, v, L, L0, (long long)vals[s], LQ ? (long long)qv[s] : 0, c0, cv);
        if (better(x, b)) b = x;
        keys[s] = -1;
        vals[s] = 0;
        if (LQ) qv[s] = 0;
      }
    }
    b = block_best_of<LQ>(b, sm);
    if (threadIdx.x == 0) {
      write_slot<LQ>(P, P.bin_base[5] + i, v, b, c0);
      if (b.L >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)cv);
    }
  }
  __syncthreads();
}

// Hubs (d > deg_cta), done by block 0 for the sub-round's hub list: prefixes of work chunks (P.hub_chunk
// entries), table slots (hub_cap(d) each) and choice items (kSlotChunk slots); cut into batches of
// about P.hub_batch_slots slots (a hub starts a new batch when its slot prefix crosses a multiple of
// that size); table base of each hub inside its batch. With kept tables there is one batch, every hub
// keeps its own table base, and only hubs whose table is not current get accumulation chunks (the
// first sub-round of a clustering from singletons scans every row directly: `direct`).
__device__ void hub_prefix(const LpProblem &P, SubCounters &C, const SubCounters &V, Smem &sm, bool direct) {
  const unsigned cnt = V.bin_count[6];
  __shared__ long long s_cap, s_ch, s_sc, s_nbat, s_prev_bid;
  __shared__ long long t_bid[kThreads];
  if (threadIdx.x == 0) {
    s_cap = s_ch = s_sc = s_nbat = 0;
    s_prev_bid = -1;
  }
  __syncthreads();
  long long sum_d = 0, sum_cap = 0, sum_built = 0;
  for (unsigned base = 0; base < cnt; base += kThreads) {
    const unsigned i = base + threadIdx.x;
    const bool valid = i < cnt;
    long long d = 0, cap = 0, ch = 0, sc = 0, ktb = 0;
    if (valid) {
      const int v = P.bin[6][i];
      d = P.g.row_begin(v + 1) - P.g.row_begin(v);
      // a row has at most min(d, nl) distinct labels (refinement: nl = k blocks); with few labels the
      // table is indexed by the label itself
      cap = P.hub_dense ? P.nl : min(hub_cap(d), hub_cap(P.nl));
      ch = (d + P.hub_chunk - 1) >> P.hub_chunk_shift;
      if (P.hub_keep && !direct) {
        const int h = P.hub_id[P.vbase + v];
        if (h < 0) {  // (every vertex above deg_cta has a hub index)
          table_full(P.ctr, 6);
          ch = 0;
          cap = 0;
        } else {
          ktb = P.hub_pbase[h];
          if (P.hub_valid[h]) {
            ch = 0;  // current: no accumulation
          } else {
            P.hub_valid[h] = 1;
            P.hub_keycnt[h] = (unsigned long long)min(d, (long long)P.nl);
            sum_built += d;
          }
        }
      } else {
        sum_built += d;
      }
      sc = (cap + kSlotChunk - 1) / kSlotChunk;
      P.hub_c0[i] = 0;
      sum_d += d;
      sum_cap += cap;
    }
    const long long capx = s_cap + block_excl_scan64(cap, sm.tmp, &sm.tot);
    const long long cap_t = sm.tot;
    const long long chx = s_ch + block_excl_scan64(ch, sm.tmp, &sm.tot);
    const long long ch_t = sm.tot;
    const long long scx = s_sc + block_excl_scan64(sc, sm.tmp, &sm.tot);
    const long long sc_t = sm.tot;
    const long long bid = P.hub_keep ? 0 : capx / P.hub_batch_slots;
    t_bid[threadIdx.x] = bid;
    __syncthreads();
    const long long prev = threadIdx.x > 0 ? t_bid[threadIdx.x - 1] : s_prev_bid;
    const long long flag = (valid && bid != prev) ? 1 : 0;
    const long long bx = s_nbat + block_excl_scan64(flag, sm.tmp, &sm.tot);
    const long long nb_t = sm.tot;
    if (valid) {
      P.hub_prefix[i] = (unsigned)chx;
      P.hub_capx[i] = capx;
      P.hub_scx[i] = (unsigned)scx;
    }
    if (flag) {
      P.hub_bstart[bx] = i;
      P.hub_bbase[bx] = capx;
    }
    __syncthreads();
    if (valid) {
      P.hub_tb[i] = P.hub_keep ? ktb : capx - P.hub_bbase[bx + flag - 1];
      // (a sizing invariant: a batch's tables fit the allocation; checked, not assumed)
      if (P.hub_tb[i] + cap > P.hub_table_slots) table_full(P.ctr, 5);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_cap += cap_t;
      s_ch += ch_t;
      s_sc += sc_t;
      s_nbat += nb_t;
      s_prev_bid = t_bid[min(kThreads, (int)(cnt - base)) - 1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.hub_prefix[cnt] = (unsigned)s_ch;
    P.hub_capx[cnt] = s_cap;
    P.hub_scx[cnt] = (unsigned)s_sc;
    P.hub_bstart[s_nbat] = cnt;
    C.hub_chunks = (unsigned)s_ch;
    C.hub_batches = (unsigned)s_nbat;
  }
  __syncthreads();
  if (*(volatile int *)&P.ctr->err == GP_ERR_INTERNAL) {
    // tables would not fit: no hub work this sub-round, no hub proposals (the call reports the error)
    if (threadIdx.x == 0) {
      C.hub_chunks = 0;
      C.hub_batches = 0;
    }
    for (unsigned i = threadIdx.x; i < cnt; i += kThreads) P.mv_t[P.bin_base[6] + i] = -1;
    for (unsigned i = threadIdx.x; i <= cnt; i += kThreads) {
      P.hub_prefix[i] = 0;
      P.hub_scx[i] = 0;
    }
  }
  sum_d = block_sum_of(sum_d, sm);
  sum_cap = block_sum_of(sum_cap, sm);
  sum_built = block_sum_of(sum_built, sm);
  if (threadIdx.x == 0) {
    P.ctr->hub_entries += (unsigned long long)sum_d;
    P.ctr->hub_slots += (unsigned long long)sum_cap;
    P.ctr->hub_built_entries += (unsigned long long)sum_built;
  }
}

// largest position i in [lo, hi) with pre[i] <= x
template <class T>
__device__ __forceinline__ unsigned search_prefix(const T *pre, unsigned lo, unsigned hi, unsigned long long x) {
  while (hi - lo > 1) {
    const unsigned mid = (lo + hi) >> 1;
    if ((unsigned long long)pre[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------------------------ bulk-copy staging
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// the issuing thread's arrival, announcing `bytes` of copies that complete the phase
__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for a phase of `bar` (limit_ns of %globaltimer, and at most 2^30 polls).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < (1u << 30); it++) {
    if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// One hub chunk [beg, end) in a staging buffer: its adjacency and edge weights from the first 16-byte
// boundary at or before `beg` up to the last one at or before `end` (a bulk copy starts and ends on
// 16-byte boundaries and never reaches past `end`); the few entries after the last boundary are read
// directly.
template <int EW>
struct HubChunk {
  static constexpr int kEsz = EW == 2 ? 8 : 4;
  const int32_t *sadj;
  const unsigned char *sew;
  int64_t beg, na, ne;  // entries beg .. beg + na - 1 (weights: + ne - 1) are staged
  int aoff, eoff;       // position of entry beg in the buffer (entries)

  __device__ __forceinline__ static void geometry(const LpProblem &P, int64_t beg, int64_t end, uintptr_t *alo,
                                                  unsigned *ab, uintptr_t *elo, unsigned *eb) {
    const uintptr_t a0 = (uintptr_t)(P.g.adj + beg), a1 = (uintptr_t)(P.g.adj + end);
    *alo = a0 & ~(uintptr_t)15;
    *ab = (unsigned)((a1 & ~(uintptr_t)15) - *alo);
    *elo = 0;
    *eb = 0;
    if (EW) {
      const uintptr_t e0 = (uintptr_t)P.g.ew + (uintptr_t)beg * kEsz, e1 = (uintptr_t)P.g.ew + (uintptr_t)end * kEsz;
      *elo = e0 & ~(uintptr_t)15;
      *eb = (unsigned)((e1 & ~(uintptr_t)15) - *elo);
    }
  }
  // thread 0: the copies of chunk [beg, end) into buffer `buf`, completing the barrier's next phase
  __device__ __forceinline__ static void issue(const LpProblem &P, int64_t beg, int64_t end, unsigned char *buf,
                                               unsigned long long *bar) {
    uintptr_t alo, elo;
    unsigned ab, eb;
    geometry(P, beg, end, &alo, &ab, &elo, &eb);
    mbar_expect(bar, ab + eb);
    if (ab) bulk_copy_g2s(buf, (const void *)alo, ab, bar);
    if (eb) bulk_copy_g2s(buf + kStageAdj, (const void *)elo, eb, bar);
  }
  __device__ __forceinline__ void view(const LpProblem &P, int64_t b, int64_t end, const unsigned char *buf) {
    uintptr_t alo, elo;
    unsigned ab, eb;
    geometry(P, b, end, &alo, &ab, &elo, &eb);
    beg = b;
    sadj = reinterpret_cast<const int32_t *>(buf);
    sew = buf + kStageAdj;
    const uintptr_t a0 = (uintptr_t)(P.g.adj + b);
    aoff = (int)((a0 - alo) >> 2);
    na = (int64_t)ab / 4 - aoff;
    if (na < 0) na = 0;
    ne = 0;
    eoff = 0;
    if (EW) {
      const uintptr_t e0 = (uintptr_t)P.g.ew + (uintptr_t)b * kEsz;
      eoff = (int)((e0 - elo) / kEsz);
      ne = (int64_t)eb / kEsz - eoff;
      if (ne < 0) ne = 0;
    }
  }
  __device__ __forceinline__ int adj(const LpProblem &P, int64_t e) const {
    const int64_t x = e - beg;
    return x < na ? sadj[aoff + x] : __ldg(P.g.adj + e);
  }
  __device__ __forceinline__ long long ew(const LpProblem &P, int64_t e) const {
    if (EW == 0) return 1;
    const int64_t x = e - beg;
    if (x >= ne) return load_ew<EW>(P.g.ew, e);
    if (EW == 1) return (long long)reinterpret_cast<const int32_t *>(sew)[eoff + x];
    return reinterpret_cast<const long long *>(sew)[eoff + x];
  }
};

// Accumulation of batch [h0, h1): hub rows are cut into chunks of kHubChunkT<TB> entries. A block aggregates
// its chunk's labels in a shared-memory table first and then adds one entry per distinct label to the
// hub's table, so labels that many neighbours share cost one global atomic per chunk. With the larger
// table class the block's next chunk is copied into a staging buffer (bulk copy, thread 0) while it
// aggregates the current one. A staging wait that runs out records GP_ERR_TIMEOUT; the block then stops
// (uniformly, after the chunk's block-wide sum), waits once more for its copies in flight and returns.
template <int EW, int TB>
__device__ __noinline__ void hub_accum(const LpProblem &P, unsigned h0, unsigned h1, int lb, int nb, Smem &sm, unsigned char *dsm) {
  constexpr bool LQ = TB == 0;
  constexpr bool kStage = TB == 2;
  constexpr int kCap = kHubCap;
  constexpr int kChunk = kHubChunkT<TB>;
  unsigned long long *svals = reinterpret_cast<unsigned long long *>(dsm);
  int *skeys = reinterpret_cast<int *>(dsm + kCap * 8);
  unsigned *sq = reinterpret_cast<unsigned *>(dsm + kCap * 12);
  unsigned char *stage = dsm + kStageOff;
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ int s_to;
  for (int t = threadIdx.x; t < kCap; t += kThreads) {
    skeys[t] = -1;
    svals[t] = 0;
    if (LQ) sq[t] = 0;
  }
  const unsigned c_lo = P.hub_prefix[h0], c_hi = P.hub_prefix[h1];
  // chunk c of the batch: its hub position and entries
  auto chunk_of = [&](unsigned c, unsigned *ip, int64_t *bp, int64_t *ep) {
    const unsigned i = search_prefix(P.hub_prefix, h0, h1, c);
    const int v = P.bin[6][i];
    const int64_t rb = P.g.row_begin(v), re = P.g.row_begin(v + 1);
    *ip = i;
    *bp = rb + (int64_t)(c - P.hub_prefix[i]) * kChunk;
    *ep = min(re, *bp + kChunk);
  };
  if (kStage) {
    if (threadIdx.x == 0) {
      mbar_init(&s_bar[0]);
      mbar_init(&s_bar[1]);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_to = 0;
    }
    // this thread's earlier writes of the staging area (other phases' tables) before the bulk copies
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (kStage && threadIdx.x == 0 && c_lo + lb < c_hi) {
    unsigned i;
    int64_t b, e;
    chunk_of(c_lo + lb, &i, &b, &e);
    HubChunk<EW>::issue(P, b, e, stage, &s_bar[0]);
  }
  // a chunk's staged view (the direct loads when not staging)
  auto stage_next = [&](unsigned c, unsigned j) {
    if (kStage && threadIdx.x == 0 && c + nb < c_hi) {
      unsigned i;
      int64_t b, e;
      chunk_of(c + nb, &i, &b, &e);
      HubChunk<EW>::issue(P, b, e, stage + ((j + 1) & 1) * kStageBuf, &s_bar[(j + 1) & 1]);
    }
  };
  auto stage_wait = [&](unsigned j) -> bool {
    if (!kStage) return true;
    if (mbar_wait(&s_bar[j & 1], (j >> 1) & 1, 1000ull * P.wait_us)) return true;
    s_to = 1;
    return false;
  };
  // after a wait ran out (s_to, read after a block barrier): the copies in flight are waited for once
  // more (one second at most) and the call reports the timeout
  auto stage_abort = [&](unsigned j, unsigned c) {
    if (threadIdx.x == 0) {
      bool idle = mbar_wait(&s_bar[j & 1], (j >> 1) & 1, 1000000000ull);
      if (c + nb < c_hi) idle = mbar_wait(&s_bar[(j + 1) & 1], ((j + 1) >> 1) & 1, 1000000000ull) && idle;
      if (idle) {
        mbar_inval(&s_bar[0]);
        mbar_inval(&s_bar[1]);
      }
      atomicExch(&P.ctr->err, GP_ERR_TIMEOUT);
    }
  };
  auto stage_done = [&]() {
    if (kStage) {
      __syncthreads();
      if (threadIdx.x == 0) {
        mbar_inval(&s_bar[0]);
        mbar_inval(&s_bar[1]);
      }
    }
  };
  if (!LQ && P.hub_dense) {
    // few labels: a shared counter per label, flushed into the hub's dense table
    const int nl = (int)P.nl;
    unsigned j = 0;
    for (unsigned c = c_lo + lb; c < c_hi; c += nb, j++) {
      unsigned i;
      int64_t beg, end;
      chunk_of(c, &i, &beg, &end);
      const int v = P.bin[6][i];
      const int64_t tb = P.hub_tb[i];
      const int L0 = P.labels[P.vbase + v];
      stage_next(c, j);
      const bool ok = stage_wait(j);
      HubChunk<EW> hc;
      if (kStage) hc.view(P, beg, end, stage + (j & 1) * kStageBuf);
      long long c0 = 0;
      for (int64_t s0 = beg; s0 < end; s0 += 4 * kThreads) {
        int64_t e[4];
        int L[4];
        long long w[4];
        bool in[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          e[u] = s0 + u * kThreads + threadIdx.x;
          in[u] = ok && e[u] < end;
          L[u] = in[u] ? (kStage ? hc.adj(P, e[u]) : __ldg(P.g.adj + e[u])) : 0;
          w[u] = in[u] ? (kStage ? hc.ew(P, e[u]) : load_ew<EW>(P.g.ew, e[u])) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) L[u] = in[u] ? P.labels[L[u]] : -1;
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (in[u] && L[u] == L0) c0 += w[u];
          const bool on = in[u] && (P.hub_keep || L[u] != L0);  // kept tables hold the own label too
          const unsigned peers = __match_any_sync(kFull, on ? L[u] : -1);
          long long sum = 0;
          if (on)
            for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, w[u], __ffs(m) - 1);
          if (on && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
            atomicAdd(&svals[L[u] - P.lbase], (unsigned long long)sum);
        }
      }
      c0 = block_sum_of(c0, sm);  // also completes the counters (and makes s_to visible)
      if (kStage && s_to) {
        stage_abort(j, c);
        return;
      }
      if (P.hub_keep) c0 = 0;  // (kept tables: the choice looks the own label up)
      for (int t = threadIdx.x; t < nl; t += kThreads) {
        const unsigned long long x = svals[t];
        if (x) {
          atomicAdd(&P.hub_vals[tb + t], x);
          svals[t] = 0;
        }
      }
      if (kStage) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // (the buffer is refilled next)
      __syncthreads();
      if (threadIdx.x == 0 && c0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.hub_c0[i]), (unsigned long long)c0);
    }
    stage_done();
    return;
  }
  unsigned j = 0;
  for (unsigned c = c_lo + lb; c < c_hi; c += nb, j++) {
    unsigned i;
    int64_t beg, end;
    chunk_of(c, &i, &beg, &end);
    const int v = P.bin[6][i];
    const int64_t tb = P.hub_tb[i];
    const uint64_t cap = (uint64_t)(P.hub_capx[i + 1] - P.hub_capx[i]);
    const int L0 = P.labels[P.vbase + v];
    stage_next(c, j);
    const bool ok = stage_wait(j);
    HubChunk<EW> hc;
    if (kStage) hc.view(P, beg, end, stage + (j & 1) * kStageBuf);
    long long c0 = 0;
    // steps of 4 * kThreads entries: each thread takes four, loads first
    static_assert(kChunk % (4 * kThreads) == 0 && 2 * kChunk <= kCap, "a chunk fills at most half the table");
    for (int64_t s0 = beg; s0 < end; s0 += 4 * kThreads) {
      int64_t e[4];
      int L[4];
      long long w[4];
      unsigned q4[4];
      bool in[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        e[u] = s0 + u * kThreads + threadIdx.x;
        in[u] = ok && e[u] < end;
        L[u] = in[u] ? (kStage ? hc.adj(P, e[u]) : __ldg(P.g.adj + e[u])) : 0;
        w[u] = in[u] ? (kStage ? hc.ew(P, e[u]) : load_ew<EW>(P.g.ew, e[u])) : 0;
        q4[u] = (LQ && in[u]) ? (unsigned)__ldg(P.q + e[u]) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) L[u] = in[u] ? P.labels[L[u]] : -1;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (in[u] && L[u] == L0) c0 += w[u];
        warp_insert<EW, LQ>(skeys, svals, sq, kCap - 1, in[u] && (P.hub_keep || L[u] != L0), L[u], w[u], q4[u], P.ctr,
                            3);
      }
    }
    c0 = block_sum_of(c0, sm);  // also completes the shared table (and makes s_to visible)
    if (kStage && s_to) {
      stage_abort(j, c);
      return;
    }
    // flush into the hub's table: each thread claims the slots of four of its labels at once (the
    // claims are in flight together), then retries the ones that met another label
    static_assert(kCap % (4 * kThreads) == 0, "the flush takes four table slots per thread per step");
    for (int t0 = threadIdx.x; t0 < kCap; t0 += 4 * kThreads) {
      int Ls[4];
      uint64_t sg[4];
      bool pend[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        Ls[q] = skeys[t0 + q * kThreads];
        pend[q] = Ls[q] >= 0;
        sg[q] = pend[q] ? hub_slot(Ls[q], cap) : 0;
      }
      uint64_t probes = 0;
      while (pend[0] || pend[1] || pend[2] || pend[3]) {
        if (++probes > cap) {  // the hub's table is full: record and drop the remaining labels
          table_full(P.ctr, 4);
          break;
        }
        int ks[4];
#pragma unroll
        for (int q = 0; q < 4; q++) ks[q] = pend[q] ? atomicCAS(&P.hub_keys[tb + sg[q]], -1, Ls[q]) : 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (!pend[q]) continue;
          if (ks[q] == -1 || ks[q] == Ls[q]) {
            const int t = t0 + q * kThreads;
            atomicAdd(&P.hub_vals[tb + sg[q]], svals[t]);
            if (LQ) atomicAdd(&P.hub_qv[tb + sg[q]], (unsigned long long)sq[t]);
            pend[q] = false;
          } else {
            sg[q] = sg[q] + 1 == cap ? 0 : sg[q] + 1;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int t = t0 + q * kThreads;
        skeys[t] = -1;
        svals[t] = 0;
        if (LQ) sq[t] = 0;
      }
    }
    if (kStage) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // (the buffer is refilled next)
    __syncthreads();
    if (threadIdx.x == 0 && c0 && !P.hub_keep)
      atomicAdd(reinterpret_cast<unsigned long long *>(&P.hub_c0[i]), (unsigned long long)c0);
  }
  stage_done();
}

// Choice for batch [h0, h1), part 1: the batch's tables are scanned in items of kSlotChunk slots by all
// blocks; each item keeps its best eligible label (and clears its slots, unless the tables are kept).
template <bool LQ>
__device__ __noinline__ void hub_choose_part(const LpProblem &P, unsigned h0, unsigned h1, int lb, int nb, Smem &sm) {
  const unsigned s_lo = P.hub_scx[h0], s_hi = P.hub_scx[h1];
  Best *part = reinterpret_cast<Best *>(P.hub_part);
  constexpr int kU = 2;  // slots per thread in flight
  for (unsigned it = s_lo + lb; it < s_hi; it += nb) {
    const unsigned i = search_prefix(P.hub_scx, h0, h1, it);
    const int v = P.bin[6][i];
    const int64_t cap = P.hub_capx[i + 1] - P.hub_capx[i];
    const int64_t tb = P.hub_tb[i];
    const int64_t s0 = (int64_t)(it - P.hub_scx[i]) * kSlotChunk, s1 = min(cap, s0 + kSlotChunk);
    const int L0 = P.labels[P.vbase + v];
    long long c0 = P.hub_c0[i];
    if (P.hub_keep) {
      // a kept table holds the own label's connection; the hub's first item records it for the final step
      __shared__ long long s_c0;
      if (threadIdx.x == 0) {
        s_c0 = hub_lookup(P, tb, (uint64_t)cap, L0);
        if (it == P.hub_scx[i]) P.hub_c0[i] = s_c0;
      }
      __syncthreads();
      c0 = s_c0;
    }
    const long long cv = P.g.vweight(v);
    Best b = no_best();
    for (int64_t base = s0; base < s1; base += kU * kThreads) {
      int L[kU];
      long long cw[kU], lwL[kU];
      unsigned long long qq[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int64_t sl = base + u * kThreads + threadIdx.x;
        if (P.hub_dense) L[u] = (sl < s1 && P.hub_vals[tb + sl] != 0) ? (int)(P.lbase + sl) : -1;
        else L[u] = sl < s1 ? P.hub_keys[tb + sl] : -1;
      }
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int64_t sl = base + u * kThreads + threadIdx.x;
        cw[u] = L[u] >= 0 ? (long long)P.hub_vals[tb + sl] : 0;
        qq[u] = (LQ && L[u] >= 0) ? P.hub_qv[tb + sl] : 0ull;
      }
      // label weights only of labels that could win (more connection than the own label)
#pragma unroll
      for (int u = 0; u < kU; u++) lwL[u] = (L[u] >= 0 && L[u] != L0 && cw[u] > c0) ? P.lw[L[u]] : 0;
#pragma unroll
      for (int u = 0; u < kU; u++) {
        if (L[u] < 0) continue;
        const int64_t sl = base + u * kThreads + threadIdx.x;
        const Best x = make_cand_lw(P, v, L[u], L0, cw[u], (long long)qq[u], c0, cv, lwL[u]);
        if (better(x, b)) b = x;
        if (P.hub_keep) continue;  // kept tables stay
        if (!P.hub_dense) P.hub_keys[tb + sl] = -1;
        P.hub_vals[tb + sl] = 0;
        if (LQ) P.hub_qv[tb + sl] = 0;
      }
    }
    b = block_best_of<LQ>(b, sm);
    if (threadIdx.x == 0) part[it - s_lo] = b;
  }
}

// Choice for batch [h0, h1), part 2: one thread per hub combines its items and records the proposal.
__device__ void hub_choose_final(const LpProblem &P, unsigned h0, unsigned h1, int lb, int nb) {
  const unsigned s_lo = P.hub_scx[h0];
  const Best *part = reinterpret_cast<const Best *>(P.hub_part);
  for (unsigned i = h0 + (unsigned)lb * kThreads + threadIdx.x; i < h1; i += (unsigned)nb * kThreads) {
    Best b = no_best();
    for (unsigned it = P.hub_scx[i]; it < P.hub_scx[i + 1]; it++)
      if (better(part[it - s_lo], b)) b = part[it - s_lo];
    const int v = P.bin[6][i];
    write_slot<true>(P, P.bin_base[6] + i, v, b, P.hub_c0[i]);
    if (b.L >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)P.g.vweight(v));
  }
}

// Hubs in the first sub-round of a clustering from singletons: every entry is its own candidate, so the rows are
// scanned in chunks by all blocks (best candidate per chunk) and one thread per hub combines its
// chunks; no tables.
template <int EW, bool LQ>
__device__ void hub_direct_part(const LpProblem &P, unsigned cnt, unsigned chunks, int lb, int nb, Smem &sm) {
  Best *part = reinterpret_cast<Best *>(P.hub_part);
  for (unsigned c = lb; c < chunks; c += nb) {
    const unsigned i = search_prefix(P.hub_prefix, 0, cnt, c);
    const int v = P.bin[6][i];
    const int64_t rb = P.g.row_begin(v), re = P.g.row_begin(v + 1);
    const int64_t beg = rb + (int64_t)(c - P.hub_prefix[i]) * P.hub_chunk;
    const int64_t end = min(re, beg + P.hub_chunk);
    const int L0 = P.labels[P.vbase + v];
    const long long cv = P.g.vweight(v);
    Best b = no_best();
    for (int64_t e = beg + threadIdx.x; e < end; e += kThreads) {
      const Best x = make_cand(P, v, P.labels[__ldg(P.g.adj + e)], L0, load_ew<EW>(P.g.ew, e),
                               LQ ? (long long)__ldg(P.q + e) : 0, 0, cv);
      if (better(x, b)) b = x;
    }
    b = block_best_of<LQ>(b, sm);
    if (threadIdx.x == 0) part[c] = b;
  }
}

__device__ void hub_direct_final(const LpProblem &P, unsigned cnt, int lb, int nb) {
  const Best *part = reinterpret_cast<const Best *>(P.hub_part);
  for (unsigned i = (unsigned)lb * kThreads + threadIdx.x; i < cnt; i += (unsigned)nb * kThreads) {
    Best b = no_best();
    for (unsigned c = P.hub_prefix[i]; c < P.hub_prefix[i + 1]; c++)
      if (better(part[c], b)) b = part[c];
    const int v = P.bin[6][i];
    write_slot<true>(P, P.bin_base[6] + i, v, b, 0);
    if (b.L >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&P.demand[b.L]), (unsigned long long)P.g.vweight(v));
  }
}

// Active positions k in [0, sum of bin counts) map to proposal slots bin_base[b] + (k - start_b).
struct SlotMap {
  unsigned start[kBins + 1];
  int64_t base[kBins];
  __device__ __forceinline__ void init(const LpProblem &P, const SubCounters &C) {
    start[0] = 0;
#pragma unroll
    for (int b = 0; b < kBins; b++) {
      start[b + 1] = start[b] + C.bin_count[b];
      base[b] = P.bin_base[b];
    }
  }
  __device__ __forceinline__ unsigned total() const { return start[kBins]; }
  __device__ __forceinline__ int64_t slot(unsigned k) const {
    int b = 0;
#pragma unroll
    for (int x = 1; x < kBins; x++)
      if (k >= start[x]) b = x;
    return base[b] + (k - start[b]);
  }
};

// Admission check of every proposal; proposals to targets whose total demand does not fit are
// recorded as contested.
template <bool LQ>
__device__ void phase_admit(const LpProblem &P, SubCounters &C, const SubCounters &V, int r, int lb, int nb, Smem &sm) {
  SlotMap M;
  M.init(P, V);
  const unsigned na = M.total();
  unsigned long long mg = 0, mq = 0;
  unsigned movers = 0, moved = 0;
  uint8_t *act_next = r + 1 < P.rounds ? P.act[(r + 1) & 1] : nullptr;  // (no marks in the last round)
  for (unsigned base = (unsigned)lb * kThreads; base < na; base += (unsigned)nb * kThreads) {
    const unsigned k = base + threadIdx.x;
    bool contested = false, adm = false;
    int64_t i = 0;
    int T = -1, v = 0;
    int L0 = 0;
    int64_t rb = 0, deg = 0;
    if (k < na) {
      // target and vertex first, then the target's weights and the vertex's label and row together
      i = M.slot(k);
      T = P.mv_t[i];
      v = P.mv_v[i];
      if (T >= 0) {
        movers++;
        const long long lwT = P.lw[T], dT = P.demand[T];
        L0 = P.labels[P.vbase + v];
        rb = P.g.row_begin(v);
        deg = P.g.row_begin(v + 1) - rb;
        if (lwT + dT <= P.U) {
          adm = true;
          P.mv_adm[i] = 1;
        } else {
          contested = true;
          mg = max(mg, (unsigned long long)P.mv_gain[i]);
          if (LQ) mq = max(mq, (unsigned long long)P.mv_q[i]);
        }
      }
    }
    moved += apply_movers_pre(P, C, act_next, adm, i, v, T, L0, rb, deg);
    const unsigned pos = warp_append(&C.n_contested, contested);
    if (contested) P.ct[pos] = (unsigned)i;
  }
  // movers (statistics) add up in shared memory over the call; the round's move count gets one
  // atomic per block
  movers = warp_sum_u32(movers);
  if ((threadIdx.x & 31) == 0) {
    if (movers) atomicAdd(&sm.movers, (unsigned long long)movers);
    if (moved) atomicAdd(&sm.moves, (unsigned long long)moved);
  }
  __syncthreads();
  if (threadIdx.x == 0 && sm.moves) {
    atomicAdd(&P.ctr->moves_round[r & 1], sm.moves);
    sm.moves = 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mg = max(mg, __shfl_xor_sync(kFull, mg, o));
    mq = max(mq, __shfl_xor_sync(kFull, mq, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mg) atomicMax(&C.max_gain, mg);
    if (LQ && mq) atomicMax(&C.max_q, mq);
  }
}

// Contested order: target asc, gain desc, score sum desc (with scores), id asc.
template <bool LQ>
__device__ __forceinline__ bool mover_less(const LpProblem &P, unsigned x, unsigned y) {
  const int tx = P.mv_t[x], ty = P.mv_t[y];
  if (tx != ty) return tx < ty;
  const long long gx = P.mv_gain[x], gy = P.mv_gain[y];
  if (gx != gy) return gx > gy;
  if (LQ) {
    const long long qx = P.mv_q[x], qy = P.mv_q[y];
    if (qx != qy) return qx > qy;
  }
  return P.mv_v[x] < P.mv_v[y];
}

// Segmented inclusive prefix sums of c(v) over positions [lo, hi) of a sequence sorted by target,
// starting from the carry of the segment open before lo; a proposal is admitted while the target's
// snapshot weight plus the prefix fits. at(p) gives (target, proposal index) of position p.
template <class At>
__device__ void admit_sorted(const LpProblem &P, At at, unsigned lo, unsigned hi, long long carry_in,
                             int carry_target, int r, SubCounters *Cg, Smem &sm) {
  uint8_t *act_next = r + 1 < P.rounds ? P.act[(r + 1) & 1] : nullptr;  // (no marks in the last round)
  unsigned moved = 0;
  if (threadIdx.x == 0) {
    sm.carry = carry_in;
    sm.carry_t = carry_target;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (unsigned base = lo; base < hi; base += kThreads) {
    const unsigned p = base + threadIdx.x;
    const bool valid = p < hi;
    int T = -1, Tprev = -1;
    unsigned idx = 0;
    if (valid) {
      at(p, T, idx);
      if (p > lo) {
        unsigned dummy;
        at(p - 1, Tprev, dummy);
      } else {
        Tprev = sm.carry_t;
      }
    }
    const bool head = valid && T != Tprev;
    const long long c = valid ? P.g.vweight(P.mv_v[idx]) : 0;
    int f = head ? 1 : 0;
    long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, x, o);
      const int fy = __shfl_up_sync(kFull, f, o);
      if (lane >= o) {
        if (!f) x += y;
        f |= fy;
      }
    }
    if (lane == 31) {
      sm.sum[wid] = x;
      sm.wflag[wid] = (unsigned)f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long run = sm.carry;
      for (int w = 0; w < kWarps; w++) {
        const long long s = sm.sum[w];
        const int fl = (int)sm.wflag[w];
        sm.sum[w] = run;  // carry into warp w
        run = fl ? s : run + s;
      }
    }
    __syncthreads();
    const long long incl = f ? x : x + sm.sum[wid];
    const bool adm = valid && P.lw[T] + incl <= P.U;
    if (adm) P.mv_adm[idx] = 1;
    moved += apply_movers(P, *Cg, act_next, adm, idx, adm ? P.mv_v[idx] : 0, T);
    __syncthreads();
    const unsigned last = min(hi, base + (unsigned)kThreads) - 1;
    if (p == last) {
      sm.carry = incl;
      sm.carry_t = T;
    }
    __syncthreads();
  }
  if ((threadIdx.x & 31) == 0 && moved) atomicAdd(&P.ctr->moves_round[r & 1], (unsigned long long)moved);
}

__device__ __forceinline__ int bits_for(unsigned long long x) { return x ? 64 - __clzll(x) : 0; }

// Small contested sets (one CTA). When (target, gain desc, score desc, id) packs into 64 bits the
// keys are sorted in shared memory (bitonic); otherwise proposal indices are sorted with a comparator.
template <bool LQ>
__device__ void contest_small(const LpProblem &P, const SubCounters &C, SubCounters *Cg, unsigned cnt, int r,
                              unsigned char *dsm, Smem &sm) {
  unsigned Pp = 1;
  while (Pp < cnt) Pp <<= 1;
  const unsigned long long maxg = C.max_gain, maxq = C.max_q;
  const int bv = bits_for((unsigned long long)(P.g.n > 0 ? P.g.n - 1 : 0));
  const int bq = LQ ? bits_for(maxq) : 0;
  const int bg = bits_for(maxg);
  const int bt = bits_for((unsigned long long)(P.nl > 0 ? P.nl - 1 : 0));
  __syncthreads();
  if (bv + bq + bg + bt <= 63) {  // top bit clear: real keys never equal the padding
    unsigned long long *key = reinterpret_cast<unsigned long long *>(dsm);
    const int sq = bv, sg = bv + bq, st = bv + bq + bg;
    for (unsigned i = threadIdx.x; i < Pp; i += kThreads) {
      unsigned long long k = ~0ull;
      if (i < cnt) {
        const unsigned idx = P.ct[i];
        k = (unsigned long long)(unsigned)P.mv_v[idx];
        if (LQ && bq) k |= (maxq - (unsigned long long)P.mv_q[idx]) << sq;
        if (bg) k |= (maxg - (unsigned long long)P.mv_gain[idx]) << sg;
        if (bt) k |= (unsigned long long)(P.mv_t[idx] - P.lbase) << st;
      }
      key[i] = k;
    }
    __syncthreads();
    for (unsigned k = 2; k <= Pp; k <<= 1) {
      for (unsigned j = k >> 1; j > 0; j >>= 1) {
        for (unsigned t = threadIdx.x; t < Pp / 2; t += kThreads) {
          const unsigned i = 2 * j * (t / j) + (t % j), l = i + j;
          const bool up = (i & k) == 0;
          const unsigned long long x = key[i], y = key[l];
          if ((x > y) == up && x != y) {
            key[i] = y;
            key[l] = x;
          }
        }
        __syncthreads();
      }
    }
    const unsigned long long vmask = bv >= 64 ? ~0ull : ((1ull << bv) - 1);
    admit_sorted(
        P,
        [&](unsigned p, int &T, unsigned &idx) {
          const unsigned long long k = key[p];
          T = (int)((bt ? (long long)(k >> st) : 0) + P.lbase);
          idx = (unsigned)P.mv_of_v[(int)(k & vmask)];
        },
        0, cnt, 0, -1, r, Cg, sm);
    if (threadIdx.x == 0) P.ctr->contest_packed += 1;
    return;
  }
  unsigned *key = reinterpret_cast<unsigned *>(dsm);
  for (unsigned i = threadIdx.x; i < Pp; i += kThreads) key[i] = i < cnt ? P.ct[i] : 0xffffffffu;
  __syncthreads();
  for (unsigned k = 2; k <= Pp; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned t = threadIdx.x; t < Pp / 2; t += kThreads) {
        const unsigned i = 2 * j * (t / j) + (t % j), l = i + j;
        const bool up = (i & k) == 0;
        const unsigned x = key[i], y = key[l];
        bool swap;
        if (x == 0xffffffffu) swap = (y != 0xffffffffu) == up;
        else if (y == 0xffffffffu) swap = !up;
        else swap = mover_less<LQ>(P, y, x) == up;
        if (swap) {
          key[i] = y;
          key[l] = x;
        }
      }
      __syncthreads();
    }
  }
  admit_sorted(
      P,
      [&](unsigned p, int &T, unsigned &idx) {
        idx = key[p];
        T = P.mv_t[idx];
      },
      0, cnt, 0, -1, r, Cg, sm);
  if (threadIdx.x == 0) P.ctr->contest_small += 1;
}

__device__ __forceinline__ unsigned long long field_key(const LpProblem &P, unsigned idx, int field,
                                                        unsigned long long maxg, unsigned long long maxq) {
  switch (field) {
    case 0: return (unsigned long long)(unsigned)P.mv_v[idx];
    case 1: return maxq - (unsigned long long)P.mv_q[idx];
    case 2: return maxg - (unsigned long long)P.mv_gain[idx];
    default: return (unsigned long long)(P.mv_t[idx] - P.lbase);
  }
}

// Large contested sets: stable LSD radix sort over the problem's blocks, then segmented admission.
// When (target, gain desc, score desc, id) fits 64 bits the key is built once per mover and carried
// with its proposal index (contiguous reads); otherwise the fields are gathered from the proposal
// arrays in every pass, least significant first (id, score sum desc, gain desc, target).
template <bool LQ>
__device__ bool contest_large(const LpProblem &P, const SubCounters &C, SubCounters *Cg, unsigned cnt, int r, int lb,
                              int nb, const GridBarrier &bar, Smem &sm, unsigned char *dsm) {
  const unsigned long long maxg = C.max_gain, maxq = C.max_q;
  const int nbits[4] = {bits_for((unsigned long long)(P.g.n > 0 ? P.g.n - 1 : 0)), LQ ? bits_for(maxq) : 0,
                        bits_for(maxg), bits_for((unsigned long long)(P.nl > 0 ? P.nl - 1 : 0))};
  const int tbits = nbits[0] + nbits[1] + nbits[2] + nbits[3];
  const bool packed = tbits <= 64;
  const int sq = nbits[0], sg = nbits[0] + nbits[1], st = nbits[0] + nbits[1] + nbits[2];
  const unsigned chunk = (cnt + nb - 1) / nb;
  const unsigned lo = min(cnt, (unsigned)lb * chunk), hi = min(cnt, lo + chunk);
  unsigned *src = P.ct, *dst = P.ct2;
  unsigned long long *ks = P.ck, *kd = P.ck2;
  const int wid = threadIdx.x >> 5;
  // radix workspace in the dynamic shared memory (the choice tables are idle during the contest):
  // digit counts, per-digit output bases and per-warp digit counts
  unsigned *const s_hist = reinterpret_cast<unsigned *>(dsm);
  unsigned long long *const s_base = reinterpret_cast<unsigned long long *>(dsm + 256 * sizeof(unsigned));
  unsigned (*const s_wcnt)[256] =
      reinterpret_cast<unsigned (*)[256]>(dsm + 256 * (sizeof(unsigned) + sizeof(unsigned long long)));
  static_assert(256 * (4 + 8) + kWarps * 256 * 4 <= (int)kDynSmem, "radix workspace fits the dynamic smem");
  if (packed) {
    for (unsigned p = lo + threadIdx.x; p < hi; p += kThreads) {
      const unsigned idx = src[p];
      unsigned long long k = (unsigned long long)(unsigned)P.mv_v[idx];
      if (LQ && nbits[1]) k |= (maxq - (unsigned long long)P.mv_q[idx]) << sq;
      if (nbits[2]) k |= (maxg - (unsigned long long)P.mv_gain[idx]) << sg;
      if (nbits[3]) k |= (unsigned long long)(P.mv_t[idx] - P.lbase) << st;
      ks[p] = k;
    }
    __syncthreads();
  }
  // passes: packed keys in 8-bit digits; otherwise (field, shift) pairs
  int field = 0, shift = 0;
  if (!packed)
    while (field < 4 && nbits[field] == 0) field++;
  while (packed ? shift < tbits : field < 4) {
    auto digit = [&](unsigned p) -> int {
      return packed ? (int)((ks[p] >> shift) & 255)
                    : (int)((field_key(P, src[p], field, maxg, maxq) >> shift) & 255);
    };
    for (int t = threadIdx.x; t < 256; t += kThreads) s_hist[t] = 0;
    __syncthreads();
    for (unsigned p = lo + threadIdx.x; p < hi; p += kThreads) atomicAdd(&s_hist[digit(p)], 1u);
    __syncthreads();
    // digit-major counts: hist[d * nb + block]
    for (int t = threadIdx.x; t < 256; t += kThreads) P.hist[(size_t)t * nb + lb] = s_hist[t];
    if (!grid_sync(bar)) return false;
    // one warp per digit scans the per-block counts (coalesced, 32 blocks per step)
    {
      const int lane = threadIdx.x & 31;
      for (unsigned d = (unsigned)lb * kWarps + wid; d < 256; d += (unsigned)nb * kWarps) {
        unsigned long long run = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
          const int bb = b0 + lane;
          const unsigned long long h = bb < nb ? P.hist[(size_t)d * nb + bb] : 0;
          unsigned long long inc = h;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
          }
          if (bb < nb) P.hoff[(size_t)bb * 256 + d] = run + inc - h;
          run += __shfl_sync(kFull, inc, 31);
        }
        if (lane == 0) P.hoff[(size_t)nb * 256 + d] = run;
      }
    }
    if (!grid_sync(bar)) return false;
    {
      // this block's start per digit: digits below (exclusive scan of the totals) + blocks before
      const int t = threadIdx.x;
      const long long tot = t < 256 ? (long long)P.hoff[(size_t)nb * 256 + t] : 0;
      const long long own = t < 256 ? (long long)P.hoff[(size_t)lb * 256 + t] : 0;
      const long long ex = block_excl_scan64(tot, sm.tmp, (long long *)nullptr);
      if (t < 256) s_base[t] = (unsigned long long)(ex + own);
    }
    __syncthreads();
    for (unsigned t0 = lo; t0 < hi; t0 += kThreads) {
      const unsigned p = t0 + threadIdx.x;
      const bool valid = p < hi;
      const unsigned x = valid ? src[p] : 0;
      const unsigned long long kx = (valid && packed) ? ks[p] : 0;
      const int dg = valid ? digit(p) : 256;
      for (int k = threadIdx.x; k < kWarps * 256; k += kThreads) s_wcnt[k >> 8][k & 255] = 0;
      __syncthreads();
      const unsigned peers = __match_any_sync(kFull, dg);
      const int rank = __popc(peers & lanemask_lt());
      if (valid && rank == 0) s_wcnt[wid][dg] = __popc(peers);
      __syncthreads();
      if (valid) {
        unsigned pre = 0;
        for (int w = 0; w < wid; w++) pre += s_wcnt[w][dg];
        const unsigned long long pos = s_base[dg] + pre + rank;
        dst[pos] = x;
        if (packed) kd[pos] = kx;
      }
      __syncthreads();
      if (threadIdx.x < 256) {
        unsigned s2 = 0;
        for (int w = 0; w < kWarps; w++) s2 += s_wcnt[w][threadIdx.x];
        s_base[threadIdx.x] += s2;
      }
      __syncthreads();
    }
    if (!grid_sync(bar)) return false;
    unsigned *t = src;
    src = dst;
    dst = t;
    unsigned long long *tk = ks;
    ks = kd;
    kd = tk;
    shift += 8;
    if (!packed && shift >= nbits[field]) {
      shift = 0;
      field++;
      while (field < 4 && nbits[field] == 0) field++;
    }
  }
  // carries between block slices: per block (sum of the trailing segment, whether the slice has a
  // segment head, target of its last element), resolved in order by one thread
  long long tail = 0;
  int has_head = 0, last_t = -1;
  if (lo < hi) {
    last_t = P.mv_t[src[hi - 1]];
    long long part = 0;
    int hs = 0;
    for (unsigned p = lo + threadIdx.x; p < hi; p += kThreads) {
      const unsigned idx = src[p];
      if (P.mv_t[idx] == last_t) part += P.g.vweight(P.mv_v[idx]);
      else hs = 1;
    }
    tail = block_sum_of(part, sm);
    has_head = __syncthreads_or(hs);
  }
  if (threadIdx.x == 0) {
    P.hoff[(size_t)lb * 4 + 0] = (unsigned long long)tail;
    P.hoff[(size_t)lb * 4 + 1] = (unsigned long long)has_head;
    P.hoff[(size_t)lb * 4 + 2] = (unsigned long long)(long long)last_t;
    P.hoff[(size_t)lb * 4 + 3] = (unsigned long long)(hi > lo ? 1 : 0);
  }
  if (!grid_sync(bar)) return false;
  if (lb == 0) {
    // stage the per-block summaries in shared memory (coalesced), resolve them in order, write back
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(dsm);  // 4 words per block
    for (int x = threadIdx.x; x < nb * 4; x += kThreads) stage[x] = P.hoff[x];
    __syncthreads();
    if (threadIdx.x == 0) {
      long long run = 0, run_t = -1;
      for (int bb = 0; bb < nb; bb++) {
        const long long t = (long long)stage[bb * 4 + 0];
        const int hh = (int)stage[bb * 4 + 1];
        const long long lt = (long long)stage[bb * 4 + 2];
        const bool nonempty = stage[bb * 4 + 3] != 0;
        stage[bb * 4 + 0] = (unsigned long long)run;  // becomes the carry into block bb
        stage[bb * 4 + 1] = (unsigned long long)run_t;
        if (!nonempty) continue;
        if (!hh && lt == run_t) run += t;
        else run = t;
        run_t = lt;
      }
    }
    __syncthreads();
    for (int bb = threadIdx.x; bb < nb; bb += kThreads) {
      P.hoff[(size_t)nb * 4 + bb * 2 + 0] = stage[bb * 4 + 0];
      P.hoff[(size_t)nb * 4 + bb * 2 + 1] = stage[bb * 4 + 1];
    }
  }
  if (!grid_sync(bar)) return false;
  const long long carry = (long long)P.hoff[(size_t)nb * 4 + lb * 2 + 0];
  const int carry_t = (int)(long long)P.hoff[(size_t)nb * 4 + lb * 2 + 1];
  if (lo < hi)
    admit_sorted(
        P,
        [&](unsigned p, int &T, unsigned &idx) {
          idx = src[p];
          T = P.mv_t[idx];
        },
        lo, hi, carry, carry_t, r, Cg, sm);
  if (lb == 0 && threadIdx.x == 0) {
    P.ctr->contest_large += 1;
    P.ctr->contest_large_items += cnt;
  }
  return true;
}

template <int EW, int TB>
__device__ bool lp_problem(const LpProblem *prob, unsigned char *dsm) {
  constexpr bool LQ = TB == 0;
  __shared__ __align__(16) unsigned char p_raw[sizeof(LpProblem)];
  __shared__ Smem sm;
  LpProblem &P = *reinterpret_cast<LpProblem *>(p_raw);
  __syncthreads();  // the block's previous problem is done with the shared state
  {
    const unsigned *src = reinterpret_cast<const unsigned *>(prob);
    unsigned *dst = reinterpret_cast<unsigned *>(p_raw);
    for (unsigned i = threadIdx.x; i < sizeof(LpProblem) / 4; i += kThreads) dst[i] = src[i];
  }
  __syncthreads();
  const int lb = (int)blockIdx.x - P.block_begin, nb = P.block_count;
  LpCounters *ctr = P.ctr;
  // (built from the shared problem copy at every use, so that none of it stays in registers)
#define bar (GridBarrier{P.bar, &P.ctr->err, (unsigned)nb, (unsigned)lb, P.wait_us})
  // block 0 of the problem accumulates barrier-to-barrier time per phase (all blocks meet there) in
  // shared memory and writes the totals once at the end
  __shared__ unsigned long long pacc[8];
  if (threadIdx.x < 8) pacc[threadIdx.x] = 0;
  unsigned long long tmark = 0;
  auto tick = [&](int phase) {
    if (lb == 0 && threadIdx.x == 0) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (phase >= 0) pacc[phase] += now - tmark;
      tmark = now;
    }
  };
  // block-local copies of the sub-round counters (read once after a barrier)
  __shared__ SubCounters sV, sVp;
  // (one 32-bit word per thread, all loads in flight together; the bin counts come from binres)
  static_assert(offsetof(SubCounters, bin_count) == 0, "bin counts lead the counters");
  auto load_view = [&](const SubCounters &src, int t) {
    if (threadIdx.x < 8)
      sV.bin_count[threadIdx.x] = reinterpret_cast<const volatile unsigned *>(P.binres)[(t % 3) * 256 + threadIdx.x * 32];
    else if (threadIdx.x < sizeof(SubCounters) / 4)
      reinterpret_cast<unsigned *>(&sV)[threadIdx.x] =
          reinterpret_cast<const volatile unsigned *>(&src)[threadIdx.x];
    __syncthreads();
  };
  if (threadIdx.x < 8) {
    sm.vis[threadIdx.x] = 0;
    sm.edg[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) {
    sm.moves = 0;
    sm.movers = 0;
    for (int b = 0; b < 8; b++) sV.bin_count[b] = 0;
    sV.n_movers = sV.n_contested = sV.hub_chunks = sV.n_big = sV.hub_batches = 0;
    sV.max_gain = sV.max_q = 0;
  }
  tick(-1);
  int t_last = -1;
  for (int r = 0; r < P.rounds; r++) {
    const uint64_t rmix = mix64(P.smix ^ (uint64_t)r);
    for (int s = 0; s < 2; s++) {
      const int t = 2 * r + s;
      SubCounters &C = ctr->sc[t % 3];
      SubCounters &Cn = ctr->sc[(t + 1) % 3];
      if (lb == 0) {
        // counter set t+1 was last used by sub-round t-2, which every block has finished
        if (threadIdx.x < 8) P.binres[((t + 1) % 3) * 256 + threadIdx.x * 32] = 0;
        if (threadIdx.x == 0) {
          Cn.n_movers = 0;
          Cn.n_contested = 0;
          Cn.hub_chunks = 0;
          Cn.n_inval = 0;
          Cn.n_big = 0;
          Cn.hub_batches = 0;
          Cn.max_gain = 0;
          Cn.max_q = 0;
        }
      }
      __shared__ unsigned s_stale;
      if (threadIdx.x == 0) {
        sVp = sV;  // the counters of sub-round t-1
        P.sub_t = t;
        // kept hub tables that went stale in sub-round t-1 (its counters are final: every block has
        // passed the barrier after its last update)
        s_stale = (P.hub_keep && t > 0) ? *(volatile unsigned *)&ctr->sc[(t + 2) % 3].n_inval : 0u;
      }
      __syncthreads();
      phase_classify(P, C, t > 0 ? &sVp : nullptr, r, s, rmix, lb, nb, sm);
      if (s_stale) hub_clear_stale(P, s_stale, lb, nb);
      if (!grid_sync(bar)) return false;
      load_view(C, t);
      tick(0);
      t_last = t;
      unsigned active = 0;
      for (int b = 0; b < kBins; b++) active += sV.bin_count[b];
      if (active > 0) {
        // only the first sub-round sees every label as a singleton (the second follows its moves)
        const bool direct = P.singletons && t == 0;
        const bool hubs_now = P.has_hubs && sV.bin_count[6];
        if (lb == 0 && hubs_now) {
          hub_prefix(P, C, sV, sm, direct);
          tick(7);
        }
        // while block 0 prepares the hub list, the other blocks take its share of the choice
        const int clb = (hubs_now && nb > 1) ? lb - 1 : lb, cnb = (hubs_now && nb > 1) ? nb - 1 : nb;
        if (clb >= 0) {
          choose_groups<EW, LQ>(P, sV, clb, cnb);
          choose_warp<EW, TB>(P, sV, clb, cnb, dsm, direct);
          choose_cta<EW, TB>(P, sV, clb, cnb, dsm, sm, direct);
        }
        if (!grid_sync(bar)) return false;
        tick(1);
        if (P.has_hubs && sV.bin_count[6] && direct) {
          load_view(C, t);  // hub chunks
          hub_direct_part<EW, LQ>(P, sV.bin_count[6], sV.hub_chunks, lb, nb, sm);
          if (!grid_sync(bar)) return false;
          tick(2);
          hub_direct_final(P, sV.bin_count[6], lb, nb);
          if (!grid_sync(bar)) return false;
          tick(6);
        } else if (P.has_hubs && sV.bin_count[6]) {
          load_view(C, t);  // hub batches
          const unsigned nbat = sV.hub_batches;
          for (unsigned bt = 0; bt < nbat; bt++) {
            const unsigned h0 = P.hub_bstart[bt], h1 = P.hub_bstart[bt + 1];
            // (kept tables: only hubs whose table is not current have chunks; none: no pass)
            if (!P.hub_keep || sV.hub_chunks) {
              hub_accum<EW, TB>(P, h0, h1, lb, nb, sm, dsm);
              if (!grid_sync(bar)) return false;
            }
            tick(2);
            hub_choose_part<LQ>(P, h0, h1, lb, nb, sm);
            if (!grid_sync(bar)) return false;
            hub_choose_final(P, h0, h1, lb, nb);
            tick(6);
          }
          if (!grid_sync(bar)) return false;
          tick(6);
        }
        if (lb == 0 && threadIdx.x == 0 && s == 0) ctr->moves_round[(r + 1) & 1] = 0;
        phase_admit<LQ>(P, C, sV, r, lb, nb, sm);
        if (!grid_sync(bar)) return false;
        load_view(C, t);  // contested count and key ranges
        tick(3);
        const unsigned nc = sV.n_contested;
        if (nc > 0) {
          if (nc <= kContestSmall) {
            if (lb == 0) contest_small<LQ>(P, sV, &C, nc, r, dsm, sm);
          } else {
            if (!contest_large<LQ>(P, sV, &C, nc, r, lb, nb, bar, sm, dsm)) return false;
          }
          if (!grid_sync(bar)) return false;
          load_view(C, t);  // high-degree movers listed by the contest
          tick(4);
        }
        if (sV.n_big > 0) {
          mark_big(P, C, sV.n_big, r, lb, nb);
          if (!grid_sync(bar)) return false;
          tick(4);
        }
      } else if (lb == 0 && threadIdx.x == 0 && s == 0) {
        ctr->moves_round[(r + 1) & 1] = 0;
      }
    }
    // round end: every block reads the round's move count (final after the last barrier)
    __shared__ unsigned long long s_mr;
    if (threadIdx.x == 0) s_mr = *(volatile unsigned long long *)&ctr->moves_round[r & 1];
    __syncthreads();
    const unsigned long long mr = s_mr;
    if (lb == 0 && threadIdx.x == 0) {
      ctr->rounds += 1;
      ctr->moves += mr;
    }
    __syncthreads();
    if (mr == 0) break;
  }
  // label weights of the last sub-round's moves (every block has passed its final barrier)
  if (t_last >= 0) settle_moves(P, sV, lb, nb);
  __syncthreads();
  if (threadIdx.x < 8) {
    if (sm.vis[threadIdx.x]) atomicAdd(&ctr->bin_visits[threadIdx.x], sm.vis[threadIdx.x]);
    if (sm.edg[threadIdx.x]) atomicAdd(&ctr->bin_edges[threadIdx.x], sm.edg[threadIdx.x]);
  }
  if (threadIdx.x == 0 && sm.movers) atomicAdd(&ctr->movers, sm.movers);
  tick(5);
  if (lb == 0 && threadIdx.x == 0)
    for (int k = 0; k < 8; k++) ctr->phase_ns[k] = pacc[k];
  return true;
}

#undef bar

// One launch runs every problem: block b runs the problems blk_list[blk_start[b] .. blk_start[b+1])
// in order. A problem of several blocks is the only problem of each of its blocks; problems of one
// block may share a block with others (small graphs of a batch).
template <int EW, int TB>
__global__ void __launch_bounds__(kThreads, 4) k_lp(const LpProblem *probs, const int *blk_start, const int *blk_list) {
  extern __shared__ __align__(16) unsigned char dsm[];
  for (int q = blk_start[blockIdx.x]; q < blk_start[blockIdx.x + 1]; q++)
    if (!lp_problem<EW, TB>(probs + blk_list[q], dsm)) return;
}

// ------------------------------------------------------------------------------------ host helpers
// Degree classes and CSR entries of every job of a launch: counts[9 j + bin] vertices per bin and
// counts64[j] entries. Vertex x of the concatenation belongs to the job j with pre[j] <= x < pre[j+1].
// With at most kClsSmemJobs jobs the counts add up in shared memory first (one global atomic per
// block and counter instead of one per warp: the counters of a job share a cache line).
constexpr int kClsSmemJobs = 16;

__global__ void k_degree_classes(const DGraph *gs, const int64_t *pre, int njobs, int deg_warp, int deg_cta,
                                 unsigned *counts, unsigned long long *entries, unsigned long long *hubstat) {
  __shared__ unsigned s_counts[9 * kClsSmemJobs];
  __shared__ unsigned long long s_entries[kClsSmemJobs], s_hub[3 * kClsSmemJobs];
  const bool local = njobs <= kClsSmemJobs;
  if (local) {
    for (int t = threadIdx.x; t < 9 * kClsSmemJobs; t += blockDim.x) s_counts[t] = 0;
    for (int t = threadIdx.x; t < kClsSmemJobs; t += blockDim.x) s_entries[t] = 0;
    for (int t = threadIdx.x; t < 3 * kClsSmemJobs; t += blockDim.x) s_hub[t] = 0;
    __syncthreads();
  }
  unsigned *cnt_out = local ? s_counts : counts;
  unsigned long long *ent_out = local ? s_entries : entries, *hub_out = local ? s_hub : hubstat;
  const int64_t total = pre[njobs];
  const int lane = threadIdx.x & 31;
  for (int64_t x0 = blockIdx.x * (int64_t)blockDim.x; x0 < total; x0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = x0 + threadIdx.x;
    int j = -1, bin = -1;
    int64_t d = 0;
    if (x < total) {
      int lo = 0, hi = njobs;  // largest j with pre[j] <= x
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= x) lo = mid;
        else hi = mid;
      }
      j = lo;
      const DGraph &g = gs[j];
      const int64_t v = x - pre[j];
      d = g.row_begin(v + 1) - g.row_begin(v);
      if (d > 0) bin = bin_of(d, deg_warp, deg_cta);
    }
    // one atomic per distinct (job, bin) and per distinct job in the warp
    const unsigned pk = __match_any_sync(kFull, (j << 3) | (bin & 7));
    if (bin >= 0 && lane == __ffs(pk) - 1) atomicAdd(&cnt_out[9 * j + bin], (unsigned)__popc(pk));
    const unsigned pj = __match_any_sync(kFull, j);
    // (at most 32 degrees of one graph: below 2^32, as a graph has at most 2^31 entries)
    const unsigned long long dsum = __reduce_add_sync(pj, (unsigned)d);
    if (j >= 0 && lane == __ffs(pj) - 1 && dsum) atomicAdd(&ent_out[j], dsum);
    if (bin == 6) {  // hub: table slots hub_cap(d); per job the largest table and their sum
      const unsigned long long cap = (unsigned long long)hub_cap(d);
      atomicMax(&hub_out[3 * j], cap);
      atomicAdd(&hub_out[3 * j + 1], cap);
    }
    if (d > kWideDeg) atomicAdd(&hub_out[3 * j + 2], 1ull);  // vertices that need the larger tables
  }
  if (local) {
    __syncthreads();
    for (int t = threadIdx.x; t < 9 * njobs; t += blockDim.x)
      if (s_counts[t]) atomicAdd(&counts[t], s_counts[t]);
    for (int t = threadIdx.x; t < njobs; t += blockDim.x)
      if (s_entries[t]) atomicAdd(&entries[t], s_entries[t]);
    for (int t = threadIdx.x; t < 3 * njobs; t += blockDim.x) {
      if (!s_hub[t]) continue;
      if (t % 3) atomicAdd(&hubstat[t], s_hub[t]);
      else atomicMax(&hubstat[t], s_hub[t]);
    }
  }
}

// Hub indices and kept-table bases of one LP problem: every vertex above deg_cta gets an index and a
// table of `cap` slots (2 min(d, nl) rounded up to 64, or nl for dense tables) at a base taken from a
// counter (the layout depends on the schedule; results do not). Indices or slots beyond what the launch
// allocated (against the degree classes' counts) are recorded as an internal error.
__global__ void k_hub_index(DGraph g, int64_t vbase, int deg_cta, int64_t nl, int dense, int nhub, int64_t slots,
                            int32_t *hub_id, int64_t *pbase, int64_t *pcap, unsigned long long *next,
                            LpCounters *ctr) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = g.row_begin(v + 1) - g.row_begin(v);
    int h = -1;
    if (d > deg_cta) {
      const int64_t cap = dense ? nl : min(hub_cap(d), hub_cap(nl));
      const unsigned long long x = atomicAdd(&next[0], 1ull);
      const unsigned long long b = atomicAdd(&next[1], (unsigned long long)cap);
      if (x < (unsigned long long)nhub && (int64_t)b + cap <= slots) {
        h = (int)x;
        pbase[h] = (int64_t)b;
        pcap[h] = cap;
      } else {
        table_full(ctr, 7);
      }
    }
    hub_id[vbase + v] = h;
  }
}

constexpr int kSmallK = 2048;

__global__ void k_block_weights(DGraph g, const int32_t *part, int64_t k, int64_t *bw, int *bad) {
  __shared__ unsigned long long sbw[kSmallK];
  const bool small = k <= kSmallK;
  if (small) {
    for (int b = threadIdx.x; b < k; b += blockDim.x) sbw[b] = 0;
    __syncthreads();
  }
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int b = part[v];
    if (b < 0 || b >= k) {
      if (bad) atomicExch(bad, 1);
      continue;
    }
    if (small) atomicAdd(&sbw[b], (unsigned long long)g.vweight(v));
    else atomicAdd(reinterpret_cast<unsigned long long *>(&bw[b]), (unsigned long long)g.vweight(v));
  }
  if (small) {
    __syncthreads();
    for (int b = threadIdx.x; b < k; b += blockDim.x)
      if (sbw[b]) atomicAdd(reinterpret_cast<unsigned long long *>(&bw[b]), sbw[b]);
  }
}

template <int EW, int TB>
int max_coop_blocks(int *out) {
  static int cached[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (!cached[EW][TB]) {
    GP_CUDA(cudaFuncSetAttribute(k_lp<EW, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmemT<TB>));
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lp<EW, TB>, kThreads, kDynSmemT<TB>));
    cached[EW][TB] = std::max(1, per_sm);
  }
  *out = cached[EW][TB] * num_sms();
  return GP_OK;
}

template <int TB>
int coop_capacity_tb(int ew, int *out) {
  return ew == 0 ? max_coop_blocks<0, TB>(out) : ew == 1 ? max_coop_blocks<1, TB>(out) : max_coop_blocks<2, TB>(out);
}

int coop_capacity(int ew, int tb, int *out) {
  return tb == 0 ? coop_capacity_tb<0>(ew, out) : tb == 1 ? coop_capacity_tb<1>(ew, out) : coop_capacity_tb<2>(ew, out);
}

template <int EW, int TB>
int launch_lp(const LpProblem *probs_dev, const int *blk_start_dev, const int *blk_list_dev, int grid, cudaStream_t s) {
  count_launch();
  void *args[] = {(void *)&probs_dev, (void *)&blk_start_dev, (void *)&blk_list_dev};
  GP_CUDA(cudaLaunchCooperativeKernel((void *)k_lp<EW, TB>, grid, kThreads, args, kDynSmemT<TB>, s));
  return GP_OK;
}

template <int TB>
int launch_lp_tb(int ew, const LpProblem *p, const int *bs, const int *bl, int grid, cudaStream_t s) {
  return ew == 0 ? launch_lp<0, TB>(p, bs, bl, grid, s) : ew == 1 ? launch_lp<1, TB>(p, bs, bl, grid, s)
                                                                  : launch_lp<2, TB>(p, bs, bl, grid, s);
}

}  // namespace

LpConfig lp_config_from(const gp_params *p) {
  LpConfig c;
  if (p) {
    if (p->deg_warp > 0) c.deg_warp = (int)p->deg_warp;
    if (p->deg_cta > 0) c.deg_cta = (int)p->deg_cta;
  }
  c.deg_warp = std::max(32, std::min(c.deg_warp, kWarpCap / 2));
  c.deg_cta = std::max(c.deg_warp, std::min(c.deg_cta, kCtaCap / 2));
  if (p && p->hub_batch_slots > 0) c.hub_batch_slots = p->hub_batch_slots;
  if (p && p->verts_per_block > 0) c.verts_per_block = p->verts_per_block;
  if (p && p->hub_keep_slots != 0) c.hub_keep_slots = std::max<int64_t>(0, p->hub_keep_slots);
  c.hub_keep_pct = std::max(1, std::min(c.hub_keep_pct, 95));
  c.hub_batch_slots = std::max<int64_t>(kMinHubBatchSlots, std::min<int64_t>(c.hub_batch_slots, kMaxHubBatchSlots));
  c.verts_per_block = std::max<int64_t>(kMinVertsPerBlock, std::min<int64_t>(c.verts_per_block, kMaxVertsPerBlock));
  return c;
}

int block_weights(const DGraph &g, const int32_t *part, int64_t k, int64_t *bw, int *bad_dev, cudaStream_t s) {
  GP_CUDA(cudaMemsetAsync(bw, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(k, 1), s));
  if (g.n == 0) return GP_OK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, num_sms() * 4));
  (::gp::count_launch(), k_block_weights<<<grid, 256, 0, s>>>(g, part, k, bw, bad_dev));
  GP_LAUNCH_CHECK();
  return GP_OK;
}

// Statistics, error flags and profile entries of n counter blocks (host copies). vb/eb: algorithmic
// bytes per visit and per scanned entry of each job; stats: NULL or per-job outputs; edges/moves:
// NULL or summed totals.
// Algorithmic bytes per proposed move: the label write (4), the label-weight update (8) and the
// admission key, written and read (16).
constexpr int64_t kMoverBytes = 28;

static int account_counters(const LpCounters *hc, int n, const int64_t *vb, const int64_t *eb, gp_lp_stats *const *stats,
                            int64_t *edges_sum, int64_t *moves_sum, const char *const *jnames) {
  int64_t tot_edges = 0, tot_moves = 0;
  for (int j = 0; j < n; j++) {
    const LpCounters &h = hc[j];
    if (h.err == GP_ERR_INTERNAL) {
      set_error("label propagation: a table filled up (site " + std::to_string(h.pad) + ")");
      return GP_ERR_INTERNAL;
    }
    if (h.err) {
      set_error("label propagation: a bounded device barrier gave up");
      return GP_ERR_TIMEOUT;
    }
    int64_t vis = 0, edg = 0;
    for (int b = 0; b < 8; b++) {
      vis += (int64_t)h.bin_visits[b];
      edg += (int64_t)h.bin_edges[b];
    }
    // algorithmic bytes: per visit two offsets, own label, own weight, one label-weight read (4);
    // per scanned entry: adjacency, neighbour label, edge weight (and score); per proposed move its
    // label write, weight update and admission key
    prof_add_counts(jnames ? jnames[j] : "lp_persistent", vis, edg,
                    vis * vb[j] + edg * eb[j] + (int64_t)h.movers * kMoverBytes);
    tot_edges += edg;
    tot_moves += (int64_t)h.moves;
    if (stats && stats[j]) {
      stats[j]->rounds = (int64_t)h.rounds;
      stats[j]->moves = (int64_t)h.moves;
      stats[j]->movers = (int64_t)h.movers;
      stats[j]->visits = vis;
      stats[j]->edges = edg;
    }
  }
  if (edges_sum) *edges_sum = tot_edges;
  if (moves_sum) *moves_sum = tot_moves;
  if (profiling()) {
    // phase times of refinement calls are kept apart (names with "_refine")
    static const char *names[2][8] = {
        {"lp_phase_classify", "lp_phase_choose", "lp_phase_hub_accum", "lp_phase_admit", "lp_phase_contest",
         "lp_phase_final", "lp_phase_hub_choose", "lp_phase_hub_prefix"},
        {"lp_phase_classify_refine", "lp_phase_choose_refine", "lp_phase_hub_accum_refine", "lp_phase_admit_refine",
         "lp_phase_contest_refine", "lp_phase_final_refine", "lp_phase_hub_choose_refine",
         "lp_phase_hub_prefix_refine"}};
    for (int r = 0; r < 2; r++)
      for (int ph = 0; ph < 8; ph++) {
        double ms = 0;
        bool any = false;
        for (int j = 0; j < n; j++) {
          const bool is_refine = jnames && std::strcmp(jnames[j], "lp_persistent_refine") == 0;
          if (is_refine != (r == 1)) continue;
          ms += hc[j].phase_ns[ph] * 1e-6;
          any = true;
        }
        if (any) prof_add_time(names[r][ph], ms);
      }
    double cs = 0, cp = 0, cl = 0, cli = 0, he = 0, hs = 0;
    for (int j = 0; j < n; j++) {
      cs += hc[j].contest_small;
      cp += hc[j].contest_packed;
      cl += hc[j].contest_large;
      cli += hc[j].contest_large_items;
      he += hc[j].hub_entries;
      hs += hc[j].hub_slots;
    }
    prof_add_counts("lp_contest_small_calls", (int64_t)cs, 0, 0);
    prof_add_counts("lp_contest_packed_calls", (int64_t)cp, 0, 0);
    prof_add_counts("lp_contest_large_calls", (int64_t)cl, (int64_t)cli, 0);  // edges: contested movers
    prof_add_counts("lp_hub_work", (int64_t)hs, (int64_t)he, 0);  // items: table slots, edges: entries
    double hb = 0, hst = 0;
    for (int j = 0; j < n; j++) {
      hb += hc[j].hub_built_entries;
      hst += hc[j].hub_stale;
    }
    // items: kept tables gone stale, edges: hub entries accumulated (the rest followed the moves)
    prof_add_counts("lp_hub_built", (int64_t)hst, (int64_t)hb, 0);
  }
  return GP_OK;
}

size_t lp_counters_bytes() { return sizeof(LpCounters); }

int lp_classes_launch(const DGraph &g, const LpConfig &cfg, unsigned long long *words_dev, Workspace &ws) {
  cudaStream_t s = ws.stream();
  GP_CUDA(cudaMemsetAsync(words_dev, 0, sizeof(unsigned long long) * kLpClassWords, s));
  if (g.n <= 0) return GP_OK;
  DGraph *gs_dev;
  int64_t *pre_dev;
  GP_TRY(ws.get(&gs_dev, 1));
  GP_TRY(ws.get(&pre_dev, 2));
  const int64_t pre[2] = {0, g.n};
  GP_CUDA(cudaMemcpyAsync(gs_dev, &g, sizeof(DGraph), cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemcpyAsync(pre_dev, pre, sizeof(pre), cudaMemcpyHostToDevice, s));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, num_sms() * 8));
  // words: [0, 5) the 9 unsigned class counts, [5] entries, [6, 9) hub statistics and wide vertices
  (::gp::count_launch(), k_degree_classes<<<grid, 256, 0, s>>>(gs_dev, pre_dev, 1, cfg.deg_warp, cfg.deg_cta,
                                                                 reinterpret_cast<unsigned *>(words_dev),
                                                                 words_dev + 5, words_dev + 6));
  GP_LAUNCH_CHECK();
  return GP_OK;
}

void lp_classes_from(const unsigned long long *words, const LpConfig &cfg, LpClassInfo *ci) {
  const unsigned *cls = reinterpret_cast<const unsigned *>(words);
  ci->valid = true;
  ci->deg_warp = cfg.deg_warp;
  ci->deg_cta = cfg.deg_cta;
  for (int b = 0; b < 9; b++) ci->cls[b] = cls[b];
  ci->entries = words[5];
  ci->hub_max_cap = words[6];
  ci->hub_cap_sum = words[7];
  ci->wide = words[8];
}

int lp_collect(LpDeferred &def, cudaStream_t s, int64_t *edges, int64_t *moves, Readback *extra) {
  if (edges) *edges = 0;
  if (moves) *moves = 0;
  Readback local;
  Readback &rb = extra ? *extra : local;
  std::vector<LpCounters> hc(def.count);
  if (def.count) rb.add(hc.data(), def.dev, sizeof(LpCounters) * def.count);
  GP_TRY(rb.run(s));
  if (def.count == 0) return GP_OK;
  const int st = account_counters(hc.data(), def.count, def.visit_bytes.data(), def.entry_bytes.data(), nullptr, edges,
                                  moves, def.names.data());
  def.count = 0;
  def.visit_bytes.clear();
  def.entry_bytes.clear();
  def.names.clear();
  return st;
}

// Several independent LP runs in one cooperative launch (same edge-weight type and score use).
int run_lp_multi(const LpJob *jobs, int njobs, cudaStream_t s, const LpConfig &cfg_in, LpDeferred *deferred) {
  if (njobs <= 0) return GP_OK;
  const int ew = jobs[0].g.ew_mode();
  const bool lq = jobs[0].q != nullptr;
  // scored runs have the smaller shared-memory tables (16-byte slots)
  LpConfig cfg = cfg_in;
  if (lq) {
    cfg.deg_warp = std::min(cfg.deg_warp, kWarpCapT<0> / 2);
    cfg.deg_cta = std::max(cfg.deg_warp, std::min(cfg.deg_cta, kCtaCapT<0> / 2));
  }
  for (int j = 0; j < njobs; j++) {
    if (jobs[j].stats) std::memset(jobs[j].stats, 0, sizeof(gp_lp_stats));
    if (jobs[j].g.ew_mode() != ew || (jobs[j].q != nullptr) != lq) {
      set_error("run_lp_multi: jobs of one launch must share weight type and score use");
      return GP_ERR_INTERNAL;
    }
    if (jobs[j].g.n >= (int64_t)1 << 31 || jobs[j].nl >= (int64_t)1 << 31) {
      set_error("label propagation supports n < 2^31");
      return GP_ERR_UNSUPPORTED;
    }
  }
  Workspace ws(s);
  const int nsm = num_sms();
  // degree classes and entry counts of all jobs (one kernel, one copy back), unless every job brings
  // them from an earlier call on the same graph and schedule
  std::vector<unsigned> hcls(9 * (size_t)njobs);
  std::vector<unsigned long long> hent(njobs);
  std::vector<unsigned long long> hhub(3 * (size_t)njobs);
  bool cached = true;
  for (int j = 0; j < njobs; j++) {
    const LpClassInfo *ci = jobs[j].classes;
    cached = cached && ci && ci->valid && ci->deg_warp == cfg.deg_warp && ci->deg_cta == cfg.deg_cta;
  }
  if (cached) {
    for (int j = 0; j < njobs; j++) {
      const LpClassInfo &ci = *jobs[j].classes;
      for (int b = 0; b < 9; b++) hcls[9 * (size_t)j + b] = ci.cls[b];
      hent[j] = ci.entries;
      hhub[3 * (size_t)j] = ci.hub_max_cap;
      hhub[3 * (size_t)j + 1] = ci.hub_cap_sum;
      hhub[3 * (size_t)j + 2] = ci.wide;
    }
  } else {
    std::vector<DGraph> hg(njobs);
    std::vector<int64_t> pre(njobs + 1, 0);
    for (int j = 0; j < njobs; j++) {
      hg[j] = jobs[j].g;
      pre[j + 1] = pre[j] + jobs[j].g.n;
    }
    DGraph *gs_dev;
    int64_t *pre_dev;
    unsigned *classes;
    unsigned long long *entries;
    GP_TRY(ws.get(&gs_dev, (size_t)njobs));
    GP_TRY(ws.get(&pre_dev, (size_t)njobs + 1));
    GP_TRY(ws.zeros(&classes, (size_t)9 * njobs));
    GP_TRY(ws.zeros(&entries, (size_t)njobs));
    unsigned long long *hubstat;
    GP_TRY(ws.zeros(&hubstat, (size_t)3 * njobs));
    GP_CUDA(cudaMemcpyAsync(gs_dev, hg.data(), sizeof(DGraph) * njobs, cudaMemcpyHostToDevice, s));
    GP_CUDA(cudaMemcpyAsync(pre_dev, pre.data(), sizeof(int64_t) * (njobs + 1), cudaMemcpyHostToDevice, s));
    if (pre[njobs] > 0) {
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((pre[njobs] + 255) / 256, nsm * 8));
      (::gp::count_launch(), k_degree_classes<<<grid, 256, 0, s>>>(gs_dev, pre_dev, njobs, cfg.deg_warp, cfg.deg_cta,
                                                                       classes, entries, hubstat));
      GP_LAUNCH_CHECK();
    }
    Readback rb;
    rb.add(hcls.data(), classes, sizeof(unsigned) * hcls.size());
    rb.add(hent.data(), entries, sizeof(unsigned long long) * njobs);
    rb.add(hhub.data(), hubstat, sizeof(unsigned long long) * hhub.size());
    GP_TRY(rb.run(s));
    for (int j = 0; j < njobs; j++) {
      LpClassInfo *ci = jobs[j].classes;
      if (!ci) continue;
      ci->valid = true;
      ci->deg_warp = cfg.deg_warp;
      ci->deg_cta = cfg.deg_cta;
      for (int b = 0; b < 9; b++) ci->cls[b] = hcls[9 * (size_t)j + b];
      ci->entries = hent[j];
      ci->hub_max_cap = hhub[3 * (size_t)j];
      ci->hub_cap_sum = hhub[3 * (size_t)j + 1];
      ci->wide = hhub[3 * (size_t)j + 2];
    }
  }
  // table class: scored runs 0; plain runs the larger tables only where a vertex of degree above
  // kWideDeg (or a warp bin above 128) needs them. Without such vertices the classes computed for
  // deg_cta up to 2048 are those of deg_cta = 1024 as well.
  bool wide = cfg.deg_warp > kWarpCapT<1> / 2;
  for (int j = 0; j < njobs; j++) wide = wide || hhub[3 * (size_t)j + 2] > 0;
  const int tb = lq ? 0 : (wide ? 2 : 1);
  if (tb == 1) cfg.deg_cta = std::max(cfg.deg_warp, std::min(cfg.deg_cta, kCtaCapT<1> / 2));
  int cap_blocks = 0;
  GP_TRY(coop_capacity(ew, tb, &cap_blocks));
  // Blocks: a job gets at most one block per cfg.verts_per_block vertices. When all jobs fit the co-resident
  // capacity that way, they do; otherwise work is balanced by a cost model (entries + 4 per vertex
  // + a fixed per-problem latency term): jobs above twice the mean block load get several blocks,
  // the rest run one block each, packed onto the remaining blocks longest first.
  std::vector<int64_t> useful(njobs);
  int64_t sum_useful = 0;
  for (int j = 0; j < njobs; j++) {
    // (the large contest stages 32 bytes per block of a problem in the dynamic shared memory)
    useful[j] = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(cap_blocks, (int64_t)(kDynSmem / 32)),
                                                       (jobs[j].g.n + cfg.verts_per_block - 1) / cfg.verts_per_block));
    sum_useful += useful[j];
  }
  std::vector<int> nblk(njobs, 1), home(njobs, -1);
  std::vector<std::vector<int>> packed;
  if (sum_useful <= cap_blocks) {
    for (int j = 0; j < njobs; j++) nblk[j] = (int)useful[j];
  } else {
    constexpr double kProblemCost = 65536.0;
    std::vector<double> cost(njobs);
    double total = 0;
    for (int j = 0; j < njobs; j++) {
      cost[j] = (double)hent[j] + 4.0 * (double)jobs[j].g.n + kProblemCost;
      total += cost[j];
    }
    const double wstar = total / cap_blocks;
    int64_t multi = 0;
    for (int j = 0; j < njobs; j++)
      if (cost[j] > 2 * wstar) {
        nblk[j] = (int)std::min<int64_t>(useful[j], std::max<int64_t>(2, (int64_t)(cost[j] / wstar)));
        multi += nblk[j];
      }
    int nsingle = 0;
    for (int j = 0; j < njobs; j++) nsingle += nblk[j] == 1 ? 1 : 0;
    const int64_t want_single = nsingle ? std::max<int64_t>(1, cap_blocks / 8) : 0;
    if (multi + want_single > cap_blocks) {
      // shrink the multi-block jobs proportionally
      const double f = (double)(cap_blocks - want_single) / (double)multi;
      multi = 0;
      for (int j = 0; j < njobs; j++)
        if (nblk[j] > 1) {
          nblk[j] = std::max(1, (int)(nblk[j] * f));
          multi += nblk[j];
        }
    }
    nsingle = 0;
    for (int j = 0; j < njobs; j++) nsingle += nblk[j] == 1 ? 1 : 0;
    const int nb_single = (int)std::min<int64_t>(nsingle, cap_blocks - multi);
    packed.assign(nb_single, {});
    std::vector<int> order;
    for (int j = 0; j < njobs; j++)
      if (nblk[j] == 1) order.push_back(j);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y] || (cost[x] == cost[y] && x < y); });
    std::vector<double> load(nb_single, 0.0);
    for (int j : order) {
      int best = 0;
      for (int b = 1; b < nb_single; b++)
        if (load[b] < load[best]) best = b;
      load[best] += cost[j];
      packed[best].push_back(j);
      home[j] = best;
    }
  }
  // block lists: multi-block (and, without packing, all) jobs first, then the packed blocks
  std::vector<int> blk_start{0}, blk_list;
  std::vector<int> first_block(njobs, -1);
  for (int j = 0; j < njobs; j++) {
    if (home[j] >= 0) continue;
    first_block[j] = (int)blk_start.size() - 1;
    for (int b = 0; b < nblk[j]; b++) {
      blk_list.push_back(j);
      blk_start.push_back((int)blk_list.size());
    }
  }
  for (auto &pb : packed) {
    const int blk = (int)blk_start.size() - 1;
    for (int j : pb) {
      first_block[j] = blk;
      blk_list.push_back(j);
    }
    blk_start.push_back((int)blk_list.size());
  }
  const int grid = (int)blk_start.size() - 1;
  if (grid > cap_blocks) {
    set_error("run_lp_multi: block assignment exceeds the co-resident capacity");
    return GP_ERR_INTERNAL;
  }
  std::vector<LpProblem> hp(njobs);
  LpCounters *ctr_all;
  unsigned *bar_all;
  GP_TRY(ws.zeros(&ctr_all, (size_t)njobs));
  GP_TRY(ws.zeros(&bar_all, (size_t)njobs * kBarrierStride));
  unsigned *binres_all;
  GP_TRY(ws.zeros(&binres_all, (size_t)njobs * 3 * 256));
  // every job's demand array in one zeroed allocation (one memset for the launch, not one per job)
  int64_t *demand_all;
  {
    size_t total = 0;
    for (int j = 0; j < njobs; j++) total += (size_t)std::max<int64_t>(jobs[j].nl, 1);
    GP_TRY(ws.zeros(&demand_all, total));
  }
  size_t demand_off = 0;
  int64_t keep_total = 0;  // slots of the kept hub tables of the launch
  for (int j = 0; j < njobs; j++) {
    const LpJob &jb = jobs[j];
    LpProblem &P = hp[j];
    std::memset(&P, 0, sizeof(P));
    P.g = jb.g;
    P.vbase = jb.vbase;
    P.lbase = jb.lbase;
    P.nl = jb.nl;
    P.U = jb.U;
    P.hub_batch_slots = cfg.hub_batch_slots;
    P.hub_chunk = kHubChunkT<0>;
    P.hub_chunk_shift = 10;
    static_assert(kHubChunkT<0> == 1 << 10 && kHubChunkT<1> == 1 << 10 && kHubChunkT<2> == 1 << 10,
                  "hub chunks are powers of two");
    P.wait_us = (unsigned)std::min<unsigned long long>(std::max<unsigned long long>(wait_limit_ns() / 1000, 0),
                                                        0xffffffffull);
    P.smix = mix64(jb.seed);
    P.rounds = jb.g.n > 0 ? jb.rounds : 0;
    P.singletons = jb.singletons ? 1 : 0;
    P.deg_warp = cfg.deg_warp;
    P.deg_cta = cfg.deg_cta;
    P.labels = jb.labels;
    P.lw = jb.lw;
    P.q = jb.q;
    P.block_begin = first_block[j];
    P.block_count = nblk[j];
    const size_t n = (size_t)std::max<int64_t>(jb.g.n, 1);
    int64_t slots_total = 0;
    for (int b = 0; b < kBins; b++) {
      GP_TRY(ws.get(&P.bin[b], (size_t)std::max<unsigned>(hcls[9 * j + b], 1)));
      if (b < 4) GP_TRY(ws.get(&P.binx[b], (size_t)std::max<unsigned>(hcls[9 * j + b], 1)));
      P.bin_base[b] = slots_total;
      slots_total += hcls[9 * j + b];
    }
    GP_TRY(ws.get(&P.mv_v, n));
    GP_TRY(ws.get(&P.mv_t, n));
    GP_TRY(ws.get(&P.mv_from, n));
    GP_TRY(ws.get(&P.mv_gain, n));
    GP_TRY(ws.get(&P.mv_q, n));
    GP_TRY(ws.get(&P.mv_adm, n));
    GP_TRY(ws.get(&P.mv_of_v, n));
    P.demand = demand_all + demand_off - jb.lbase;  // indexed by global label
    demand_off += (size_t)std::max<int64_t>(jb.nl, 1);
    GP_TRY(ws.get(&P.ct, n));
    GP_TRY(ws.get(&P.ct2, n));
    GP_TRY(ws.get(&P.ck, n));
    GP_TRY(ws.get(&P.ck2, n));
    // marking items: at most one per kBigChunkKept entries of every row plus one per vertex above kBigDegKept
    // (all of them in bins 4-6, which start above 32)
    static_assert(kBigDegKept >= 32, "big movers lie in the warp, CTA and hub bins");
    static_assert(kBigChunkKept <= kBigChunk, "the kept-table items bound the others");
    GP_TRY(ws.get(&P.big,
                  (size_t)(hent[j] / kBigChunkKept + hcls[9 * j + 4] + hcls[9 * j + 5] + hcls[9 * j + 6] + 1)));
    GP_TRY(ws.get(&P.act[0], n));
    GP_TRY(ws.get(&P.act[1], n));
    P.act[0] -= jb.vbase;  // indexed by global vertex id
    P.act[1] -= jb.vbase;
    GP_TRY(ws.get(&P.hist, (size_t)nblk[j] * 256 + 16));
    GP_TRY(ws.get(&P.hoff, (size_t)nblk[j] * 256 + 256 + 16));
    P.ctr = ctr_all + j;
    P.binres = binres_all + (size_t)j * 3 * 256;
    P.bar = bar_all + (size_t)j * kBarrierStride;
    const unsigned nhub = hcls[9 * j + 6];
    if (nhub) {
      // dense tables need nl <= 2 (deg_cta + 1) <= hub_cap(d) for every hub (the tables are sized by
      // hub_cap(d)) and the counters in the CTA's shared table
      // (the counters take the value half of the 2048-slot shared table)
      P.hub_dense = (!lq && jb.nl <= 2 * ((int64_t)cfg.deg_cta + 1) && jb.nl <= kHubCap) ? 1 : 0;
      // tables of one batch of hubs (reused batch after batch), or of every hub when they are kept,
      // partial choices, per-hub arrays
      const int64_t max_cap = (int64_t)hhub[3 * (size_t)j], cap_sum = (int64_t)hhub[3 * (size_t)j + 1];
      const int64_t keep_need = P.hub_dense ? (int64_t)nhub * jb.nl : cap_sum;
      const bool keep = cfg.hub_keep_slots > 0 && keep_total + keep_need <= cfg.hub_keep_slots;
      if (keep) keep_total += keep_need;
      // (kept dense tables take nl slots per hub; hashed ones at most hub_cap(d))
      const int64_t slots = keep ? std::max<int64_t>(keep_need, 1)
                                 : std::min<int64_t>(cfg.hub_batch_slots, cap_sum) + max_cap;
      P.hub_table_slots = slots;
      // items of one batch: at most slots / kSlotChunk full items plus one partial item per hub; the
      // round-0 direct path keeps one item per chunk of every hub row
      const int64_t items = std::max<int64_t>(slots / kSlotChunk, (int64_t)(hent[j] / kHubChunk)) + (int64_t)nhub + 16;
      GP_TRY(ws.get(&P.hub_keys, (size_t)slots));
      GP_CUDA(cudaMemsetAsync(P.hub_keys, 0xff, sizeof(int32_t) * (size_t)slots, s));
      GP_TRY(ws.zeros(&P.hub_vals, (size_t)slots));
      if (lq) GP_TRY(ws.zeros(&P.hub_qv, (size_t)slots));
      GP_TRY(ws.get(&P.hub_part, (size_t)items * sizeof(Best)));
      GP_TRY(ws.get(&P.hub_c0, (size_t)nhub));
      GP_TRY(ws.get(&P.hub_prefix, (size_t)nhub + 1));
      GP_TRY(ws.get(&P.hub_capx, (size_t)nhub + 1));
      GP_TRY(ws.get(&P.hub_scx, (size_t)nhub + 1));
      GP_TRY(ws.get(&P.hub_tb, (size_t)nhub));
      GP_TRY(ws.get(&P.hub_bstart, (size_t)nhub + 1));
      GP_TRY(ws.get(&P.hub_bbase, (size_t)nhub + 1));
      P.has_hubs = 1;
      if (keep) {
        P.hub_keep = 1;
        P.hub_keep_pct = cfg.hub_keep_pct;
        P.hub_n = (int)nhub;
        GP_TRY(ws.get(&P.hub_id, n));
        P.hub_id -= jb.vbase;  // indexed by global vertex id
        GP_TRY(ws.get(&P.hub_pbase, (size_t)nhub));
        GP_TRY(ws.get(&P.hub_pcap, (size_t)nhub));
        GP_TRY(ws.zeros(&P.hub_keycnt, (size_t)nhub));
        GP_TRY(ws.zeros(&P.hub_valid, (size_t)nhub));
        GP_TRY(ws.get(&P.hub_inval, (size_t)nhub));
        unsigned long long *next;
        GP_TRY(ws.zeros(&next, 2));
        const int grid_h = (int)std::max<int64_t>(1, std::min<int64_t>((jb.g.n + 255) / 256, (int64_t)nsm * 8));
        (::gp::count_launch(), k_hub_index<<<grid_h, 256, 0, s>>>(jb.g, jb.vbase, cfg.deg_cta, jb.nl, P.hub_dense,
                                                                    (int)nhub, slots, P.hub_id, P.hub_pbase,
                                                                    P.hub_pcap, next, P.ctr));
        GP_LAUNCH_CHECK();
      }
    }
  }
  LpProblem *probs_dev;
  int *bs_dev, *bl_dev;
  GP_TRY(ws.get(&probs_dev, hp.size()));
  GP_TRY(ws.get(&bs_dev, blk_start.size()));
  GP_TRY(ws.get(&bl_dev, blk_list.size()));
  GP_CUDA(cudaMemcpyAsync(probs_dev, hp.data(), sizeof(LpProblem) * hp.size(), cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemcpyAsync(bs_dev, blk_start.data(), sizeof(int) * blk_start.size(), cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemcpyAsync(bl_dev, blk_list.data(), sizeof(int) * blk_list.size(), cudaMemcpyHostToDevice, s));
  {
    ProfScope ps(jobs[0].prof, s);
    int st;
    if (tb == 0) st = launch_lp_tb<0>(ew, probs_dev, bs_dev, bl_dev, grid, s);
    else if (tb == 1) st = launch_lp_tb<1>(ew, probs_dev, bs_dev, bl_dev, grid, s);
    else st = launch_lp_tb<2>(ew, probs_dev, bs_dev, bl_dev, grid, s);
    GP_TRY(st);
  }
  if (deferred) {
    // keep the counters on the device for lp_collect
    if (deferred->count + njobs > deferred->capacity) {
      set_error("run_lp_multi: deferred counter buffer is full");
      return GP_ERR_INTERNAL;
    }
    GP_CUDA(cudaMemcpyAsync(static_cast<LpCounters *>(deferred->dev) + deferred->count, ctr_all,
                            sizeof(LpCounters) * njobs, cudaMemcpyDeviceToDevice, s));
    deferred->count += njobs;
    for (int j = 0; j < njobs; j++) {
      const DGraph &g = jobs[j].g;
      deferred->visit_bytes.push_back(2 * g.offset_bytes() + 4 + g.vw_bytes() + 4);
      deferred->entry_bytes.push_back(8 + g.ew_bytes() + (jobs[j].q ? 4 : 0));
      deferred->names.push_back(jobs[j].prof);
    }
    return GP_OK;
  }
  std::vector<LpCounters> hc(njobs);
  GP_CUDA(cudaMemcpyAsync(hc.data(), ctr_all, sizeof(LpCounters) * njobs, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> vb(njobs), eb(njobs);
  for (int j = 0; j < njobs; j++) {
    const DGraph &g = jobs[j].g;
    vb[j] = 2 * g.offset_bytes() + 4 + g.vw_bytes() + 4;
    eb[j] = 8 + g.ew_bytes() + (jobs[j].q ? 4 : 0);
  }
  std::vector<gp_lp_stats *> st(njobs);
  std::vector<const char *> names(njobs);
  for (int j = 0; j < njobs; j++) {
    st[j] = jobs[j].stats;
    names[j] = jobs[j].prof;
  }
  return account_counters(hc.data(), njobs, vb.data(), eb.data(), st.data(), nullptr, nullptr, names.data());
}

int run_lp(const DGraph &g, const int32_t *q, int32_t *labels, int64_t *lw, int64_t nl, int64_t U, int rounds,
           uint64_t seed, gp_lp_stats *stats, cudaStream_t s, const LpConfig &cfg, bool singletons,
           LpClassInfo *classes, LpDeferred *deferred, const char *prof) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (g.n == 0 || rounds <= 0) return GP_OK;
  LpJob j;
  j.g = g;
  j.q = q;
  j.labels = labels;
  j.lw = lw;
  j.nl = nl;
  j.U = U;
  j.rounds = rounds;
  j.seed = seed;
  j.stats = stats;
  j.singletons = singletons;
  j.classes = classes;
  j.prof = prof;
  return run_lp_multi(&j, 1, s, cfg, deferred);
}

}  // namespace gp
