// Register kernel: the chunked sketch with its FP32 accumulator in registers.
//
// Paper Sec. 4.1 (every element of A is added, with its sign, into its k target rows, Listing 1),
// with the chunked FP32 pre-combine of the tile kernel: the partial sums of a work item are added
// into the per-chunk FP32 totals P, and the chunk-finish kernel scales, rounds (Sec. 4.2) and adds
// the chunk totals into Y in chunk order.
//
// Why registers. One input row feeds k target rows, so a scatter kernel makes k*n updates per row of
// A (2 updates per byte at k = 8). A shared-memory FP32 reduction has no native instruction on this
// GPU (a load / add / compare-and-swap loop), so the tile kernel is bounded by that sequence. Here the
// accumulator lives in registers, where an update is one fused add, and shared memory only carries
// the rows of A to the threads that own their targets.
//
// Work item: rows [r0, r1) of chunk t (all of it or a slice), 32 columns [32g, 32g+32) and a target
// group of kRegTargets = 1024 consecutive output rows [tr0, tr0 + 1024) (the rows of one or more
// blocks of S, or part of one block). Thread i owns output row tr0 + i: its 32 columns sit in 32
// registers.
//
// The rows are staged in boxes of up to 768 rows x 32 columns (double-buffered TMA copies). Per box:
//   1. hash: each row's SplitMix64 outputs give its target row in every block of the group (the same
//      generator as every other kernel); a shared-memory counter per target row (native integer
//      atomic) hands out a slot in that row's list of 16-bit (row of the box, sign) entries;
//   2. accumulate: every thread walks its own list; for an entry it reads the row's 128 bytes with
//      eight 16-byte loads and adds them, signed, with packed FP32 FMAs. Lane l reads the row's
//      16-byte chunks in the order q XOR (l mod 8), q = 0..7, so at every step the 8 lanes of a
//      quarter-warp (one shared-memory wavefront for 16-byte loads) hit 8 distinct chunks, hence 8
//      distinct bank groups, whichever rows they read; register group q of lane l therefore holds
//      columns 4(q XOR (l mod 8)) .. +3.
// The hash of a box needs only row indices, not the staged values, so it runs one box ahead: lists,
// list lengths and overflow lists are double-buffered, and box b+1 is hashed in the same phase as
// box b is accumulated (one CTA barrier per box; the hash's integer and atomic latency overlaps the
// other warps' shared-memory loads).
// A list holds `cap` entries, about lambda + 1.5 sqrt(lambda) for lambda = box rows / B, the mean
// number of entries an output row receives per box: longer lists would make every warp wait for its
// longest one. Rows beyond a full list go to an overflow list (sized for every entry a box can
// produce), which the CTA's quarter-warps add into the chunk totals with FP32 vector reductions (one
// 128-byte row per quarter-warp access). At the end of the item every thread adds its 32 sums into P.
//
// All rounding happens in the FP32 additions of the partial sums (any order within the chunk, as in
// the tile kernel's atomic mode) and in the chunk finish; the result is the chunk total of the
// canonical order up to the FP32 summation order inside the chunk.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sk_internal.h"
#include "sk_tile.cuh"

namespace sk {

namespace {

constexpr int kRegThreads = 1024;
constexpr int kRegTargets = kRegThreads;  // output rows per work item: one per thread
constexpr int kRegCopyRows = 128;         // rows per TMA copy (16 KiB)
constexpr int kRegMaxSub = 6;             // TMA copies per staged box (768 rows < kRegThreads: one row per thread)

// A work item, written to shared memory by one thread (two descriptors: the current and the next item).
struct RegItem {
  int64_t r0, r1;                 // global rows
  int32_t tr0, ntr;               // first output row of the group, output rows in it
  int32_t jlo, jhi, plo, np;      // blocks that reach the group, and their 64-bit stream outputs
  int32_t nbox, xcol, ybase, tl;  // boxes, first column, row of A of r0, chunk index (from t_first)
};

// Shared memory (byte offsets): two list-length arrays | 4 overflow counters (by box sequence mod 4) |
// 2 mbarriers | 2 item descriptors (these at fixed offsets) | two staged boxes | two list tables
// (kRegTargets x cap 16-bit entries, slot-major: [slot][output row]) | two overflow lists (ovf_cap
// 32-bit entries: output row << 16 | row of the box | sign << 15).
constexpr uint32_t kRegCnt = 0;
constexpr uint32_t kRegNov = 2u * kRegTargets * 4u;
constexpr uint32_t kRegBar = kRegNov + 16u;
constexpr uint32_t kRegItem = kRegBar + 16u;
constexpr uint32_t kRegStage = (kRegItem + 2u * (uint32_t)sizeof(RegItem) + 127u) & ~127u;

struct RegSmem {
  uint32_t tab, tab_stride, ovf, total;
};

__host__ __device__ inline RegSmem reg_smem(int32_t nsub, int32_t cap, int32_t ovf_cap) {
  RegSmem L;
  L.tab = kRegStage + 2u * (uint32_t)nsub * kRegCopyRows * 128u;
  L.tab_stride = ((uint32_t)kRegTargets * (uint32_t)cap * 2u + 15u) & ~15u;
  L.ovf = L.tab + 2u * L.tab_stride;
  L.total = L.ovf + 2u * (uint32_t)ovf_cap * 4u;
  return L;
}

struct RegGrid {
  TileDesc D;
  int64_t row_begin, row_end;  // global rows processed
  int64_t R;                   // chunk rows
  int64_t t_first;             // first chunk index
  int64_t items;               // chunks * slices * ncg * ntg
  int32_t ncg, ntg, slices;
  int32_t nsub;                // TMA copies per staged box (box = nsub * kRegCopyRows rows)
  int32_t cap;                 // list entries per output row and box
  int32_t ovf_cap;             // overflow-list entries per box
  RegSmem S;                   // shared-memory layout
  float* P;                    // per-chunk FP32 totals, chunk-major, d x n each (zero on entry)
  unsigned* status;            // sticky status word
};

// 16-byte FP32 vector reduction into global memory (P), or per-column atomics where a 16-byte
// access would not be aligned or would pass column n.
__device__ __forceinline__ void red_quad(float* p, int64_t n, int64_t col0, float4 v) {
  if ((n & 3) == 0 && col0 + 3 < n) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
  } else {
    atomicAdd(p, v.x);
    if (col0 + 1 < n) atomicAdd(p + 1, v.y);
    if (col0 + 2 < n) atomicAdd(p + 2, v.z);
    if (col0 + 3 < n) atomicAdd(p + 3, v.w);
  }
}

__device__ __forceinline__ void reg_item(const RegGrid& G, int64_t w, int32_t rbox, RegItem* I) {
  const int32_t tg = (int32_t)(w % G.ntg);
  int64_t rest = w / G.ntg;
  const int32_t g = (int32_t)(rest % G.ncg);
  rest /= G.ncg;
  const int32_t sl = (int32_t)(rest % G.slices);
  const int64_t tl = rest / G.slices;
  const int64_t t = G.t_first + tl;
  const int64_t c0 = max(t * G.R, G.row_begin);
  const int64_t c1 = min((t + 1) * G.R, G.row_end);
  const int64_t r0 = c0 + (c1 - c0) * sl / G.slices;
  const int64_t r1 = c0 + (c1 - c0) * (sl + 1) / G.slices;
  const int64_t B = G.D.B;
  const int64_t d = B * G.D.k;
  const int64_t tr0 = (int64_t)tg * kRegTargets;
  const int64_t ntr = min((int64_t)kRegTargets, d - tr0);
  I->r0 = r0;
  I->r1 = r1;
  I->tr0 = (int32_t)tr0;
  I->ntr = (int32_t)ntr;
  I->jlo = (int32_t)(tr0 / B);
  I->jhi = (int32_t)((tr0 + ntr - 1) / B);
  I->plo = I->jlo >> 1;
  I->np = (I->jhi >> 1) - I->plo + 1;
  I->nbox = (int32_t)((r1 - r0 + rbox - 1) / rbox);
  I->xcol = g * 32;
  I->ybase = (int32_t)(r0 - G.D.row_base);
  I->tl = (int32_t)tl;
}

// Step 1 for box b of the item (box sequence number seq): this thread's row (if the box has it) into
// the lists of buffer seq & 1, or into the overflow list.
template <int NSUB>
__device__ __forceinline__ void reg_hash(const RegGrid& G, const RegItem* I, int32_t b, uint32_t seq,
                                         unsigned char* sm) {
  const int32_t tid = (int32_t)threadIdx.x;
  constexpr int32_t rbox = NSUB * kRegCopyRows;
  const int64_t rb0 = I->r0 + (int64_t)b * rbox;
  if ((int64_t)tid >= I->r1 - rb0 || tid >= rbox) return;
  uint16_t* tab = reinterpret_cast<uint16_t*>(sm + G.S.tab + (seq & 1u) * G.S.tab_stride);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(sm + kRegCnt) + (seq & 1u) * kRegTargets;
  uint32_t* ovf = reinterpret_cast<uint32_t*>(sm + G.S.ovf) + (seq & 1u) * (uint32_t)G.ovf_cap;
  uint32_t* nov = reinterpret_cast<uint32_t*>(sm + kRegNov) + (seq & 3u);
  const uint32_t B = G.D.B;
  const int32_t np = I->np, plo = I->plo, jlo = I->jlo, jhi = I->jhi, tr0 = I->tr0;
  const uint32_t ntr = (uint32_t)I->ntr;
  for (int32_t pr = 0; pr < np; ++pr) {
    const uint32_t p = (uint32_t)(plo + pr);
    const uint64_t h = row_pair_bits(G.D.seed, (uint64_t)(rb0 + tid), G.D.kp, p);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int32_t j = 2 * (int32_t)p + e;
      if (j < jlo || j > jhi) continue;
      const uint32_t wd = e ? (uint32_t)h : (uint32_t)(h >> 32);
      const int32_t tgt = j * (int32_t)B + (int32_t)word_to_slot(wd, B) - tr0;  // d < 2^31
      if ((uint32_t)tgt >= ntr) continue;
      const uint32_t ent = (uint32_t)tid | ((wd & 1u) << 15);
      const uint32_t pos = atomicAdd(cnt + tgt, 1u);
      if (pos < (uint32_t)G.cap) {
        tab[pos * kRegTargets + (uint32_t)tgt] = (uint16_t)ent;
      } else {
        const uint32_t o = atomicAdd(nov, 1u);
        if (o < (uint32_t)G.ovf_cap) ovf[o] = ((uint32_t)tgt << 16) | ent;  // holds every entry of a box
      }
    }
  }
}

// Thread 0: stage box b of the item into buffer buf (arm the buffer's mbarrier with the box's bytes,
// then NSUB 128-row TMA copies). The CTA barrier before the call has ordered every thread's reads of
// the buffer; the proxy fence orders them before the asynchronous writes.
template <int NSUB>
__device__ __forceinline__ void reg_issue_box(const CUtensorMap* tmap, const RegItem* I, int32_t b, int32_t buf,
                                              unsigned char* sm) {
  constexpr uint32_t box_bytes = (uint32_t)NSUB * kRegCopyRows * 128u;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kRegBar) + buf;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, box_bytes);
#pragma unroll
  for (int c = 0; c < NSUB; ++c)
    tma_load_2d(sm + kRegStage + (size_t)buf * box_bytes + (size_t)c * kRegCopyRows * 128, tmap, I->xcol,
                I->ybase + (b * NSUB + c) * kRegCopyRows, bar);
}

// NSUB: TMA copies per staged box (box = NSUB * 128 rows), a compile-time constant so that the box
// layout and the copy issue (on every box's critical path) are fixed.
template <int NSUB>
__global__ void __launch_bounds__(kRegThreads, 1) reg_kernel(const RegGrid G, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int tid = threadIdx.x;
  if (blockDim.x != kRegThreads || G.nsub != NSUB || G.cap < 1 || G.ovf_cap < 0) {
    if (tid == 0 && G.status) atomicOr(G.status, kStatusBounds);
    return;
  }
  constexpr int32_t rbox = NSUB * kRegCopyRows;
  constexpr uint32_t box_bytes = (uint32_t)rbox * 128u;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kRegBar);
  RegItem* items = reinterpret_cast<RegItem*>(sm + kRegItem);
  uint32_t* nov = reinterpret_cast<uint32_t*>(sm + kRegNov);
  if (tid == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    mbar_fence_init();
    reg_item(G, blockIdx.x, rbox, items);
  }
  if (tid < 4) nov[tid] = 0u;
  reinterpret_cast<uint32_t*>(sm + kRegCnt)[tid] = 0u;
  reinterpret_cast<uint32_t*>(sm + kRegCnt)[kRegTargets + tid] = 0u;
  const uint32_t l16 = (uint32_t)(tid & 7) << 4;  // this lane's chunk rotation (bytes), lane mod 8
  // Bit b of `par`: parity of the next phase of buffer b's mbarrier (toggled after every wait; in
  // thread 0 only after a wait that succeeded). Bit b of `pend` (thread 0): a box copied into buffer b
  // has not been seen complete yet. `sq`: boxes this CTA has started (picks list buffers and counters).
  uint32_t par = 0u, pend = 0u, sq = 0u, cur = 0u;
  float2 acc[8][2];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
  bool aborted = false;
  for (int64_t w = blockIdx.x; w < G.items; w += gridDim.x, cur ^= 1u) {
    __syncthreads();  // this item's descriptor is written; the last item's readers of the other are done
    const RegItem* I = items + cur;
    if (tid == 0) {
      for (int b = 0; b < min(2, I->nbox); ++b) {
        reg_issue_box<NSUB>(&tmap, I, b, b, sm);
        pend |= 1u << b;
      }
    }
    if (tid == 32 && w + gridDim.x < G.items) reg_item(G, w + gridDim.x, rbox, items + (cur ^ 1u));
    reg_hash<NSUB>(G, I, 0, sq, sm);
    __syncthreads();
    const int32_t nbox = I->nbox;
    for (int32_t b = 0; b < nbox; ++b, ++sq) {
      const int buf = b & 1;
      // 1. Hash the next box (its lists are the other buffer, emptied a box ago).
      if (b + 1 < nbox) reg_hash<NSUB>(G, I, b + 1, sq + 1u, sm);
      const bool ok = mbar_wait_bounded(bars + buf, (par >> buf) & 1u);
      if (ok || tid != 0) par ^= 1u << buf;
      if (tid == 0 && ok) pend &= ~(1u << buf);
      const unsigned char* st = sm + kRegStage + (size_t)buf * box_bytes;
      uint32_t* cn = reinterpret_cast<uint32_t*>(sm + kRegCnt) + (sq & 1u) * kRegTargets;
      if (ok) {
        // 2a. Overflow rows, one per quarter-warp: 8 lanes read the row's 128 bytes and reduce them
        //     into the chunk totals of their output row.
        const uint32_t no = min(nov[sq & 3u], (uint32_t)G.ovf_cap);
        const uint32_t* ov = reinterpret_cast<const uint32_t*>(sm + G.S.ovf) + (sq & 1u) * (uint32_t)G.ovf_cap;
        const int ql = tid & 7;
        const int64_t n = G.D.n;
        const int64_t col0 = (int64_t)I->xcol + 4 * ql;
        for (uint32_t o = (uint32_t)(tid >> 3); o < no; o += kRegThreads / 8) {
          const uint32_t e = ov[o];
          float4 v = *reinterpret_cast<const float4*>(st + ((e & 0x7FFFu) << 7) + ql * 16);
          if (e & 0x8000u) v = make_float4(-v.x, -v.y, -v.z, -v.w);
          float* Pt = G.P + (int64_t)I->tl * ((int64_t)G.D.B * G.D.k * n);
          if (col0 < n) red_quad(Pt + ((int64_t)I->tr0 + (e >> 16)) * n + col0, n, col0, v);
        }
        // 2b. This thread's list.
        const uint16_t* tb = reinterpret_cast<const uint16_t*>(sm + G.S.tab + (sq & 1u) * G.S.tab_stride);
        const uint32_t ns = min(cn[tid], (uint32_t)G.cap);
        for (uint32_t i = 0; i < ns; ++i) {
          const uint32_t e = tb[i * kRegTargets + tid];
          const uint32_t ra = ((e & 0x7FFFu) << 7) | l16;
          const float sg = __uint_as_float(((e & 0x8000u) << 16) | 0x3F800000u);
          const float2 s2 = make_float2(sg, sg);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(st + (ra ^ ((uint32_t)q << 4)));
            acc[q][0] = __ffma2_rn(make_float2(v.x, v.y), s2, acc[q][0]);
            acc[q][1] = __ffma2_rn(make_float2(v.z, v.w), s2, acc[q][1]);
          }
        }
        cn[tid] = 0u;
      }
      if (tid == 0) nov[(sq + 2u) & 3u] = 0u;  // last read two boxes ago; next written after this barrier
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if (tid == 0 && b + 2 < nbox) {
        reg_issue_box<NSUB>(&tmap, I, b + 2, buf, sm);
        pend |= 1u << buf;
      }
    }
    if (aborted) break;
    // 3. The item's partial sums into the chunk totals (zero sums add nothing).
    if (tid < I->ntr) {
      const int64_t n = G.D.n;
      float* prow = G.P + (int64_t)I->tl * ((int64_t)G.D.B * G.D.k * n) + ((int64_t)I->tr0 + tid) * n;
      const int64_t xcol = I->xcol;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t col0 = xcol + (int64_t)(((uint32_t)q << 2) ^ (l16 >> 2));
        const float4 v = make_float4(acc[q][0].x, acc[q][0].y, acc[q][1].x, acc[q][1].y);
        if (col0 < n && (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)) red_quad(prow + col0, n, col0, v);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
  }
  if (aborted && tid == 0) {
    if (G.status) atomicOr(G.status, kStatusTimeout);
    // Leave only after this CTA's copies in flight have landed (bounded). At most one box per
    // buffer is outstanding; it completes the phase of parity bit b of `par`.
    for (int b = 0; b < 2; ++b)
      if ((pend >> b) & 1u) mbar_wait_bounded(bars + b, (par >> b) & 1u);
  }
}

}  // namespace

size_t reg_smem_bytes(int32_t nsub, int32_t cap, int32_t ovf_cap) { return reg_smem(nsub, cap, ovf_cap).total; }

// Blocks of S that reach the widest target group of a sketch with d rows and block height B.
int32_t reg_blocks_per_group(int64_t d, int64_t B) {
  int32_t nbg = 1;
  for (int64_t tr0 = 0; tr0 < d; tr0 += kRegTargets) {
    const int64_t tr1 = std::min<int64_t>(d, tr0 + kRegTargets) - 1;
    nbg = std::max<int32_t>(nbg, (int32_t)(tr1 / B - tr0 / B + 1));
  }
  return nbg;
}

int32_t reg_threads() { return kRegThreads; }

int32_t reg_targets() { return kRegTargets; }

// List capacity for lambda entries per output row and box (a Poisson mean): about
// lambda + 1.5 sqrt(lambda), at least 2. A thread's list costs as many steps as the longest list of its
// warp, so short lists keep the warp's steps close to lambda; the entries past the capacity (about 6 %
// at lambda = 1.5) take the overflow list.
static int32_t list_cap(double lam) {
  return std::max<int32_t>(2, (int32_t)std::lround(lam + 1.5 * std::sqrt(lam)));
}

// Box height and list capacity for a sketch with d rows and block height B: the largest box (up to
// kRegMaxSub copies) whose buffers, lists and overflow lists fit in `smem_limit` bytes, with the
// capacity from list_cap for lambda = box rows / B, or cap_fixed if positive. The overflow list holds
// every entry a box can produce (box rows x blocks reaching a target group), so no entry is ever
// dropped. False if nothing fits.
bool reg_choose_box(int64_t d, int64_t B, size_t smem_limit, int32_t cap_fixed, int32_t* nsub, int32_t* cap) {
  const int32_t nbg = reg_blocks_per_group(d, B);
  for (int32_t s = kRegMaxSub; s >= 1; --s) {
    const double lam = (double)(s * kRegCopyRows) / (double)std::max<int64_t>(B, 1);
    const int32_t c = cap_fixed > 0 ? cap_fixed : list_cap(lam);
    if (reg_smem(s, c, s * kRegCopyRows * nbg).total <= smem_limit) {
      *nsub = s;
      *cap = c;
      return true;
    }
  }
  return false;
}

cudaError_t launch_reg(const TileLaunch& L, cudaStream_t st, int32_t* launches) {
  if (L.a_type != kAF32 || !L.P || L.reg_nsub < 1 || L.reg_nsub > kRegMaxSub || L.reg_cap < 1)
    return cudaErrorInvalidValue;
  RegGrid G;
  memset(&G, 0, sizeof(G));
  const int64_t B = L.d / L.k;
  G.D.A = L.A;
  G.D.Y = L.Y;
  G.D.lda = L.lda;
  G.D.n = L.n;
  G.D.row_base = L.row_begin;
  G.D.seed = L.seed;
  G.D.scale = L.scale;
  G.D.B = (uint32_t)B;
  G.D.k = (uint32_t)L.k;
  G.D.kp = (uint32_t)((L.k + 1) / 2);
  G.D.log2NC = 5;
  G.D.S = 1;
  G.D.kb = L.k;
  G.D.col_off = L.col_off;
  G.D.a_type = kAF32;
  G.row_begin = L.row_begin;
  G.row_end = L.row_end;
  G.R = L.R;
  G.t_first = L.row_begin / L.R;
  const int64_t chunks = (L.row_end - 1) / L.R - G.t_first + 1;
  G.ncg = (int32_t)((L.n + 31) / 32);
  G.ntg = (int32_t)((L.d + kRegTargets - 1) / kRegTargets);
  G.slices = std::max(1, L.slices);
  G.items = chunks * G.slices * G.ncg * G.ntg;
  G.nsub = L.reg_nsub;
  G.cap = L.reg_cap;
  G.P = L.P;
  G.status = L.status;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  G.ovf_cap = G.nsub * kRegCopyRows * reg_blocks_per_group(L.d, B);  // every entry of a box
  G.S = reg_smem(G.nsub, G.cap, G.ovf_cap);
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  if (!encode_a_map(&tmap, L.A, kAF32, L.lda, L.n, L.row_end - L.row_begin, 32, kRegCopyRows))
    return cudaErrorInvalidValue;
  const size_t smem = G.S.total;
  void (*kern)(const RegGrid, const CUtensorMap) = nullptr;
  switch (G.nsub) {
    case 1: kern = reg_kernel<1>; break;
    case 2: kern = reg_kernel<2>; break;
    case 3: kern = reg_kernel<3>; break;
    case 4: kern = reg_kernel<4>; break;
    case 5: kern = reg_kernel<5>; break;
    default: kern = reg_kernel<6>; break;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t grid = L.grid > 0 ? L.grid : (int64_t)sms;
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, G.items));
  kern<<<(unsigned)grid, kRegThreads, smem, st>>>(G, tmap);
  if (launches) *launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (L.no_finish) return cudaSuccess;
  return launch_chunk_finish(G.D, L.rule, G.P, G.t_first, chunks, st, launches);
}

}  // namespace sk
