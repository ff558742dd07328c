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
// Per staged box of rows (up to 768 rows x 32 columns, double-buffered TMA copies):
//   1. hash: each row's SplitMix64 outputs give its target row in every block of the group (the same
//      generator as every other kernel); a shared-memory counter per target row (native integer
//      atomic) hands out a slot in that row's list of 16-bit (row of the box, sign) entries;
//   2. accumulate: every thread walks its own list; for an entry it reads the row's 128 bytes with
//      eight 16-byte loads and adds them, signed, with packed FP32 FMAs. Lane l reads the row's
//      16-byte chunks in the order l, l+1, ... (mod 8), so at every step the 8 lanes of a
//      quarter-warp (one shared-memory wavefront for 16-byte loads) hit 8 distinct chunks, hence 8
//      distinct bank groups, whichever rows they read; register group q of lane l therefore holds
//      columns 4((q + l) mod 8) .. +3.
// A list holds `cap` entries, about lambda + 1.5 sqrt(lambda) for lambda = box rows / B, the mean
// number of entries an output row receives per box: longer lists would make every warp wait for its
// longest one. Rows beyond a full list go to an overflow list, which the CTA's quarter-warps add into
// the chunk totals with FP32 vector reductions (one 128-byte row per quarter-warp access). At the end
// of the item every thread adds its 32 sums into P.
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
constexpr int kRegMaxSub = 6;             // TMA copies per staged box
constexpr int kRegOvf = 2048;             // overflow-list entries (a box that overflows more adds the rest
                                          // directly from the hashing thread)

struct RegGrid {
  TileDesc D;
  int64_t row_begin, row_end;  // global rows processed
  int64_t R;                   // chunk rows
  int64_t t_first;             // first chunk index
  int64_t items;               // chunks * slices * ncg * ntg
  int32_t ncg, ntg, slices;
  int32_t nsub;                // TMA copies per staged box (box = nsub * kRegCopyRows rows)
  int32_t cap;                 // list entries per output row and box
  float* P;                    // per-chunk FP32 totals, chunk-major, d x n each (zero on entry)
  unsigned* status;            // sticky status word
};

struct RegSmem {
  size_t stage_off, tab_off, cnt_off, ovf_off, bar_off, total;
};

// Shared memory: two staged boxes | list entries (kRegTargets x cap, 16-bit: row of the box in bits
// 0..14, sign in bit 15) | list lengths | overflow list (kRegOvf 32-bit entries: output row of the
// group << 16 | row of the box | sign << 15) | 2 overflow counters | 2 mbarriers.
__host__ __device__ inline RegSmem reg_smem(int32_t nsub, int32_t cap) {
  RegSmem L;
  L.stage_off = 0;
  L.tab_off = (size_t)2 * nsub * kRegCopyRows * 128;
  L.cnt_off = L.tab_off + (((size_t)kRegTargets * cap * 2 + 15) & ~(size_t)15);
  L.ovf_off = L.cnt_off + (size_t)kRegTargets * 4;
  L.bar_off = L.ovf_off + (size_t)kRegOvf * 4 + 8;
  L.total = L.bar_off + 2 * 8;
  return L;
}

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

__global__ void __launch_bounds__(kRegThreads, 1) reg_kernel(const RegGrid G, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RegSmem SL = reg_smem(G.nsub, G.cap);
  unsigned char* stage = smem_raw + SL.stage_off;
  uint16_t* tab = reinterpret_cast<uint16_t*>(smem_raw + SL.tab_off);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem_raw + SL.cnt_off);
  uint32_t* ovf = reinterpret_cast<uint32_t*>(smem_raw + SL.ovf_off);
  uint32_t* novf = ovf + kRegOvf;  // two counters, used by alternate boxes
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + SL.bar_off);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int ql = lane & 7;  // lane in its quarter-warp
  const int qid = tid >> 3;  // quarter-warp of the CTA (overflow rows)
  if (blockDim.x != kRegThreads || G.nsub < 1 || G.nsub > kRegMaxSub || G.cap < 1) {
    if (tid == 0 && G.status) atomicOr(G.status, kStatusBounds);
    return;
  }
  const int32_t rbox = G.nsub * kRegCopyRows;
  const uint32_t box_bytes = (uint32_t)rbox * 128u;
  const uint32_t cap = (uint32_t)G.cap;
  if (tid == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    mbar_fence_init();
    novf[0] = novf[1] = 0u;
  }
  cnt[tid] = 0u;
  __syncthreads();
  const TileDesc& D = G.D;
  const uint32_t B = D.B;
  const int64_t d = (int64_t)B * D.k;
  const int64_t n = D.n;
  const int64_t dn = d * n;
  // Byte offset, inside a 128-byte row, of the chunk this lane reads at step q: (q + lane) mod 8.
  uint32_t off[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) off[q] = (uint32_t)((q + lane) & 7) << 4;
  // Bit b of `par`: parity of the next phase of buffer b's mbarrier (toggled after every wait; in
  // thread 0 only after a wait that succeeded). Bit b of `pend` (thread 0): a box copied into buffer b
  // has not been seen complete yet.
  uint32_t par = 0u, pend = 0u;
  uint32_t nbox_done = 0u;  // boxes processed by this CTA (picks the overflow counter)
  float2 acc[8][2];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
  bool aborted = false;
  for (int64_t w = blockIdx.x; w < G.items && !aborted; w += gridDim.x) {
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
    // Output rows of the group and the blocks (and 64-bit stream outputs) that reach them.
    const int64_t tr0 = (int64_t)tg * kRegTargets;
    const int64_t ntr = min((int64_t)kRegTargets, d - tr0);
    const uint32_t jlo = (uint32_t)(tr0 / B);
    const uint32_t jhi = (uint32_t)((tr0 + ntr - 1) / B);
    const uint32_t plo = jlo >> 1;
    const uint32_t np = (jhi >> 1) - plo + 1;
    const int32_t nbox = (int32_t)((r1 - r0 + rbox - 1) / rbox);
    const int32_t xcol = g * 32;
    const int32_t ybase = (int32_t)(r0 - D.row_base);
    float* Pt = G.P + tl * dn;
    if (tid == 0) {
      fence_proxy_async_smem();  // the previous item read both buffers through the generic proxy
      for (int b = 0; b < min(2, nbox); ++b) {
        mbar_arrive_expect_tx(bars + b, box_bytes);
        for (int s = 0; s < G.nsub; ++s)
          tma_load_2d(stage + (size_t)b * box_bytes + (size_t)s * kRegCopyRows * 128, &tmap, xcol,
                      ybase + b * rbox + s * kRegCopyRows, bars + b);
        pend |= 1u << b;
      }
    }
    for (int32_t b = 0; b < nbox; ++b, ++nbox_done) {
      const int buf = b & 1;
      const bool ok = mbar_wait_bounded(bars + buf, (par >> buf) & 1u);
      if (ok || tid != 0) par ^= 1u << buf;
      if (tid == 0 && ok) pend &= ~(1u << buf);
      const unsigned char* st = stage + (size_t)buf * box_bytes;
      const int64_t rb0 = r0 + (int64_t)b * rbox;
      const int32_t nr = (int32_t)min((int64_t)rbox, r1 - rb0);
      uint32_t* nov = novf + (nbox_done & 1u);
      // 1. Hash: list entries of the box's rows.
      for (int32_t row = tid; row < nr && ok; row += kRegThreads) {
        for (uint32_t pr = 0; pr < np; ++pr) {
          const uint32_t p = plo + pr;
          const uint64_t h = row_pair_bits(D.seed, (uint64_t)(rb0 + row), D.kp, p);
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const uint32_t j = 2u * p + (uint32_t)e;
            if (j < jlo || j > jhi) continue;
            const uint32_t wd = e ? (uint32_t)h : (uint32_t)(h >> 32);
            const int64_t tgt = (int64_t)j * B + word_to_slot(wd, B) - tr0;
            if ((uint64_t)tgt >= (uint64_t)ntr) continue;
            const uint32_t ent = (uint32_t)row | ((wd & 1u) << 15);
            const uint32_t pos = atomicAdd(cnt + tgt, 1u);
            if (pos < cap) {
              tab[(uint32_t)tgt * cap + pos] = (uint16_t)ent;
            } else {
              const uint32_t o = atomicAdd(nov, 1u);
              if (o < (uint32_t)kRegOvf) {
                ovf[o] = ((uint32_t)tgt << 16) | ent;
              } else {
                // Overflow list full too: add this row's 32 values into the chunk totals here.
                const float4* src = reinterpret_cast<const float4*>(st + ((uint32_t)row << 7));
                float* prow = Pt + (tr0 + tgt) * n;
                for (int c = 0; c < 8; ++c) {
                  const int64_t col0 = (int64_t)xcol + 4 * c;
                  if (col0 >= n) break;
                  float4 v = src[c];
                  if (wd & 1u) v = make_float4(-v.x, -v.y, -v.z, -v.w);
                  red_quad(prow + col0, n, col0, v);
                }
              }
            }
          }
        }
      }
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      // 2. Accumulate this thread's list.
      {
        const uint32_t ns = min(cnt[tid], cap);
        const uint16_t* te = tab + (uint32_t)tid * cap;
        for (uint32_t i = 0; i < ns; ++i) {
          const uint32_t e = te[i];
          const unsigned char* rp = st + ((e & 0x7FFFu) << 7);
          const float sg = __uint_as_float(((e & 0x8000u) << 16) | 0x3F800000u);
          const float2 s2 = make_float2(sg, sg);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(rp + off[q]);
            acc[q][0] = __ffma2_rn(make_float2(v.x, v.y), s2, acc[q][0]);
            acc[q][1] = __ffma2_rn(make_float2(v.z, v.w), s2, acc[q][1]);
          }
        }
        cnt[tid] = 0u;
      }
      // 3. Overflow rows, one per quarter-warp: 8 lanes read the row's 128 bytes and reduce them into
      //    the chunk totals of their output row.
      {
        const uint32_t no = min(*nov, (uint32_t)kRegOvf);
        const int64_t col0 = (int64_t)xcol + 4 * ql;
        for (uint32_t o = (uint32_t)qid; o < no; o += kRegThreads / 8) {
          const uint32_t e = ovf[o];
          float4 v = *reinterpret_cast<const float4*>(st + ((e & 0x7FFFu) << 7) + ql * 16);
          if (e & 0x8000u) v = make_float4(-v.x, -v.y, -v.z, -v.w);
          if (col0 < n) red_quad(Pt + (tr0 + (e >> 16)) * n + col0, n, col0, v);
        }
      }
      if (tid == 0) novf[(nbox_done + 1u) & 1u] = 0u;  // the next box's counter (last read a box ago)
      __syncthreads();
      if (tid == 0 && b + 2 < nbox) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bars + buf, box_bytes);
        for (int s = 0; s < G.nsub; ++s)
          tma_load_2d(stage + (size_t)buf * box_bytes + (size_t)s * kRegCopyRows * 128, &tmap, xcol,
                      ybase + (b + 2) * rbox + s * kRegCopyRows, bars + buf);
        pend |= 1u << buf;
      }
    }
    if (aborted) break;
    // 4. The item's partial sums into the chunk totals (zero sums add nothing).
    if (tid < ntr) {
      float* prow = Pt + (tr0 + tid) * n;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t col0 = (int64_t)xcol + (int64_t)off[q] / 4;
        const float4 v = make_float4(acc[q][0].x, acc[q][0].y, acc[q][1].x, acc[q][1].y);
        if (col0 < n && (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)) red_quad(prow + col0, n, col0, v);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
  }
  if (aborted) {
    if (tid == 0) {
      if (G.status) atomicOr(G.status, kStatusTimeout);
      // Leave only after this CTA's copies in flight have landed (bounded). At most one box per
      // buffer is outstanding; it completes the phase of parity bit b of `par`.
      for (int b = 0; b < 2; ++b)
        if ((pend >> b) & 1u) mbar_wait_bounded(bars + b, (par >> b) & 1u);
    }
  }
}

}  // namespace

size_t reg_smem_bytes(int32_t nsub, int32_t cap) { return reg_smem(nsub, cap).total; }

int32_t reg_threads() { return kRegThreads; }

int32_t reg_targets() { return kRegTargets; }

// List capacity for lambda entries per output row and box (a Poisson mean): about
// lambda + 1.5 sqrt(lambda), at least 2. A thread's list costs as many steps as the longest list of its
// warp, so short lists keep the warp's steps close to lambda; the entries past the capacity (about 6 %
// at lambda = 1.5) take the overflow list.
static int32_t list_cap(double lam) {
  return std::max<int32_t>(2, (int32_t)std::lround(lam + 1.5 * std::sqrt(lam)));
}

// Box height and list capacity for block height B: the largest box (up to kRegMaxSub copies) whose
// buffers and lists fit in `smem_limit` bytes, with the capacity from list_cap for
// lambda = box rows / B, or cap_fixed if positive. False if nothing fits.
bool reg_choose_box(int64_t B, size_t smem_limit, int32_t cap_fixed, int32_t* nsub, int32_t* cap) {
  for (int32_t s = kRegMaxSub; s >= 1; --s) {
    const double lam = (double)(s * kRegCopyRows) / (double)std::max<int64_t>(B, 1);
    const int32_t c = cap_fixed > 0 ? cap_fixed : list_cap(lam);
    if (reg_smem(s, c).total <= smem_limit) {
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
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  if (!encode_a_map(&tmap, L.A, kAF32, L.lda, L.n, L.row_end - L.row_begin, 32, kRegCopyRows))
    return cudaErrorInvalidValue;
  const size_t smem = reg_smem(G.nsub, G.cap).total;
  cudaError_t e = cudaFuncSetAttribute(reg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t grid = L.grid > 0 ? L.grid : (int64_t)sms;
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, G.items));
  reg_kernel<<<(unsigned)grid, kRegThreads, smem, st>>>(G, tmap);
  if (launches) *launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (L.no_finish) return cudaSuccess;
  return launch_chunk_finish(G.D, L.rule, G.P, G.t_first, chunks, st, launches);
}

}  // namespace sk
