// One work item of the chunked sketch: rows [r0, r1) (all or a slice of chunk t), columns
// [g*NC, g*NC + NC) and blocks [j0, j0 + kbe) of S, accumulated in an FP32 shared-memory tile and
// then flushed.
//
// Paper Sec. 4.1 (scatter of every element of A to its zeta target rows, Listing 1) and Sec. 4.2
// (FP16 quantization of each contribution, packed half2 atomics, Listing 2). Two changes from the
// paper's per-element design: (1) contributions of the R rows of one chunk that reach the same
// output are first summed in FP32 on chip, and the chunk total is what gets scaled, quantized and
// added into Y; (2) S is never read from memory: its nonzero pattern is regenerated from the
// SplitMix64 stream (one 64-bit output per input row and pair of blocks).
//
// Shared-memory layout of the accumulator: lines of LW = S*NC floats. Block jl of the group (jl in
// [0, kb)) owns lines (jl / S) * B + s for its B target rows s, in slot (jl % S) of width NC.
// A warp is split into G = 32/NC lane groups of NC lanes (one lane per column); in one pass the G
// lane groups handle G (row, block) pairs of the same row batch. When kb >= G the G pairs of a pass
// lie in G different slots, so the 32 lanes touch 32 different banks.
//
// A chunk split into several slices (work items on different CTAs) is combined in two levels: each
// slice adds its FP32 partials into a per-chunk FP32 buffer in global memory, and the CTA that
// finishes the chunk's last slice scales, quantizes and adds the chunk total into Y. The result is
// the chunk total of the canonical order up to the FP32 summation order inside the chunk.
#pragma once

#include "sk_device.cuh"

namespace sk {

struct TileDesc {
  const void* A;    // row 0 of A is global row `row_base`; elements of type a_type
  void* Y;          // d x n, float or binary16
  int64_t lda;
  int64_t n;
  int64_t row_base;
  uint64_t seed;
  float scale;      // fl32(1/sqrt(k))
  uint32_t B;       // rows per block of S
  uint32_t k;       // blocks (nonzeros per column)
  uint32_t kp;      // ceil(k/2): 64-bit stream outputs per input row
  int32_t log2NC;   // columns per work item = 1 << log2NC (2..5)
  int32_t S;        // slots per accumulator line
  int32_t kb;       // blocks per block group
  int64_t col_off;  // global column index of column 0 (keys the rounding random bits)
  const void* tmap; // 2-D tensor map over A (box NC x RB*mb), or null: direct loads
  int32_t mb;       // hash rounds (of RB = 32/kp rows) per TMA box
  int32_t lr;       // 1: every work item holds all k blocks and takes the lane-row TMA path
  int32_t vec;      // 1: n = 1, one thread per row (tile_scatter_vec)
  int32_t a_type;   // element type of A (AType: FP32, binary16, bfloat16)
  int64_t ldy;      // row stride of Y in elements (0: n); the chunk finish of a column slab writes
                    // columns [0, n) of a wider Y
};

// Launch parameters of the chunked kernels (tile kernel and owner kernel).
struct TileGrid {
  TileDesc D;
  int64_t row_begin, row_end;  // global rows processed
  int64_t R;                   // chunk rows
  int64_t t_first;             // first chunk index
  int64_t items;               // chunks * slices * nbg * ncg
  int32_t ncg, nbg, slices;
  int32_t acc_floats;          // floats of the accumulator (multiple of 4)
  float* P;                    // slices > 1: per-chunk FP32 totals, chunk-major, d x n each (zero)
  unsigned* status;            // sticky status word (kStatus*), may be null
  int32_t use_tma;             // 1: A arrives through the tensor map
  int32_t depth;               // TMA ring slots per warp
};

// Per-warp TMA staging ring: `depth` slots of RB x NC floats (128-byte aligned) and their mbarriers.
// `uses` counts the batches this warp has consumed so far; slot and phase parity derive from it.
struct WarpRing {
  float* slots;
  uint64_t* bars;
  int32_t depth;
  int32_t slot_floats;
  uint32_t uses;
};

// Bytes of one staging slot for RB rows of NC floats (at least 128, a multiple of 128).
__host__ __device__ inline int32_t ring_slot_bytes(int32_t RB, int32_t NC) {
  const int32_t b = RB * NC * 4;
  return ((b + 127) / 128) * 128;
}
constexpr int kMaxRingDepth = 4;

// 32-bit words per warp of the per-batch target buffer.
constexpr int kWordsPerWarp = 64;


// Floats of the accumulator tile for a descriptor.
__host__ __device__ inline int64_t tile_acc_floats(uint32_t B, int32_t kb, int32_t S, int32_t NC) {
  return (int64_t)((kb + S - 1) / S) * (int64_t)B * (int64_t)S * (int64_t)NC;
}

// Shared-memory carve-up of the tile kernels: accumulator | per-warp target words | per-warp TMA
// ring slots (128-byte aligned) | per-warp ring mbarriers.
struct SmemPlan {
  size_t acc_bytes, wbuf_off, slots_off, bars_off, total;
  int32_t slot_bytes, depth;
};

__host__ __device__ inline SmemPlan smem_plan(int64_t acc_floats, int nwarps, int32_t slot_bytes, int32_t depth) {
  SmemPlan L;
  L.acc_bytes = (size_t)acc_floats * 4;
  L.wbuf_off = (L.acc_bytes + 127) & ~(size_t)127;
  L.slots_off = L.wbuf_off + (size_t)nwarps * kWordsPerWarp * 4;
  L.slots_off = (L.slots_off + 127) & ~(size_t)127;
  L.bars_off = L.slots_off + (size_t)nwarps * depth * slot_bytes;
  L.total = L.bars_off + (size_t)nwarps * depth * 8;
  L.slot_bytes = slot_bytes;
  L.depth = depth;
  return L;
}

// Set up this warp's staging ring (lane 0 initializes the mbarriers).
__device__ __forceinline__ WarpRing make_ring(unsigned char* smem_raw, const SmemPlan& L, int warp) {
  WarpRing r;
  r.slots = reinterpret_cast<float*>(smem_raw + L.slots_off + (size_t)warp * L.depth * L.slot_bytes);
  r.bars = reinterpret_cast<uint64_t*>(smem_raw + L.bars_off) + warp * L.depth;
  r.depth = L.depth;
  r.slot_floats = L.slot_bytes / 4;
  r.uses = 0;
  if ((threadIdx.x & 31) == 0) {
    for (int s = 0; s < L.depth; ++s) mbar_init(r.bars + s, 1);
    mbar_fence_init();
  }
  __syncwarp();
  return r;
}

// Scatter rows [r0, r1) of the work item into the zeroed accumulator `acc`. Called by every warp of
// the CTA; warp `warp` of `nwarps` takes row batches warp, warp + nwarps, ... `wbuf` is this warp's
// kWordsPerWarp-word scratch: for each (row, block) of the current batch it holds the accumulator
// offset (in floats, without the column) of the row's target in that block, with the sign in bit 31.
// With a tensor map, the warp's batches of A arrive through its TMA ring (ring.depth batches in
// flight); otherwise each lane loads its batch's values directly. Returns false if a bounded wait
// gave up (after waiting, again bounded, for the warp's copies still in flight).
template <int PPR, typename TA>
__device__ __forceinline__ bool tile_scatter_t(const TileDesc& D, int64_t r0, int64_t r1, int32_t g, int32_t j0,
                                               int32_t kbe, float* acc, uint32_t* wbuf, WarpRing& ring, int warp,
                                               int nwarps) {
  const int lane = threadIdx.x & 31;
  const int NC = 1 << D.log2NC;
  const int G = 32 >> D.log2NC;
  const int q = lane >> D.log2NC;
  const int c = lane & (NC - 1);
  const int S = D.S;
  const int LW = S * NC;
  const uint32_t B = D.B;
  const int kp = (int)D.kp;
  const int64_t col = (int64_t)g * NC + c;
  const bool col_ok = col < D.n;
  const TA* __restrict__ Abase = static_cast<const TA*>(D.A) + (col_ok ? col : 0);
  float* __restrict__ acc_c = acc + c;
  // Rows of one batch: the 32 lanes compute one 64-bit stream output each, kp per row.
  const int RB = 32 / kp;
  const int64_t nrows = r1 - r0;
  const int64_t nbatch = (nrows + RB - 1) / RB;
  const int64_t nmine = (nbatch > warp) ? (nbatch - 1 - warp) / nwarps + 1 : 0;
  // Hash-round role of this lane: (row hr, pair hp) of the batch, the two blocks of the pair.
  const int hr = lane / kp;
  const int hp = lane - hr * kp;
  int hj[2], hoff[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int j = 2 * hp + e;
    const int jl = j - j0;
    hj[e] = (j < (int)D.k && jl >= 0 && jl < kbe) ? jl : -1;
    hoff[e] = (hj[e] >= 0) ? ((jl / S) * (int)B * LW + (jl % S) * NC) : 0;
  }
  const bool tma = D.tmap != nullptr;
  const int depth = ring.depth;
  const uint32_t box_bytes = (uint32_t)(RB * NC * sizeof(TA));
  auto issue = [&](int64_t kk) {
    const int64_t bt = warp + kk * nwarps;
    const uint32_t u = ring.uses + (uint32_t)kk;
    const int slot = (int)(u % (uint32_t)depth);
    uint64_t* bar = ring.bars + slot;
    mbar_arrive_expect_tx(bar, box_bytes);
    tma_load_2d(ring.slots + (size_t)slot * ring.slot_floats, D.tmap, g * NC, (int32_t)(r0 + bt * RB - D.row_base),
                bar);
  };
  if (tma && lane == 0) {
    for (int64_t kk = 0; kk < min((int64_t)depth, nmine); ++kk) issue(kk);
  }
  bool ok = true;
  for (int64_t kk = 0; kk < nmine; ++kk) {
    const int64_t bt = warp + kk * nwarps;
    const int64_t ib = r0 + bt * RB;
    const int nr = (int)min((int64_t)RB, r1 - ib);
    if (hr < nr) {
      const uint64_t h = row_pair_bits(D.seed, (uint64_t)(ib + hr), (uint32_t)kp, (uint32_t)hp);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (hj[e] >= 0) {
          const uint32_t w = e ? (uint32_t)h : (uint32_t)(h >> 32);
          const uint32_t s = word_to_slot(w, B);
          wbuf[hr * kbe + hj[e]] = ((uint32_t)hoff[e] + s * (uint32_t)LW) | (w << 31);
        }
      }
    }
    // Values of this batch: from the staging slot (row-major RB x NC box) or loaded directly.
    const TA* stage = nullptr;
    if (tma) {
      const uint32_t u = ring.uses + (uint32_t)kk;
      const int slot = (int)(u % (uint32_t)depth);
      if (!mbar_wait_bounded(ring.bars + slot, (u / (uint32_t)depth) & 1u)) {
        ok = false;
        // Drain this warp's later copies that are still in flight, then give up.
        for (int64_t k2 = kk + 1; k2 < min(kk + depth, nmine); ++k2) {
          const uint32_t u2 = ring.uses + (uint32_t)k2;
          mbar_wait_bounded(ring.bars + (u2 % (uint32_t)depth), (u2 / (uint32_t)depth) & 1u);
        }
        break;
      }
      stage = reinterpret_cast<const TA*>(ring.slots + (size_t)slot * ring.slot_floats);
    }
    __syncwarp();
    // This lane's updates of the batch, enumerated as entries e = 0..E-1, processed in groups of 8
    // with a batched compare-and-swap (shared-memory FP32 atomic add has no native instruction).
    if (PPR > 0 && tma) {
      // Fast path: PPR (row, block) passes per row, unrolled. Columns past n read TMA zero fill,
      // so their lanes add zeros into accumulator columns that are never flushed.
#pragma unroll 2
      for (int rl = 0; rl < nr; ++rl) {
        const float a = a_to_f32(stage[rl * NC + c]);
        const uint32_t* wr = wbuf + rl * kbe + q;
#pragma unroll
        for (int pp = 0; pp < (PPR > 0 ? PPR : 1); ++pp) {
          if (pp * G + q < kbe) {
            const uint32_t w = wr[pp * G];
            atomicAdd(acc_c + (w & 0x7FFFFFFFu), __uint_as_float(__float_as_uint(a) ^ (w & 0x80000000u)));
          }
        }
      }
    } else if (kbe >= G) {
      for (int rl = 0; rl < nr; ++rl) {
        const float a = tma ? a_to_f32(stage[rl * NC + c]) : (col_ok ? ld_a(Abase + (ib + rl - D.row_base) * D.lda) : 0.f);
        const uint32_t* wr = wbuf + rl * kbe;
        for (int jl = q; jl < kbe; jl += G) {
          const uint32_t w = wr[jl];
          const float v = __uint_as_float(__float_as_uint(a) ^ (w & 0x80000000u));
          if (col_ok) atomicAdd(acc_c + (w & 0x7FFFFFFFu), v);
        }
      }
    } else {
      // Fewer blocks than lane groups: a pass covers RP = G / kbe rows.
      const int RP = G / kbe;
      const int roff = q / kbe;
      const int jl = q - roff * kbe;
      if (roff < RP && col_ok) {
        for (int rl = roff; rl < nr; rl += RP) {
          const float a = tma ? a_to_f32(stage[rl * NC + c]) : ld_a(Abase + (ib + rl - D.row_base) * D.lda);
          const uint32_t w = wbuf[rl * kbe + jl];
          const float v = __uint_as_float(__float_as_uint(a) ^ (w & 0x80000000u));
          atomicAdd(acc_c + (w & 0x7FFFFFFFu), v);
        }
      }
    }
    __syncwarp();
    if (tma && lane == 0 && kk + depth < nmine) {
      fence_proxy_async_smem();
      issue(kk + depth);
    }
  }
  ring.uses += (uint32_t)nmine;
  return ok;
}

// TMA fast path (kb >= G): each warp takes boxes of SB = RB*mb rows (row boxes warp, warp + nwarps,
// ...), ring.depth of them in flight through its mbarrier ring; inside a box, mb hash rounds of RB
// rows each; PPR (row, block) passes per row, unrolled. Slot and phase parity advance incrementally.
// Columns past n read TMA zero fill, so those lanes add zeros into accumulator columns that are never
// flushed. Returns false if a bounded wait gave up (after draining this warp's copies in flight).
template <int PPR, typename TA>
__device__ __forceinline__ bool tile_scatter_tma(const TileDesc& D, int64_t r0, int64_t r1, int32_t g, int32_t j0,
                                                 int32_t kbe, float* acc, uint32_t* wbuf, WarpRing& ring, int warp,
                                                 int nwarps) {
  const int lane = threadIdx.x & 31;
  const int NC = 1 << D.log2NC;
  const int G = 32 >> D.log2NC;
  const int q = lane >> D.log2NC;
  const int c = lane & (NC - 1);
  const int S = D.S;
  const int LW = S * NC;
  const uint32_t B = D.B;
  const int kp = (int)D.kp;
  float* __restrict__ acc_c = acc + c;
  const int RB = 32 / kp;
  const int SB = RB * D.mb;
  const int32_t nrows = (int32_t)(r1 - r0);
  const int32_t nbox = (nrows + SB - 1) / SB;
  const int32_t nmine = (nbox > warp) ? (nbox - 1 - warp) / nwarps + 1 : 0;
  const int hr = lane / kp;
  const int hp = lane - hr * kp;
  int hj[2];
  uint32_t hoff[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int j = 2 * hp + e;
    const int jl = j - j0;
    hj[e] = (j < (int)D.k && jl >= 0 && jl < kbe) ? jl : -1;
    hoff[e] = (hj[e] >= 0) ? (uint32_t)((jl / S) * (int)B * LW + (jl % S) * NC) : 0u;
  }
  const int depth = ring.depth;
  const uint32_t box_bytes = (uint32_t)(SB * NC * sizeof(TA));
  const int32_t ybase = (int32_t)(r0 - D.row_base);
  const int xcol = g * NC;
  int slot = (int)(ring.uses % (uint32_t)depth);
  uint32_t par = (ring.uses / (uint32_t)depth) & 1u;
  if (lane == 0) {
    int s2 = slot;
    for (int32_t kk = 0; kk < min(depth, nmine); ++kk) {
      mbar_arrive_expect_tx(ring.bars + s2, box_bytes);
      tma_load_2d(ring.slots + (size_t)s2 * ring.slot_floats, D.tmap, xcol, ybase + (warp + kk * nwarps) * SB,
                  ring.bars + s2);
      s2 = (s2 + 1 == depth) ? 0 : s2 + 1;
    }
  }
  bool ok = true;
  for (int32_t kk = 0; kk < nmine; ++kk) {
    const int32_t box0 = (warp + kk * nwarps) * SB;  // first row of the box, relative to r0
    if (!mbar_wait_bounded(ring.bars + slot, par)) {
      ok = false;
      int s2 = slot;
      uint32_t p2 = par;
      for (int32_t k2 = kk + 1; k2 < min(kk + depth, nmine); ++k2) {
        s2 = (s2 + 1 == depth) ? 0 : s2 + 1;
        if (s2 == 0) p2 ^= 1u;
        mbar_wait_bounded(ring.bars + s2, p2);
      }
      break;
    }
    const TA* stage = reinterpret_cast<const TA*>(ring.slots + (size_t)slot * ring.slot_floats);
    for (int hb = 0; hb < D.mb; ++hb) {
      const int32_t rb0 = box0 + hb * RB;
      const int nr = min(RB, nrows - rb0);
      if (nr <= 0) break;
      if (hr < nr) {
        const uint64_t h = row_pair_bits(D.seed, (uint64_t)(r0 + rb0 + hr), (uint32_t)kp, (uint32_t)hp);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (hj[e] >= 0) {
            const uint32_t w = e ? (uint32_t)h : (uint32_t)(h >> 32);
            wbuf[hr * kbe + hj[e]] = (hoff[e] + word_to_slot(w, B) * (uint32_t)LW) | (w << 31);
          }
        }
      }
      __syncwarp();
      const TA* st = stage + hb * RB * NC + c;
#pragma unroll 2
      for (int rl = 0; rl < nr; ++rl) {
        const float a = a_to_f32(st[rl * NC]);
        const uint32_t* wr = wbuf + rl * kbe + q;
#pragma unroll
        for (int pp = 0; pp < PPR; ++pp) {
          if (pp * G + q < kbe) {
            const uint32_t w = wr[pp * G];
            atomicAdd(acc_c + (w & 0x7FFFFFFFu), __uint_as_float(__float_as_uint(a) ^ (w & 0x80000000u)));
          }
        }
      }
      __syncwarp();
    }
    if (lane == 0 && kk + depth < nmine) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(ring.bars + slot, box_bytes);
      tma_load_2d(ring.slots + (size_t)slot * ring.slot_floats, D.tmap, xcol,
                  ybase + (warp + (kk + depth) * nwarps) * SB, ring.bars + slot);
    }
    slot = (slot + 1 == depth) ? 0 : slot + 1;
    if (slot == 0) par ^= 1u;
  }
  ring.uses += (uint32_t)nmine;
  return ok;
}

// Shared-memory FP32 reduction (no result); `addr` is a shared-window byte address.
__device__ __forceinline__ void red_shared_f32(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

// One hash round of the lane-row path for lane (r, hp): its row's values at
// `arow` (NC floats of the staged box), the lane's E blocks (2, or 1 when k = 1) at accumulator byte
// addresses base[e] (target row and column still to add). PRED = false is the straight-line form for
// rounds in which every lane holds a row and all its blocks exist.
// `z` is the SplitMix64 state of the lane's stream output (seed + index * golden gamma).
template <int NC, bool PRED, typename TA, int E = 2>
__device__ __forceinline__ void lr_round(const TileDesc& D, uint64_t z, int rot, int flip, const TA* arow,
                                         const uint32_t base[2], const bool bv[2], uint32_t LW) {
  const uint64_t h = splitmix_finalize(z);
  uint32_t ad[2], sg[2];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t w = (e ^ flip) ? (uint32_t)h : (uint32_t)(h >> 32);
    ad[e] = base[e] + 4u * word_to_slot(w, D.B) * LW;
    sg[e] = w << 31;
  }
  // (a partial unroll at NC = 32 keeps the loads in flight within the register budget)
#pragma unroll(NC > 16 ? 8 : NC)
  for (int c = 0; c < NC; ++c) {
    const uint32_t col = (uint32_t)(c + rot) & (uint32_t)(NC - 1);
    const uint32_t a = __float_as_uint(a_to_f32(arow[col]));
    if (!PRED || bv[0]) red_shared_f32(ad[0] + 4u * col, __uint_as_float(a ^ sg[0]));
    if (E > 1 && (!PRED || bv[1])) red_shared_f32(ad[1] + 4u * col, __uint_as_float(a ^ sg[1]));
  }
}

// Lane-row TMA path, for work items that hold all k blocks (j0 = 0, kbe = k). Within a hash round of
// RB = 32/kp rows, lane (r, hp) owns row r and the pair of blocks (2hp, 2hp+1): it computes that
// pair's 64-bit stream output, keeps both targets and signs in registers and adds its row's NC values
// into both targets, column (c + rot) mod NC at step c with rot = r + RB * floor(hp / S). A
// lane-dependent flip decides which block of the pair comes first, so that at a given step lane
// (r, hp) writes slot (2hp + flip) mod S. With S*NC = 32 floats per line and kp >= S, the lanes that
// share a slot are the RB*kp/S = NC lanes (r, hp') with hp' = hp mod S, and rot takes NC distinct
// values over them: the 32 lanes of one access hit 32 distinct banks (k = 8 with NC = 8 or 16, for
// example); other shapes stay correct with some bank conflicts. No per-update target word is read
// from shared memory and no warp-level exchange is needed, so a round is straight-line code.
// Boxes, ring and bounded waits are as in tile_scatter_tma. Columns past n read TMA zero fill and
// add zeros into accumulator columns that are never flushed.
template <int NC, typename TA>
__device__ __forceinline__ bool tile_scatter_lr(const TileDesc& D, int64_t r0, int64_t r1, int32_t g, float* acc,
                                                WarpRing& ring, int warp, int nwarps) {
  const int lane = threadIdx.x & 31;
  const int S = D.S;
  const uint32_t LW = (uint32_t)(S * NC);
  const uint32_t B = D.B;
  const int kp = (int)D.kp;
  const int RB = 32 / kp;
  const int SB = RB * D.mb;
  const int r = lane / kp;
  const int hp = lane - r * kp;
  // k = 1 (CountSketch): one block per lane, no flip, so that the valid block is e = 0 on every lane
  // and the round has a single, warp-uniform update per column.
  const bool single = (D.k == 1);
  const int flip = single ? 0 : (((2 * hp) / S + r / NC) & 1);
  const int rot = r + RB * (hp / S);
  const uint32_t acc_s = (uint32_t)__cvta_generic_to_shared(acc);
  uint32_t base[2];
  bool bv[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int j = 2 * hp + (e ^ flip);
    bv[e] = r < RB && j < (int)D.k;
    base[e] = acc_s + 4u * ((uint32_t)(j / S) * B * LW + (uint32_t)((j % S) * NC));
  }
  // Every lane holds a row of a full round and all its blocks exist (warp-uniform).
  const bool full_lanes = (RB * kp == 32) && (((D.k & 1u) == 0) || single);
  const int32_t nrows = (int32_t)(r1 - r0);
  const int32_t nbox = (nrows + SB - 1) / SB;
  const int32_t nmine = (nbox > warp) ? (nbox - 1 - warp) / nwarps + 1 : 0;
  const int depth = ring.depth;
  const uint32_t box_bytes = (uint32_t)(SB * NC * sizeof(TA));
  const int32_t ybase = (int32_t)(r0 - D.row_base);
  const int xcol = g * NC;
  int slot = (int)(ring.uses % (uint32_t)depth);
  uint32_t par = (ring.uses / (uint32_t)depth) & 1u;
  if (lane == 0) {
    int s2 = slot;
    for (int32_t kk = 0; kk < min(depth, nmine); ++kk) {
      mbar_arrive_expect_tx(ring.bars + s2, box_bytes);
      tma_load_2d(ring.slots + (size_t)s2 * ring.slot_floats, D.tmap, xcol, ybase + (warp + kk * nwarps) * SB,
                  ring.bars + s2);
      s2 = (s2 + 1 == depth) ? 0 : s2 + 1;
    }
  }
  bool ok = true;
  for (int32_t kk = 0; kk < nmine; ++kk) {
    const int32_t box0 = (warp + kk * nwarps) * SB;  // first row of the box, relative to r0
    if (!mbar_wait_bounded(ring.bars + slot, par)) {
      ok = false;
      int s2 = slot;
      uint32_t p2 = par;
      for (int32_t k2 = kk + 1; k2 < min(kk + depth, nmine); ++k2) {
        s2 = (s2 + 1 == depth) ? 0 : s2 + 1;
        if (s2 == 0) p2 ^= 1u;
        mbar_wait_bounded(ring.bars + s2, p2);
      }
      break;
    }
    const TA* stage = reinterpret_cast<const TA*>(ring.slots + (size_t)slot * ring.slot_floats);
    const int32_t nr_box = min(SB, nrows - box0);
    // Stream output index of (row, pair) = row * kp + hp + 1; the next round's is RB * kp further on.
    const uint64_t idx0 = (uint64_t)(r0 + box0 + r) * (uint64_t)kp + (uint64_t)hp + 1ull;
    uint64_t z = D.seed + idx0 * kSplitMixGamma;
    const uint64_t dz = (uint64_t)(RB * kp) * kSplitMixGamma;
    if (full_lanes && nr_box == SB) {
      if (single) {
        for (int hb = 0; hb < D.mb; ++hb, z += dz)
          lr_round<NC, false, TA, 1>(D, z, rot, flip, stage + (hb * RB + r) * NC, base, bv, LW);
      } else {
        for (int hb = 0; hb < D.mb; ++hb, z += dz)
          lr_round<NC, false, TA, 2>(D, z, rot, flip, stage + (hb * RB + r) * NC, base, bv, LW);
      }
    } else {
      for (int hb = 0; hb < D.mb; ++hb, z += dz) {
        const int rr = hb * RB + r;  // row of the box
        if (r < RB && rr < nr_box) {
          if (single) lr_round<NC, true, TA, 1>(D, z, rot, flip, stage + rr * NC, base, bv, LW);
          else lr_round<NC, true, TA, 2>(D, z, rot, flip, stage + rr * NC, base, bv, LW);
        }
      }
    }
    __syncwarp();
    if (lane == 0 && kk + depth < nmine) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(ring.bars + slot, box_bytes);
      tma_load_2d(ring.slots + (size_t)slot * ring.slot_floats, D.tmap, xcol,
                  ybase + (warp + (kk + depth) * nwarps) * SB, ring.bars + slot);
    }
    slot = (slot + 1 == depth) ? 0 : slot + 1;
    if (slot == 0) par ^= 1u;
  }
  ring.uses += (uint32_t)nmine;
  return ok;
}

// Vector path (n = 1): the accumulator is one FP32 value per target row, acc[jl*B + s], so the lanes
// of an access spread over the banks with their (pseudo-random) targets. Each thread takes rows
// r0 + tid, r0 + tid + blockDim, ... of the work item, loads the row's value (consecutive threads
// read consecutive rows), evaluates the row's stream outputs for blocks j0 .. j0+kbe-1 and adds the
// signed value into each block's target. Rows whose value is zero add nothing and are skipped.
template <typename TA>
__device__ __forceinline__ void tile_scatter_vec(const TileDesc& D, int64_t r0, int64_t r1, int32_t j0, int32_t kbe,
                                                 float* acc) {
  const uint32_t acc_s = (uint32_t)__cvta_generic_to_shared(acc);
  const TA* A = static_cast<const TA*>(D.A);
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const uint32_t a = __float_as_uint(ld_a(A + (i - D.row_base) * D.lda));
    if ((a << 1) == 0u) continue;
    uint64_t h = 0;
    for (int jl = 0; jl < kbe; ++jl) {
      const int j = j0 + jl;
      if (jl == 0 || (j & 1) == 0) h = row_pair_bits(D.seed, (uint64_t)i, D.kp, (uint32_t)j >> 1);
      const uint32_t w = block_word(h, (uint32_t)j);
      const uint32_t line = (uint32_t)jl * D.B + word_to_slot(w, D.B);
      red_shared_f32(acc_s + 4u * line, __uint_as_float(a ^ (w << 31)));
    }
  }
}

// Dispatch: the vector or lane-row path when the host set it up, else on the passes per row of the
// work item (blocks per lane group) for the unrolled path.
template <typename TA>
__device__ __forceinline__ bool tile_scatter_typed(const TileDesc& D, int64_t r0, int64_t r1, int32_t g, int32_t j0,
                                                   int32_t kbe, float* acc, uint32_t* wbuf, WarpRing& ring, int warp,
                                                   int nwarps) {
  if (D.vec) {
    if (D.n != 1 || D.log2NC != 2) return false;
    tile_scatter_vec<TA>(D, r0, r1, j0, kbe, acc);
    return true;
  }
  if (D.lr) {
    // Set up by the host only for one block group with a tensor map; refuse anything else, since its
    // boxes would not match what the host encoded.
    if (D.tmap == nullptr || j0 != 0 || kbe != (int32_t)D.k) return false;
    switch (D.log2NC) {
      case 2: return tile_scatter_lr<4, TA>(D, r0, r1, g, acc, ring, warp, nwarps);
      case 3: return tile_scatter_lr<8, TA>(D, r0, r1, g, acc, ring, warp, nwarps);
      case 4: return tile_scatter_lr<16, TA>(D, r0, r1, g, acc, ring, warp, nwarps);
      case 5: return tile_scatter_lr<32, TA>(D, r0, r1, g, acc, ring, warp, nwarps);
      default: return false;
    }
  }
  const int G = 32 >> D.log2NC;
  const int ppr = (kbe >= G) ? (kbe + G - 1) / G : 0;
  // Boxes of several hash rounds (mb > 1) are only set up by the host when every work item takes the
  // fast path; anything else would wait for bytes that never come, so refuse it.
  if (D.tmap != nullptr && D.mb > 1 && !(ppr == 1 || ppr == 2 || ppr == 4 || ppr == 8)) return false;
  if (D.tmap != nullptr) {
    switch (ppr) {
      case 1: return tile_scatter_tma<1, TA>(D, r0, r1, g, j0, kbe, acc, wbuf, ring, warp, nwarps);
      case 2: return tile_scatter_tma<2, TA>(D, r0, r1, g, j0, kbe, acc, wbuf, ring, warp, nwarps);
      case 4: return tile_scatter_tma<4, TA>(D, r0, r1, g, j0, kbe, acc, wbuf, ring, warp, nwarps);
      case 8: return tile_scatter_tma<8, TA>(D, r0, r1, g, j0, kbe, acc, wbuf, ring, warp, nwarps);
      default: break;
    }
  }
  return tile_scatter_t<0, TA>(D, r0, r1, g, j0, kbe, acc, wbuf, ring, warp, nwarps);
}

// Scale and (FP16 rules) quantize four consecutive columns of output row r (chunk t): x = fl32(scale
// * v) for FP32, else the binary16 values of the rule with one Philox call giving the four uniforms
// (paper Sec. 4.2).
template <int RULE>
__device__ __forceinline__ void scale_quad(const TileDesc& D, uint32_t r, int64_t col0, float4 v, int64_t t, float x[4],
                                           uint16_t q[4]) {
  x[0] = __fmul_rn(D.scale, v.x);
  x[1] = __fmul_rn(D.scale, v.y);
  x[2] = __fmul_rn(D.scale, v.z);
  x[3] = __fmul_rn(D.scale, v.w);
  if (RULE != kFP32) {
    float u[4] = {0.f, 0.f, 0.f, 0.f};
    if (rule_draws_bits<RULE>()) {
      // Columns col_off + col0 .. +3 of the global column space; their uniforms come from at most
      // two Philox calls (words (column mod 4) of counter column quad floor(column / 4)).
      const int64_t cg = D.col_off + col0;
      if ((cg & 3) == 0) {
        uniforms4(D.seed, r, (uint32_t)(cg >> 2), (uint64_t)t, u);
      } else {
        float ua[4], ub[4];
        uniforms4(D.seed, r, (uint32_t)(cg >> 2), (uint64_t)t, ua);
        uniforms4(D.seed, r, (uint32_t)(cg >> 2) + 1u, (uint64_t)t, ub);
        const int o = (int)(cg & 3);
#pragma unroll
        for (int e = 0; e < 4; ++e) u[e] = (o + e < 4) ? ua[o + e] : ub[o + e - 4];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) q[e] = quantize16<RULE>(x[e], u[e]);
  }
}

// Scale, quantize and add four consecutive columns of output row r (chunk t) into Y: FP32 adds use
// one 16-byte vector reduction, FP16 adds two packed half2 atomics (paper Listing 2).
template <int RULE>
__device__ __forceinline__ void emit_quad(const TileDesc& D, uint32_t r, int64_t col0, float4 v, int64_t t) {
  const int64_t n = D.n;
  float x[4];
  uint16_t q[4];
  scale_quad<RULE>(D, r, col0, v, t, x, q);
  if (RULE == kFP32) {
    float* y = reinterpret_cast<float*>(D.Y) + (int64_t)r * n + col0;
    if ((n & 3) == 0 && col0 + 3 < n) {
      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y), "f"(x[0]), "f"(x[1]), "f"(x[2]),
                   "f"(x[3])
                   : "memory");
    } else {
      atomicAdd(y, x[0]);
      if (col0 + 1 < n) atomicAdd(y + 1, x[1]);
      if (col0 + 2 < n) atomicAdd(y + 2, x[2]);
      if (col0 + 3 < n) atomicAdd(y + 3, x[3]);
    }
  } else {
    uint16_t* y = reinterpret_cast<uint16_t*>(D.Y) + (int64_t)r * n + col0;
    if ((n & 1) == 0) {
      atomic_add16x2<RULE>(y, q[0], q[1]);  // col0 + 1 < n since n even
      if (col0 + 3 < n) atomic_add16x2<RULE>(y + 2, q[2], q[3]);
    } else {
      atomic_add16<RULE>(y, q[0]);
      if (col0 + 1 < n) atomic_add16<RULE>(y + 1, q[1]);
      if (col0 + 2 < n) atomic_add16<RULE>(y + 2, q[2]);
      if (col0 + 3 < n) atomic_add16<RULE>(y + 3, q[3]);
    }
  }
}

// Finish the chunks [t_first, t_first + chunks) of one output quad (row r, columns col0 .. col0+3):
// in ascending chunk order, read the chunk total from P (chunk-major, d x n each), clear it, scale,
// quantize and add it into Y with the rule's arithmetic (binary32 add or binary16 add, round to
// nearest), then write Y back once. Chunk totals that are zero in all four columns add nothing.
template <int RULE>
__device__ __forceinline__ void finish_quad(const TileDesc& D, uint32_t r, int64_t col0, float* P, int64_t t_first,
                                            int64_t chunks, int64_t dn) {
  const int64_t n = D.n;
  const int ne = (int)min((int64_t)4, n - col0);
  const bool vec = (n & 3) == 0;
  const int64_t off = (int64_t)r * n + col0;                         // in P (d x n per chunk)
  const int64_t offy = (int64_t)r * (D.ldy > 0 ? D.ldy : n) + col0;  // in Y
  float yf[4] = {0.f, 0.f, 0.f, 0.f};
  uint16_t yh[4] = {0, 0, 0, 0};
  bool loaded = false, touched = false;
  for (int64_t tl = 0; tl < chunks; ++tl) {
    float* p = P + tl * dn + off;
    float4 v;
    if (vec) {
      v = __ldcg(reinterpret_cast<const float4*>(p));
    } else {
      v.x = __ldcg(p);
      v.y = ne > 1 ? __ldcg(p + 1) : 0.f;
      v.z = ne > 2 ? __ldcg(p + 2) : 0.f;
      v.w = ne > 3 ? __ldcg(p + 3) : 0.f;
    }
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
    if (vec) {
      __stcg(reinterpret_cast<float4*>(p), make_float4(0.f, 0.f, 0.f, 0.f));
    } else {
      for (int e = 0; e < ne; ++e) __stcg(p + e, 0.f);
    }
    if (!loaded) {
      loaded = true;
      if (RULE == kFP32) {
        const float* y = reinterpret_cast<const float*>(D.Y) + offy;
        for (int e = 0; e < ne; ++e) yf[e] = y[e];
      } else {
        const uint16_t* y = reinterpret_cast<const uint16_t*>(D.Y) + offy;
        for (int e = 0; e < ne; ++e) yh[e] = y[e];
      }
    }
    float x[4];
    uint16_t q[4];
    scale_quad<RULE>(D, r, col0, v, t_first + tl, x, q);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (e < ne) {
        if (RULE == kFP32) yf[e] = __fadd_rn(yf[e], x[e]);
        else yh[e] = add16<RULE>(yh[e], q[e]);
      }
    }
    touched = true;
  }
  if (!touched) return;
  if (RULE == kFP32) {
    float* y = reinterpret_cast<float*>(D.Y) + offy;
    for (int e = 0; e < ne; ++e) y[e] = yf[e];
  } else {
    uint16_t* y = reinterpret_cast<uint16_t*>(D.Y) + offy;
    for (int e = 0; e < ne; ++e) y[e] = yh[e];
  }
}

// Visit the accumulator quads of a work item: f in [0, kbe*B*NC/4) -> (smem pointer, row, col0).
struct QuadIter {
  int nq, S, LW, NC;
  uint32_t B;
  __device__ __forceinline__ void at(int64_t f, int32_t g, int32_t j0, float* acc, float*& p, uint32_t& r,
                                     int64_t& col0) const {
    const int c4 = (int)(f % nq);
    const int64_t rest = f / nq;
    const uint32_t s = (uint32_t)(rest % B);
    const int jl = (int)(rest / B);
    p = &acc[((jl / S) * (int64_t)B + s) * LW + (jl % S) * NC + 4 * c4];
    r = (uint32_t)(j0 + jl) * B + s;
    col0 = (int64_t)g * NC + 4 * c4;
  }
};

__device__ __forceinline__ QuadIter quad_iter(const TileDesc& D) {
  QuadIter it;
  it.NC = 1 << D.log2NC;
  it.nq = it.NC >> 2;
  it.S = D.S;
  it.LW = D.S * it.NC;
  it.B = D.B;
  return it;
}

// Flush a work item that holds a whole chunk: quantize and add into Y, zero the accumulator.
// Quads whose four partial sums are all zero are skipped (adding a quantized zero leaves Y as is).
template <int RULE>
__device__ __forceinline__ void tile_flush(const TileDesc& D, int64_t t, int32_t g, int32_t j0, int32_t kbe,
                                           float* acc) {
  if (D.vec) {
    // one value per target row (n = 1)
    for (int64_t f = threadIdx.x; f < (int64_t)kbe * D.B; f += blockDim.x) {
      const float v = acc[f];
      if (v == 0.f) continue;
      acc[f] = 0.f;
      emit_quad<RULE>(D, (uint32_t)j0 * D.B + (uint32_t)f, 0, make_float4(v, 0.f, 0.f, 0.f), t);
    }
    return;
  }
  const QuadIter it = quad_iter(D);
  const int64_t total = (int64_t)kbe * D.B * it.nq;
  for (int64_t f = threadIdx.x; f < total; f += blockDim.x) {
    float* p;
    uint32_t r;
    int64_t col0;
    it.at(f, g, j0, acc, p, r, col0);
    const float4 v = *reinterpret_cast<float4*>(p);
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
    *reinterpret_cast<float4*>(p) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col0 >= D.n) continue;
    emit_quad<RULE>(D, r, col0, v, t);
  }
}

// Flush a slice of a chunk: add the FP32 partials into the chunk buffer P (d x n, row stride n),
// zero the accumulator.
__device__ __forceinline__ void tile_flush_partial(const TileDesc& D, int32_t g, int32_t j0, int32_t kbe, float* acc,
                                                   float* P) {
  if (D.vec) {
    for (int64_t f = threadIdx.x; f < (int64_t)kbe * D.B; f += blockDim.x) {
      const float v = acc[f];
      if (v == 0.f) continue;
      acc[f] = 0.f;
      atomicAdd(P + ((int64_t)j0 * D.B + f) * D.n, v);
    }
    return;
  }
  const QuadIter it = quad_iter(D);
  const int64_t total = (int64_t)kbe * D.B * it.nq;
  const int64_t n = D.n;
  for (int64_t f = threadIdx.x; f < total; f += blockDim.x) {
    float* p;
    uint32_t r;
    int64_t col0;
    it.at(f, g, j0, acc, p, r, col0);
    const float4 v = *reinterpret_cast<float4*>(p);
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
    *reinterpret_cast<float4*>(p) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col0 >= n) continue;
    float* y = P + (int64_t)r * n + col0;
    if ((n & 3) == 0 && col0 + 3 < n) {
      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                   : "memory");
    } else {
      atomicAdd(y, v.x);
      if (col0 + 1 < n) atomicAdd(y + 1, v.y);
      if (col0 + 2 < n) atomicAdd(y + 2, v.z);
      if (col0 + 3 < n) atomicAdd(y + 3, v.w);
    }
  }
}

}  // namespace sk
