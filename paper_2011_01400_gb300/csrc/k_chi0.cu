// Tensor-core (tcgen05) chi0 of step (b), Eq. chi0_matrix (Hermitised, occupations restored):
//
//   C_t[mu][nu] = scale * sum_r v_t(r) M^mu_r conj(M^nu_r),
//
// r = (k, i occ, a unocc) pair rows, v_t the Lorentzian weights 2D/(w^2 + D^2) of one frequency or
// one row of their compressed basis. In real form, with a = v_t M^mu (the weighted side) and
// b = M^nu, interleaving (re, im) along K:
//   Re C = sum (a_re b_re + a_im b_im) = A1 . B,   A1 row = (a_re, a_im)
//   Im C = sum (a_im b_re - a_re b_im) = A2 . B,   A2 row = (a_im, -a_re)
//   B row = (b_re, b_im): the M plane itself.
// One MMA with M = 128 = [A1 of 64 mu; A2 of the same 64 mu] against N <= 128 nu rows of B gives
// Re (TMEM lanes 0-63) and Im (lanes 64-127) of a 64 x N complex tile. Each weighted and split A
// row thus feeds 2 x N MMA columns, and B needs no second, permuted copy.
//
// Operand splits (the same pieces on both sides; products of combined order below the fp32
// accumulation are dropped):
//   F16  (GW_3XFP16): x s = h + l 2^-11 with h = fp16(x s), l = fp16((x s - h) 2^11); products
//        hh, hl, lh. s is a power of two per operand (one for the B plane, one per weight row on
//        the A side) that puts the largest |x s| in [2^13, 2^14): h and l then keep 11 bits each
//        for every entry down to 2^-27 of the largest, and the scales are removed exactly in FP64.
//   BF16 (GW_3XBF16): h + m + l, three bf16 pieces; products hh, hm, mh, hl, lh, mm.
//   TF32 (GW_3XTF32): h = x rounded to 10 explicit mantissa bits, l = x - h; products hh, hl, lh.
//
// Accumulation: the hh products go to accumulator D1, drained after every stage (4 MMAs per
// output) into fp32 running sums held by the epilogue warps (round to nearest), since the tensor
// core's fp32 accumulator truncates every addition; the correction products go to D2, drained once
// per segment of F stages. After each segment the sums are added in FP64 (red.global.add) into
// C_t, so a work item may cover any run of whole segments (K is split across work items).
//
// Tiles: mu blocks of 64 rows aligned to the last row (the first block may be short), nu chunks
// of at most 128 columns covering the lower triangle nu < end of the block; C's upper triangle is
// filled from the lower one afterwards. Work items (tile, K chunk, weight row) are assigned to the
// persistent CTAs on the host, longest first to the least loaded CTA.
//
// Roles (736 threads):
//   warp 0 (TMA):      B pieces, 128 rows x 128 B each per stage, SWIZZLE_128B
//   warp 22 (TMA):     raw fp32 A rows, 64 rows x 128 B per ring slot, with the slot's 16 weights
//   warps 2-5:         transform: y = v x from the ring, split, write A1 / A2 pieces in the UMMA
//                      K-major 128B-swizzled layout
//   warp 1:            one elected thread issues tcgen05.mma (M = 128, N = tile columns)
//   warps 6-21:        epilogue (four warps per TMEM lane quadrant, 32 columns each)
// All mbarrier waits are bounded; on expiry the kernel sets ST_TIMEOUT and unwinds.
#include "gw_internal.h"
#include "tc_ptx.cuh"

#include <algorithm>
#include <array>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

namespace gw {

namespace {

using namespace ptx;

constexpr int BMU = 64;                  // mu rows per tile
constexpr int BNU = 128;                 // nu columns per tile (at most)
constexpr int TILE = 128 * ROWB;         // 16 KB: one piece of A ([A1; A2]) or B (128 rows)
constexpr int SLOT = BMU * ROWB;         // 8 KB: raw ring slot, 64 rows x 32 floats (16 complex pairs)
constexpr int WBYTES = 16 * 4;           // the weights of a slot's 16 pair rows (one weight row)
constexpr int NTHREADS = 736;           // 23 warps (roles below)
constexpr uint32_t DBUF = 128;           // TMEM columns of one accumulator buffer
constexpr int LSH = 11;                  // F16: the low piece is scaled by 2^11
constexpr int TP_F16 = 1, TP_TF32 = 1;   // weight rows per work item (measured: 2 is slower)

enum { K_F16 = 0, K_BF16 = 1, K_TF32 = 2 };

// Shared memory: a ring of SB B stages (TMA runs up to SB - 1 stages ahead of the MMAs, which
// covers the L2 / HBM latency), SA buffers of split A pieces (written by the transform just in
// time), and the raw-row ring of RING slots with their weights.
// TP weight rows per work item share the loaded operands: the raw A rows and the B rows of a
// stage are loaded once and feed TP weighted A operands (each its own NT = 128 / TP accumulator
// columns), so with TP = 2 a stage of the same MMA work loads 32 KB instead of 48 KB (F16: B
// rows 2 x 64 instead of 2 x 128, raw rows unchanged), for twice the transform work per raw row
// and twice the MMA instructions. Measured, TP = 2 is slower: the kernel is paced by its issue
// loop (MMA issue, waits and commit per stage), not by the operand stream.
template <int KIND, int TP> struct Kd {
  static constexpr int NP = (KIND == K_BF16) ? 3 : 2;       // pieces per operand
  static constexpr int ESZ = (KIND == K_TF32) ? 4 : 2;      // bytes per element
  static constexpr int RPS = (KIND == K_TF32) ? 1 : 2;      // ring slots per stage
  static constexpr int RS = 16 * RPS;                       // complex pair rows per stage
  static constexpr int NT = BNU / TP;                       // nu columns per weight row
  static constexpr int BST = NP * NT * ROWB;                // one B stage (NT rows per piece)
  static constexpr int AST = TP * NP * TILE;                // one A buffer (TP weighted operands)
  // Stage s of the pipeline owns B buffer s, A buffer s and D1 accumulator s (DEPTH of each): one
  // commit per stage tells the B producer, the transform and the epilogue that the stage's MMAs
  // are done. D2 (per segment) takes the rest of TMEM.
  static constexpr int DEPTH = (KIND == K_BF16) ? 2 : 3;
  static constexpr int SB = DEPTH, SA = DEPTH, NB1 = DEPTH;  // B stages, A buffers, D1 buffers
  static constexpr int NB2 = 4 - DEPTH;                      // D2 buffers (TMEM: 4 x 128 columns)
  static constexpr uint32_t D1_COL = 0, D2_COL = NB1 * DBUF;
  static constexpr int RING = (KIND == K_BF16) ? 2 : 4;     // raw ring slots
  static constexpr int A_OFF = SB * BST;
  static constexpr int RING_OFF = A_OFF + SA * AST;
  static constexpr int WB_OFF = RING_OFF + RING * SLOT;
  static constexpr int BAR_OFF = WB_OFF + RING * TP * WBYTES;
  static constexpr int BARS = 8 * (4 * DEPTH + 2 * NB2 + 1 + 2 * RING) + 16;   // + TMEM address
  static constexpr int SMEM = BAR_OFF + BARS + 1024;
};

struct Tile {
  int m0, mhi;     // mu rows [m0, m0 + 64) loaded; rows [m0, mhi) owned by this tile
  int n0, ncols;   // nu columns [n0, n0 + ncols), ncols a multiple of 16 (<= 128)
};

struct Chi0Params {
  int N;
  int nst;              // stages over the padded pair rows
  int seg;              // stages per promotion segment
  int nchunk;           // K chunks (runs of whole segments) per tile
  const Tile* tiles;
  const int* items;     // item = (tile * nchunk + chunk) * TG + g (weight rows g TP ..), grouped per CTA
  const int* cta_off;   // [gridDim.x + 1] range of each CTA in items
  int T;                // weight rows (or batch entries)
  int TG;               // groups of TP consecutive weight rows: ceil(T / TP)
  const float* wtab;    // [T][wstride] weights (F16: already multiplied by the row's scale)
  long long wstride;
  const double* escale; // [T] factor applied to the drained sums (scale, and the F16 scales undone)
  double* out;          // [T][N][N] complex as (re, im) doubles, lower triangle accumulated
  int* status;
  int lower;            // 1: lower triangle only (Hermitian result); 0: every element
  int store;            // 1: one K chunk of one segment per output, written with plain stores (no
                        //    zeroing, no atomics); 0: FP64 atomic accumulation
  int a_bstride;        // A rows of weight row / batch entry t start at t * a_bstride
  int b_bstride;        // B rows of t start at t * b_bstride
};

struct Chi0Maps {
  CUtensorMap b[3];     // B pieces
  CUtensorMap raw;      // fp32 plane, 32 floats x 64 rows per box
};

// t: the first weight row of the item's group (TP consecutive rows, those >= T are not computed)
template <int TP>
__device__ __forceinline__ void decode(const Chi0Params& p, int item, Tile& tl, int& t, int& s0, int& s1) {
  t = (item % p.TG) * TP;
  const int tc = item / p.TG;
  tl = p.tiles[tc / p.nchunk];
  const int c = tc % p.nchunk;
  const int nseg = (p.nst + p.seg - 1) / p.seg;
  s0 = (int)((long long)c * nseg / p.nchunk) * p.seg;
  s1 = min(p.nst, (int)((long long)(c + 1) * nseg / p.nchunk) * p.seg);
}

__device__ __forceinline__ uint32_t swap_neg(uint32_t v) {   // (lo, hi) -> (hi, -lo) for 16-bit pairs
  return __byte_perm(v, 0, 0x1032) ^ 0x80000000u;
}
__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ uint32_t b2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// 32 lanes x 16 consecutive 32-bit TMEM columns
__device__ __forceinline__ void tld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// acc[j] += f * D[t + j] for this thread's 32 columns (both loads in flight, one wait)
__device__ __forceinline__ void drain(uint32_t t, float f, float (&acc)[32]) {
  uint32_t a[16], b[16];
  tld16(t, a);
  tld16(t + 16, b);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    acc[j] = fmaf(f, __uint_as_float(a[j]), acc[j]);
    acc[16 + j] = fmaf(f, __uint_as_float(b[j]), acc[16 + j]);
  }
}

template <int KIND>
__device__ __forceinline__ void mma_k(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  mma<KIND == K_TF32>(d, a, b, idesc, acc);
}

template <int KIND, int TP>
__global__ void __launch_bounds__(NTHREADS, 1) k_chi0(const __grid_constant__ Chi0Maps maps, Chi0Params p) {
  using C = Kd<KIND, TP>;
  static_assert(C::SMEM <= 232448, "shared memory budget");
  static_assert((C::NB1 + C::NB2) * DBUF <= 512, "TMEM budget");
  constexpr int NP = C::NP, SB = C::SB, SA = C::SA, BST = C::BST, AST = C::AST, RPS = C::RPS, RING = C::RING;
  constexpr int NT = C::NT, NB1 = C::NB1, NB2 = C::NB2, DEPTH = C::DEPTH;
  constexpr uint32_t D1_COL = C::D1_COL, D2_COL = C::D2_COL;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem + C::RING_OFF;
  float* wbuf = reinterpret_cast<float*>(smem + C::WB_OFF);   // [RING][TP][16]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  uint64_t* full_b = bars;                        // [DEPTH] B stage landed
  uint64_t* full_a = bars + DEPTH;                // [DEPTH] A buffer written by the transform
  uint64_t* sdone = bars + 2 * DEPTH;             // [DEPTH] the stage's MMAs done: B and A buffers
                                                  // free, D1 of the stage ready
  uint64_t* t1empty = bars + 3 * DEPTH;           // [DEPTH] D1 drained
  uint64_t* t2full = bars + 4 * DEPTH;            // [NB2] D2 of a segment ready
  uint64_t* t2empty = t2full + NB2;               // [NB2] D2 drained
  uint64_t* done = t2full + 2 * NB2;
  uint64_t* rfull = done + 1;                     // [RING]
  uint64_t* rempty = rfull + RING;                // [RING]
  uint32_t* tmem_base_p = reinterpret_cast<uint32_t*>(rempty + RING);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int it0 = p.cta_off[blockIdx.x], it1 = p.cta_off[blockIdx.x + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < DEPTH; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&full_a[s], 4);                 // one elected arrival per transform warp
      mbar_init(&sdone[s], 1);
      mbar_init(&t1empty[s], 16);               // one per epilogue warp
    }
    for (int b = 0; b < NB2; ++b) {
      mbar_init(&t2full[b], 1);
      mbar_init(&t2empty[b], 16);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(&rfull[r], 1);
      mbar_init(&rempty[r], 4 / RPS);           // the transform warps that read the slot
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_base_p, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base_p;
  const int F = p.seg;

  if (warp == 0) {
    // ---------------- TMA producer: B pieces ----------------
    if (lane == 0) {
      uint32_t gs = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok; ++it) {
        Tile tl;
        int t, s0, s1;
        decode<TP>(p, p.items[it], tl, t, s0, s1);
        for (int i = s0; i < s1; ++i, ++gs) {
          const int s = gs % SB;
          if (!mbar_wait(&sdone[s], ((gs / SB) & 1) ^ 1, p.status)) { ok = false; break; }
          uint8_t* st = smem + s * BST;
          mbar_arrive_expect_tx(&full_b[s], BST);
          const int x = i * (ROWB / C::ESZ);
#pragma unroll
          for (int pc = 0; pc < NP; ++pc)
            tma_load_2d(st + pc * NT * ROWB, &maps.b[pc], &full_b[s], x, t * p.b_bstride + tl.n0);
        }
      }
    }
  } else if (warp == 22) {
    // ---------------- TMA producer: raw A rows and their weights into the ring ----------------
    if (lane == 0) {
      uint32_t gr = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok; ++it) {
        Tile tl;
        int t, s0, s1;
        decode<TP>(p, p.items[it], tl, t, s0, s1);
        for (int i = s0 * RPS; i < s1 * RPS; ++i, ++gr) {
          const int slot = gr % RING;
          if (!mbar_wait(&rempty[slot], ((gr / RING) & 1) ^ 1, p.status)) { ok = false; break; }
          mbar_arrive_expect_tx(&rfull[slot], SLOT + TP * WBYTES);
          tma_load_2d(ring + slot * SLOT, &maps.raw, &rfull[slot], i * 32, t * p.a_bstride + tl.m0);
          // pair rows 16 i .. 16 i + 15 of each weight row of the group (16-byte aligned: weight rows
          // are a multiple of 32 floats apart); rows past T repeat the last one (not computed)
#pragma unroll
          for (int u = 0; u < TP; ++u)
            bulk_load(wbuf + (slot * TP + u) * 16, p.wtab + (long long)min(t + u, p.T - 1) * p.wstride + 16 * i,
                      WBYTES, &rfull[slot]);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t fmt = (KIND == K_TF32) ? 2u : (KIND == K_BF16 ? 1u : 0u);
      const uint32_t sbase = smem_u32(smem);
      // ring positions, their phase parities and the accumulator rounds, stepped per stage (no
      // divisions in the issue loop)
      int sb = 0, b2 = 0;                        // stage buffer (B, A and D1), D2 buffer
      uint32_t pb = 0, r2 = 0;                   // stage-round parity, D2 rounds
      bool ok = true;
      for (int it = it0; it < it1 && ok; ++it) {
        Tile tl;
        int t, s0, s1;
        decode<TP>(p, p.items[it], tl, t, s0, s1);
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(tl.ncols >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        const int nt_valid = min(TP, p.T - t);   // weight rows of the group that exist
        int spos = 0;                            // stage within the promotion segment
        for (int i = s0; i < s1; ++i) {
          const bool seg_first = spos == 0;
          const bool seg_end = spos == F - 1 || i == s1 - 1;
          // D1 buffer sb drained one round ago (the first round finds it free)
          if (!mbar_wait(&t1empty[sb], pb ^ 1u, p.status)) { ok = false; break; }
          if (seg_first && r2 > 0 && !mbar_wait(&t2empty[b2], (r2 - 1) & 1, p.status)) { ok = false; break; }
          if (!mbar_wait(&full_b[sb], pb, p.status)) { ok = false; break; }
          if (!mbar_wait(&full_a[sb], pb, p.status)) { ok = false; break; }
          tc_fence_after();
          // K-major SWIZZLE_128B descriptors; a 32-byte K step adds 2 to the address field
          const uint64_t dB0 = sdesc(sbase + sb * BST), dB1 = sdesc(sbase + sb * BST + NT * ROWB);
#pragma unroll
          for (int u = 0; u < TP; ++u) {
            if (u >= nt_valid) break;
            const uint32_t abase = sbase + C::A_OFF + sb * AST + u * NP * TILE;
            const uint64_t dA0 = sdesc(abase), dA1 = sdesc(abase + TILE);
            const uint32_t d1 = tmem + D1_COL + sb * DBUF + u * NT;
            const uint32_t d2 = tmem + D2_COL + b2 * DBUF + u * NT;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ko = (uint64_t)(2 * kk);
              const uint32_t acc2 = (seg_first && kk == 0) ? 0u : 1u;
              const uint64_t A0 = dA0 + ko, B0 = dB0 + ko, A1 = dA1 + ko, B1 = dB1 + ko;
              mma_k<KIND>(d2, A0, B1, idesc, acc2);
              mma_k<KIND>(d2, A1, B0, idesc, 1u);
              if constexpr (NP == 3) {
                const uint64_t A2 = sdesc(abase + 2 * TILE) + ko, B2 = sdesc(sbase + sb * BST + 2 * NT * ROWB) + ko;
                mma_k<KIND>(d2, A0, B2, idesc, 1u);
                mma_k<KIND>(d2, A2, B0, idesc, 1u);
                mma_k<KIND>(d2, A1, B1, idesc, 1u);
              }
              mma_k<KIND>(d1, A0, B0, idesc, kk == 0 ? 0u : 1u);
            }
          }
          mma_commit(&sdone[sb]);
          if (seg_end) {
            mma_commit(&t2full[b2]);
            if (++b2 == NB2) { b2 = 0; ++r2; }
          }
          if (++sb == DEPTH) { sb = 0; pb ^= 1u; }
          spos = seg_end ? 0 : spos + 1;
        }
      }
      mma_commit(done);
      mbar_wait(done, 0, p.status);
    }
  } else if (warp >= 2 && warp <= 5) {
    // ---------------- transform: weighted, split A1 / A2 pieces ----------------
    const int tid = threadIdx.x - 64;          // 0..127
    const int row = tid & 63;                  // mu row within the tile
    const int h = tid >> 6;                    // BF16 / F16: ring slot of the stage; TF32: half of the slot
    uint32_t gs = 0, gr = 0;
    bool ok = true;
    for (int it = it0; it < it1 && ok; ++it) {
      Tile tl;
      int t, s0, s1;
      decode<TP>(p, p.items[it], tl, t, s0, s1);
      for (int i = s0; i < s1; ++i, ++gs, gr += RPS) {
        const int s = gs % SA;
        // warp-uniform waits: the arrivals below are elected per warp
        if (!__all_sync(0xffffffffu, mbar_wait(&sdone[s], ((gs / SA) & 1) ^ 1, p.status))) { ok = false; break; }
        uint8_t* at = smem + C::A_OFF + s * AST;
        const uint32_t g = gr + (RPS == 2 ? h : 0);
        const int slot = g % RING;
        if (!__all_sync(0xffffffffu, mbar_wait(&rfull[slot], (g / RING) & 1, p.status))) { ok = false; break; }
        const uint8_t* rs = ring + slot * SLOT;
        const float* wslot = wbuf + slot * TP * 16;
        if constexpr (KIND == K_TF32) {
          // 8 pairs [8h, 8h + 8) of the slot: raw chunks 4h .. 4h + 3, A chunks 4h .. 4h + 3 (2 pairs each)
          float x[16], wv[TP][8];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(rs + swz(row, 4 * h + c));
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
#pragma unroll
          for (int u = 0; u < TP; ++u)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const float4 v = reinterpret_cast<const float4*>(wslot + 16 * u + 8 * h)[c];
              wv[u][4 * c] = v.x;
              wv[u][4 * c + 1] = v.y;
              wv[u][4 * c + 2] = v.z;
              wv[u][4 * c + 3] = v.w;
            }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&rempty[slot]);
#pragma unroll
          for (int u = 0; u < TP; ++u)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint8_t* au = at + u * NP * TILE;
            uint32_t h1[4], l1[4], h2[4], l2[4];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const float wt = wv[u][2 * c + q];
              const float yr = wt * x[4 * c + 2 * q], yi = wt * x[4 * c + 2 * q + 1];
              const float hr = tf32_rn(yr), hi = tf32_rn(yi);
              const float lr = yr - hr, li = yi - hi;
              h1[2 * q] = __float_as_uint(hr);
              h1[2 * q + 1] = __float_as_uint(hi);
              l1[2 * q] = __float_as_uint(lr);
              l1[2 * q + 1] = __float_as_uint(li);
              h2[2 * q] = __float_as_uint(hi);
              h2[2 * q + 1] = __float_as_uint(-hr);
              l2[2 * q] = __float_as_uint(li);
              l2[2 * q + 1] = __float_as_uint(-lr);
            }
            const uint32_t o1 = swz(row, 4 * h + c), o2 = swz(row + 64, 4 * h + c);
            *reinterpret_cast<uint4*>(au + o1) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
            *reinterpret_cast<uint4*>(au + o2) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
            *reinterpret_cast<uint4*>(au + TILE + o1) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
            *reinterpret_cast<uint4*>(au + TILE + o2) = make_uint4(l2[0], l2[1], l2[2], l2[3]);
          }
        } else {
          // the slot's 16 pairs of this row: raw chunks 0..7; A chunks 4h .. 4h + 3 (4 pairs each)
          float x[32], wv[TP][16];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(rs + swz(row, c));
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
#pragma unroll
          for (int u = 0; u < TP; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float4 v = reinterpret_cast<const float4*>(wslot + 16 * u)[c];
              wv[u][4 * c] = v.x;
              wv[u][4 * c + 1] = v.y;
              wv[u][4 * c + 2] = v.z;
              wv[u][4 * c + 3] = v.w;
            }
          // order these generic-proxy reads before the TMA (async-proxy) refill of the slot
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&rempty[slot]);
#pragma unroll
          for (int u = 0; u < TP; ++u)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            uint8_t* au = at + u * NP * TILE;
            uint32_t o[NP][4], o2[NP][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int pr = 4 * cc + q;
              const float wt = wv[u][pr];
              const float yr = wt * x[2 * pr], yi = wt * x[2 * pr + 1];
              if constexpr (KIND == K_F16) {
                const __half2 hh = __floats2half2_rn(yr, yi);
                const float2 hf = __half22float2(hh);
                const __half2 ll = __floats2half2_rn((yr - hf.x) * (float)(1 << LSH), (yi - hf.y) * (float)(1 << LSH));
                o[0][q] = h2_bits(hh);
                o[1][q] = h2_bits(ll);
              } else {
                const __nv_bfloat162 hh = __floats2bfloat162_rn(yr, yi);
                const float2 hf = __bfloat1622float2(hh);
                const float rr = yr - hf.x, ri = yi - hf.y;
                const __nv_bfloat162 mm = __floats2bfloat162_rn(rr, ri);
                const float2 mf = __bfloat1622float2(mm);
                const __nv_bfloat162 ll = __floats2bfloat162_rn(rr - mf.x, ri - mf.y);
                o[0][q] = b2_bits(hh);
                o[1][q] = b2_bits(mm);
                o[NP - 1][q] = b2_bits(ll);
              }
#pragma unroll
              for (int pc = 0; pc < NP; ++pc) o2[pc][q] = swap_neg(o[pc][q]);
            }
            const uint32_t off1 = swz(row, 4 * h + cc), off2 = swz(row + 64, 4 * h + cc);
#pragma unroll
            for (int pc = 0; pc < NP; ++pc) {
              *reinterpret_cast<uint4*>(au + pc * TILE + off1) = make_uint4(o[pc][0], o[pc][1], o[pc][2], o[pc][3]);
              *reinterpret_cast<uint4*>(au + pc * TILE + off2) =
                  make_uint4(o2[pc][0], o2[pc][1], o2[pc][2], o2[pc][3]);
            }
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_a[s]);
      }
    }
  } else if (warp >= 6 && warp <= 21) {
    // ---------------- epilogue: drain D1 per stage, D2 per segment, FP64 flush ----------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
    const int cg = (warp - 6) >> 2;            // TMEM columns 32*cg .. 32*cg+31 of a buffer
    constexpr int CPT = 4 / TP;                // column groups per weight row
    const int u = cg / CPT;                    // weight row t + u of the item's group
    const int cw = 32 * (cg % CPT);            // first tile column of the group
    const int lrow = quad * 32 + lane;         // TMEM lane: Re (< 64) or Im (>= 64) of mu row lrow & 63
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const float f2 = (KIND == K_F16) ? 1.0f / (float)(1 << LSH) : 1.0f;
    int b = 0, b2 = 0;
    uint32_t r1 = 0, r2 = 0;                   // stage / D2 rounds (phase parities)
    bool ok = true;
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    for (int it = it0; it < it1 && ok; ++it) {
      Tile tl;
      int t, s0, s1;
      decode<TP>(p, p.items[it], tl, t, s0, s1);
      const int ncol = (t + u < p.T) ? max(0, min(32, tl.ncols - cw)) : 0;
      const int mu = tl.m0 + (lrow & 63);
      const int part = lrow >> 6;
      const double es = p.escale[min(t + u, p.T - 1)];
      int spos = 0;
      for (int i = s0; i < s1; ++i) {
        const bool seg_end = spos == F - 1 || i == s1 - 1;
        spos = seg_end ? 0 : spos + 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&sdone[b], r1 & 1, p.status));
        if (!ok) break;
        tc_fence_after();
        // all 64 columns: the ones beyond the tile hold stale values that are never flushed
        drain(tmem + lane_off + D1_COL + b * DBUF + 32 * cg, 1.0f, acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&t1empty[b]);
        if (++b == NB1) { b = 0; ++r1; }
        if (seg_end) {
          ok = __all_sync(0xffffffffu, mbar_wait(&t2full[b2], r2 & 1, p.status));
          if (!ok) break;
          tc_fence_after();
          drain(tmem + lane_off + D2_COL + b2 * DBUF + 32 * cg, f2, acc);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&t2empty[b2]);
          if (++b2 == NB2) { b2 = 0; ++r2; }
          if (mu >= tl.m0 && mu < tl.mhi) {
            const int c0 = tl.n0 + cw;
            double* o = p.out + 2 * (((long long)(t + u) * p.N + mu) * p.N + c0) + part;
            // columns nu = c0 + j of the tile below N (and, for the lower triangle, <= mu)
            const int jmax = min(ncol, (p.lower ? mu + 1 : p.N) - c0);
            if (p.store) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < jmax) o[2 * j] = es * (double)acc[j];
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < jmax) atomicAdd(o + 2 * j, es * (double)acc[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[j] = 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// B pieces of the raw plane [rows][ldk] (elementwise; F16: x 2^eB from the plane's largest |x|)
template <int KIND>
__global__ void k_b_pieces(long long n, const float* __restrict__ raw, const unsigned* __restrict__ absmax,
                           void* p0, void* p1, void* p2, int* eB_out) {
  float s = 1.0f;
  if (KIND == K_F16) {
    int e = 0;
    const float m = __uint_as_float(*absmax);
    if (m > 0.f) frexpf(m, &e);             // m = f 2^e, f in [0.5, 1)
    s = ldexpf(1.0f, 14 - e);                // largest |x s| in [2^13, 2^14)
    if (blockIdx.x == 0 && threadIdx.x == 0) *eB_out = 14 - e;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 y = reinterpret_cast<const float2*>(raw)[e];
    if constexpr (KIND == K_F16) {
      const float yr = y.x * s, yi = y.y * s;
      const __half2 h = __floats2half2_rn(yr, yi);
      const float2 hf = __half22float2(h);
      reinterpret_cast<__half2*>(p0)[e] = h;
      reinterpret_cast<__half2*>(p1)[e] = __floats2half2_rn((yr - hf.x) * (float)(1 << LSH), (yi - hf.y) * (float)(1 << LSH));
    } else if constexpr (KIND == K_BF16) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(y.x, y.y);
      const float2 hf = __bfloat1622float2(h);
      const float r0 = y.x - hf.x, r1 = y.y - hf.y;
      const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
      const float2 mf = __bfloat1622float2(m);
      reinterpret_cast<__nv_bfloat162*>(p0)[e] = h;
      reinterpret_cast<__nv_bfloat162*>(p1)[e] = m;
      reinterpret_cast<__nv_bfloat162*>(p2)[e] = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    } else {
      const float hr = tf32_rn(y.x), hi = tf32_rn(y.y);
      reinterpret_cast<float2*>(p0)[e] = make_float2(hr, hi);
      reinterpret_cast<float2*>(p1)[e] = make_float2(y.x - hr, y.y - hi);
    }
  }
}

// Per weight row t: F16 multiplies the row by 2^eA_t (largest |v_t| |M| s_t in [2^13, 2^14));
// escale[t] = scale 2^-(eA_t + eB) (F16) or scale.
__global__ void k_wscale(int Kpad, int T, float* __restrict__ wtab, const unsigned* __restrict__ absmax,
                         const int* __restrict__ eB, double scale, int f16, double* __restrict__ escale) {
  __shared__ float red[32];
  const int t = blockIdx.x;
  float* w = wtab + (long long)t * Kpad;
  if (!f16) {
    if (threadIdx.x == 0) escale[t] = scale;
    return;
  }
  float m = 0.f;
  for (int r = threadIdx.x; r < Kpad; r += blockDim.x) m = fmaxf(m, fabsf(w[r]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x + 31) / 32) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const float bound = red[0] * __uint_as_float(*absmax);   // >= every |v_t(r) M^mu_r|
  int e = 0;
  if (bound > 0.f) frexpf(bound, &e);
  const int eA = 14 - e;
  const float s = ldexpf(1.0f, eA);
  for (int r = threadIdx.x; r < Kpad; r += blockDim.x) w[r] *= s;
  if (threadIdx.x == 0) escale[t] = ldexp(scale, -(eA + *eB));
}

// wtab[j][r] = 2 D_r / (w_j^2 + D_r^2) for r < K, 0 for the padding rows
__global__ void k_weights_h(int K, int Kpad, int nw, const float* __restrict__ delta, const double* __restrict__ freq,
                            float* __restrict__ wtab) {
  const long long total = (long long)nw * Kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % Kpad), j = (int)(e / Kpad);
    const float d = delta[r];
    const float w = (float)freq[j];
    wtab[e] = r < K ? 2.0f * d / (w * w + d * d) : 0.0f;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// 2-D map over a row-major plane [rows][ld] elements, box = 128 B of one row x box_rows rows, 128B swizzle
bool map2d(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esz, long long ld, long long rows,
           int box_rows, std::string& err) {
  EncodeTiledFn enc = encoder();
  if (!enc) {
    err = "cuTensorMapEncodeTiled is unavailable";
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

// Tiles covering the lower triangle of an N x N matrix: mu blocks of 64 aligned to row N, nu
// chunks of <= nt columns up to the block's last row.
std::vector<Tile> make_tiles(int N, bool lower, int nt) {
  std::vector<Tile> v;
  if (!lower) {
    for (int m0 = 0; m0 < N; m0 += BMU)
      for (int n0 = 0; n0 < N; n0 += nt) {
        const int w = std::min(nt, N - n0);
        v.push_back(Tile{m0, std::min(N, m0 + BMU), n0, (w + 15) / 16 * 16});
      }
    return v;
  }
  for (int mhi = N; mhi > 0; mhi -= BMU) {
    const int m0 = std::max(0, mhi - BMU);
    for (int n0 = 0; n0 < mhi; n0 += nt) {
      const int w = std::min(nt, mhi - n0);
      v.push_back(Tile{m0, mhi, n0, (w + 15) / 16 * 16});
    }
  }
  return v;
}

// relative cost of one stage of a tile for nvalid weight rows: the MMAs scale with the columns
// computed; the stage's fixed part (waits, transform, drain, commits) does not (measured: about
// 1.5x the MMA time of a full 128-column stage)
double tile_cost(const Tile& t, int nvalid) { return 192.0 + (double)(t.ncols * nvalid); }

}  // namespace

// Work lists of one launch shape (N, T, stages, segment length)
struct Chi0Lists {
  int nchunk = 0, grid = 0;
  Tile* d_tiles = nullptr;
  int* d_items = nullptr;
  int* d_off = nullptr;
  ~Chi0Lists() {
    if (d_tiles) cudaFree(d_tiles);
    if (d_items) cudaFree(d_items);
    if (d_off) cudaFree(d_off);
  }
};

// the launch shapes a plan has met (the weight-row count T may differ from one q to the next)
struct Chi0Plan {
  std::map<std::array<int, 5>, Chi0Lists*> lists;
  ~Chi0Plan() {
    for (auto& kv : lists) delete kv.second;
  }
};

void chi0_plan_free(Chi0Plan* p) { delete p; }

// Work lists for (N, T, nst, seg, TP), built once per shape: items (a tile, a K chunk and a group
// of TP weight rows) sorted by cost (longest first; same-cost items of one tile and K chunk stay
// adjacent so that concurrent CTAs share their operands in L2), each given to the least loaded CTA.
static gw_status chi0_lists(Chi0Plan** pp, int N, int T, int nst, int seg, int tp, cudaStream_t st, Chi0Lists** out,
                            std::string& err, bool lower = true) {
  if (!*pp) {
    *pp = new (std::nothrow) Chi0Plan();
    if (!*pp) {
      err = "host allocation failed";
      return GW_ERR_NOMEM;
    }
  }
  const std::array<int, 5> key{lower ? N : -N, T, nst, seg, tp};
  auto f = (*pp)->lists.find(key);
  if (f != (*pp)->lists.end()) {
    *out = f->second;
    return GW_OK;
  }
  Chi0Lists* p = new (std::nothrow) Chi0Lists();
  if (!p) {
    err = "host allocation failed";
    return GW_ERR_NOMEM;
  }
  const std::vector<Tile> tiles = make_tiles(N, lower, BNU / tp);
  const int nsm = sm_count();
  const int nseg = (nst + seg - 1) / seg;
  const int TG = (T + tp - 1) / tp;
  const long long base = (long long)tiles.size() * TG;
  int nchunk = 1;
  while (base * nchunk < 2LL * nsm && nchunk * 2 <= nseg) nchunk *= 2;
  std::vector<std::pair<double, int>> items;
  for (int ti = 0; ti < (int)tiles.size(); ++ti)
    for (int c = 0; c < nchunk; ++c) {
      const int s0 = (int)((long long)c * nseg / nchunk) * seg;
      const int s1 = std::min(nst, (int)((long long)(c + 1) * nseg / nchunk) * seg);
      for (int g = 0; g < TG; ++g)
        items.push_back({tile_cost(tiles[ti], std::min(tp, T - g * tp)) * (s1 - s0), (ti * nchunk + c) * TG + g});
    }
  std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  const int grid = (int)std::min<long long>((long long)items.size(), nsm);
  std::vector<std::vector<int>> per(grid);
  std::vector<double> load(grid, 0.0);
  for (const auto& it : items) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    per[c].push_back(it.second);
    load[c] += it.first;
  }
  std::vector<int> flat, off(grid + 1, 0);
  for (int c = 0; c < grid; ++c) {
    flat.insert(flat.end(), per[c].begin(), per[c].end());
    off[c + 1] = (int)flat.size();
  }
  g_alloc_count += 3;
  if (cudaMalloc(&p->d_tiles, sizeof(Tile) * tiles.size()) != cudaSuccess ||
      cudaMalloc(&p->d_items, sizeof(int) * flat.size()) != cudaSuccess ||
      cudaMalloc(&p->d_off, sizeof(int) * off.size()) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    err = "chi0 work-list allocation failed";
    return GW_ERR_NOMEM;
  }
  // the host vectors die with this call: copy synchronously (once per launch shape)
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(p->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_items, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    delete p;
    err = "chi0 work-list upload failed";
    return GW_ERR_CUDA;
  }
  p->nchunk = nchunk;
  p->grid = grid;
  (*pp)->lists[key] = p;
  *out = p;
  return GW_OK;
}

template <int KIND, int TP>
static gw_status launch_chi0(const Chi0Maps& maps, const Chi0Params& prm, int grid, cudaStream_t st, std::string& err) {
  const int smem = Kd<KIND, TP>::SMEM;
  cudaFuncSetAttribute(k_chi0<KIND, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  ++g_launch_count, k_chi0<KIND, TP><<<grid, NTHREADS, smem, st>>>(maps, prm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("k_chi0 launch: ") + cudaGetErrorString(e);
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

gw_status chi0h_pieces(const Chi0hArgs& a, cudaStream_t st) {
  const long long n = (long long)a.N * a.Kpad;   // complex elements of the plane
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
  if (a.kind == 0)
    ++g_launch_count, k_b_pieces<K_F16><<<grid, 256, 0, st>>>(n, a.raw, a.absmax, a.bpl[0], a.bpl[1], nullptr, a.eB);
  else if (a.kind == 1)
    ++g_launch_count, k_b_pieces<K_BF16><<<grid, 256, 0, st>>>(n, a.raw, a.absmax, a.bpl[0], a.bpl[1], a.bpl[2], a.eB);
  else
    ++g_launch_count, k_b_pieces<K_TF32><<<grid, 256, 0, st>>>(n, a.raw, a.absmax, a.bpl[0], a.bpl[1], nullptr, a.eB);
  return cudaGetLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

gw_status chi0h_run(const Chi0hArgs& a, Chi0Plan** plan, cudaStream_t st, std::string& err) {
  if (a.Kpad % 32 != 0 || a.N < 1 || a.T < 1) {
    err = "chi0: Kpad must be a multiple of 32";
    return GW_ERR_ARG;
  }
  const int RS = (a.kind == 2) ? Kd<K_TF32, 1>::RS : (a.kind == 1 ? Kd<K_BF16, 1>::RS : Kd<K_F16, 1>::RS);
  const int nst = a.Kpad / RS;
  const int seg = std::max(1, a.seg_rows / RS);
  const int tp = a.kind == 0 ? TP_F16 : a.kind == 1 ? 1 : TP_TF32;
  Chi0Lists* P = nullptr;
  gw_status s = chi0_lists(plan, a.N, a.T, nst, seg, tp, st, &P, err);
  if (s != GW_OK) return s;
  // weight-row scales (F16) and the factors of the drained sums
  ++g_launch_count, k_wscale<<<a.T, 256, 0, st>>>(a.Kpad, a.T, a.wtab, a.absmax, a.eB, a.scale, a.kind == 0 ? 1 : 0,
                                                   a.escale);
  Chi0Maps maps;
  const long long ldk = 2LL * a.Kpad;
  const CUtensorMapDataType dt = a.kind == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : a.kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int esz = a.kind == 2 ? 4 : 2;
  const int np = a.kind == 1 ? 3 : 2;
  for (int i = 0; i < np; ++i)
    if (!map2d(&maps.b[i], a.bpl[i], dt, esz, ldk, a.N, BNU / tp, err)) return GW_ERR_CUDA;
  if (!map2d(&maps.raw, a.raw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ldk, a.N, BMU, err)) return GW_ERR_CUDA;
  Chi0Params prm{};
  prm.N = a.N;
  prm.nst = nst;
  prm.seg = seg;
  prm.nchunk = P->nchunk;
  prm.tiles = P->d_tiles;
  prm.items = P->d_items;
  prm.cta_off = P->d_off;
  prm.T = a.T;
  prm.TG = (a.T + tp - 1) / tp;
  prm.wtab = a.wtab;
  prm.wstride = a.Kpad;
  prm.escale = a.escale;
  prm.out = reinterpret_cast<double*>(a.out);
  prm.status = a.status;
  prm.lower = 1;
  prm.a_bstride = 0;
  prm.b_bstride = 0;
  if (a.events) cudaEventRecord(a.events[0], st);
  if (a.kind == 0) s = launch_chi0<K_F16, TP_F16>(maps, prm, P->grid, st, err);
  else if (a.kind == 1) s = launch_chi0<K_BF16, 1>(maps, prm, P->grid, st, err);
  else s = launch_chi0<K_TF32, TP_TF32>(maps, prm, P->grid, st, err);
  if (s != GW_OK) return s;
  if (a.events) cudaEventRecord(a.events[1], st);
  return GW_OK;
}

// TF32 pieces of Hermitian matrices H (FP64 or FP32 complex, [rows][N]) as the B planes of the
// product kernel: row r, K index 2k + {0: re, 1: im}, zero for k >= N (padding to Kpad)
template <typename T>
__global__ void k_h_pieces_tf32(long long rows, int N, int Kpad, const cplx<T>* __restrict__ H, float* __restrict__ p0,
                                float* __restrict__ p1) {
  const long long total = rows * Kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / Kpad;
    const int k = (int)(e % Kpad);
    float xr = 0.f, xi = 0.f;
    if (k < N) {
      const cplx<T> v = H[r * N + k];
      xr = (float)v.re;
      xi = (float)v.im;
    }
    const float hr = tf32_rn(xr), hi = tf32_rn(xi);
    reinterpret_cast<float2*>(p0)[e] = make_float2(hr, hi);
    reinterpret_cast<float2*>(p1)[e] = make_float2(xr - hr, xi - hi);
  }
}

__global__ void k_fill_d(double* p, int n, double v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) p[e] = v;
}
__global__ void k_fill_f(float* p, int n, float v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) p[e] = v;
}

gw_status herm_gemm_run(const HermGemmArgs& a, Chi0Plan** plan, cudaStream_t st, std::string& err) {
  const int N = a.N, nb = a.nb;
  if (N < 2 || N % 2 != 0 || nb < 1) {
    err = "herm_gemm: N must be even and >= 2";
    return GW_ERR_ARG;
  }
  const int Kpad = (N + 31) / 32 * 32;
  const long long hrows = (long long)(a.h_batch ? nb : 1) * N;
  const int grid = (int)std::min<long long>((hrows * Kpad + 255) / 256, 152LL * 16);
  if (a.H64)
    ++g_launch_count, k_h_pieces_tf32<double><<<grid, 256, 0, st>>>(hrows, N, Kpad, a.H64, a.bpl[0], a.bpl[1]);
  else
    ++g_launch_count, k_h_pieces_tf32<float><<<grid, 256, 0, st>>>(hrows, N, Kpad, a.H32, a.bpl[0], a.bpl[1]);
  ++g_launch_count, k_fill_d<<<1, 256, 0, st>>>(a.escale, nb, a.alpha);
  ++g_launch_count, k_fill_f<<<(Kpad + 255) / 256, 256, 0, st>>>(a.ones, Kpad, 1.0f);
  const int RS = Kd<K_TF32, 1>::RS;
  const int nst = Kpad / RS;
  Chi0Lists* L = nullptr;
  gw_status s = chi0_lists(plan, N, nb, nst, nst, 1, st, &L, err, false);
  if (s != GW_OK) return s;
  Chi0Maps maps;
  for (int i = 0; i < 2; ++i)
    if (!map2d(&maps.b[i], a.bpl[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2LL * Kpad, hrows, BNU, err))
      return GW_ERR_CUDA;
  const long long arows = (long long)(a.a_batch ? nb : 1) * N;
  if (!map2d(&maps.raw, a.A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2LL * N, arows, BMU, err)) return GW_ERR_CUDA;
  Chi0Params prm{};
  prm.N = N;
  prm.nst = nst;
  prm.seg = nst;
  prm.nchunk = L->nchunk;
  prm.tiles = L->d_tiles;
  prm.items = L->d_items;
  prm.cta_off = L->d_off;
  prm.T = nb;
  prm.TG = nb;
  prm.wtab = a.ones;
  prm.wstride = 0;
  prm.escale = a.escale;
  prm.out = reinterpret_cast<double*>(a.C);
  prm.status = a.status;
  prm.lower = 0;
  prm.store = 1;   // one K chunk (nchunk = 1) and one segment per item: every element written once
  if (L->nchunk != 1) {
    err = "herm_gemm: the product needs one K chunk per output tile";
    return GW_ERR_STATE;
  }
  prm.a_bstride = a.a_batch ? N : 0;
  prm.b_bstride = a.h_batch ? N : 0;
  return launch_chi0<K_TF32, 1>(maps, prm, L->grid, st, err);
}

void chi0h_weights(int K, int Kpad, int nw, const float* delta, const double* freq, float* wtab, cudaStream_t st) {
  const long long total = (long long)nw * Kpad;
  ++g_launch_count, k_weights_h<<<(int)std::min<long long>((total + 255) / 256, 152LL * 32), 256, 0, st>>>(
      K, Kpad, nw, delta, freq, wtab);
}

}  // namespace gw
