// Tensor-core (tcgen05) split-precision complex contractions of the G0W0 hot path.
//
// One persistent kernel, two modes, both of the form  out_{m n} = sum_r y^m_r conj(b^n_r)  with
//   y^m_r = w(r) x^m_r  (A side: rows of an fp32 plane, weight fused into the operand load)
//   b^n_r               (B side: split planes streamed by TMA)
// and every operand row interleaving (re, im) along K. Real form:
//   Re out = sum_r (y_re b_re + y_im b_im) = A . B1^T,  B1 = (b_re,  b_im),
//   Im out = sum_r (y_im b_re - y_re b_im) = A . B2^T,  B2 = (-b_im, b_re),
// so one MMA against the stacked operand [B1; B2] (N = 2 x 64) yields Re and Im columns.
//
// MODE 0, step (b), Eq. chi0_matrix (Hermitised, occupations restored):
//   chi0_{mu nu}(w) = scale * sum_r w_w(D_r) M^mu_r conj(M^nu_r),  w_w(D) = 2 D / (w^2 + D^2),
//   r = (k, i occ, a unocc); lower tiles only, FP64 accumulation into chi0[w].
// MODE 1, step (d), Eq. GW_selfe_element with W^c:
//   U_{r nu} = sum_mu a_{r mu} W^c_{mu nu}(w') = sum_mu a_{r mu} conj(W^c_{nu mu})  (W^c Hermitian),
//   S_r(w') = Re sum_nu U_{r nu} conj(a_{r nu}),  a_r = C^mu_{nm}(k, k-q);  the row dot is
//   fused into the epilogue and accumulated into S[r][w'].
//
// Operands are split into pieces (BF16: h + m + l, TF32: h + l); the products of combined
// order >= 2^-16 (BF16: hh, hm, mh, hl, lh, mm) or 2^-11 (TF32: hh, hl, lh) are accumulated.
//
// Accumulation. The tensor-core FP32 accumulator rounds every addition toward zero, which
// biases a long sum by ~3e-8 relative per accumulation. So:
//   * hh goes to accumulator D1, which is drained after every stage (4 MMAs per output)
//     into FP32 running sums held in registers by the epilogue warps (round to nearest);
//     MODE 1 sums only K = n_aux (at most 52 MMAs per item), so there D1 is drained once per
//     segment like D2 (the truncation bias stays ~1e-6 relative of S, far inside the Sigma_c tolerance);
//   * the correction products (2^-8 smaller) go to D2, drained once per segment;
//   * after each segment the running sums are added in FP64 into the output (MODE 0), or
//     dotted with a and added to S (MODE 1, one segment per work item).
//
// Work distribution: one CTA per SM, each walking a static list of work items (output tile,
// frequency); all pipelines (barrier phases, TMEM buffers) run on across items. Item order
// keeps the data of concurrently running CTAs shared in L2 (MODE 0: frequency fastest; MODE 1:
// column block fastest, then frequency, then row block).
//
// Roles (480 threads):
//   * warp 0 (TMA):   B1 / B2 pieces, 64 rows x 128 B each per stage, SWIZZLE_128B
//   * warp 14 (TMA):  A rows of the fp32 plane, 128 rows x 128 B per slot, into a ring that runs
//                     ahead of the transform, each slot with its 16 weights (bulk copy);
//                     PRE: the pre-split A pieces into the stages, and after each item's stages
//                     the item's fp32 a tile (128 rows x BN complex) into the idle ring for the
//                     epilogue's row dot
//   * warps 2-5:      transform (not PRE): rebuild y = w x from the ring, split, write the A
//                     pieces in the UMMA K-major 128B-swizzled layout
//   * warp 1:         one elected thread issues tcgen05.mma (M = 128, N = 128) into TMEM
//   * warps 6-13:     epilogue (two warps per TMEM lane quadrant, 32 complex columns each)
// All mbarrier waits are bounded; on expiry the kernel sets ST_TIMEOUT and unwinds.
#include "gw_internal.h"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <vector>

namespace gw {

namespace {

using namespace ptx;

constexpr int BM = 128, BN = 64;                   // complex output tile
constexpr int TILE = 128 * ROWB;                   // 16 KB: A piece (128 rows) or B piece ([B1; B2], 128 rows)
constexpr int HALF = 64 * ROWB;                    // 8 KB: B1 or B2 part of a B piece
constexpr int RAW = 128 * ROWB;                    // 16 KB: one ring slot = 16 complex pairs of 128 A rows
constexpr int RAW_BOXES = 2 * BN / 32;             // fp32 boxes (32 floats x 128 rows) of one BN-column a tile
constexpr int WBYTES = 16 * 4;                     // weights of the 16 pair rows of one ring slot
constexpr int NTHREADS = 480;
constexpr int MAX_TILES = 8192;
// TMEM columns: D1 buffers at 0 and 128 (re: +0..63, im: +64..127); D2 buffers at 256 and 384
constexpr uint32_t D1_COL = 0, D2_COL = 256, DBUF = 128;

template <bool TF32, int NP_> struct Cfg {
  static constexpr int NP = NP_;                   // pieces per operand (TF32: 2; BF16: 2 or 3)
  static constexpr int STAGE = 2 * NP * TILE;      // B pieces then A pieces
  static constexpr int STAGES = 2;
  static constexpr int RPS = TF32 ? 1 : 2;         // ring slots per stage
  static constexpr int RING = (NP_ == 3) ? 2 : 4;  // ring slots
  static constexpr int RS = 16 * RPS;              // complex pair rows per stage
  static constexpr int WB_OFF = STAGES * STAGE + RING * RAW;   // the 16 weights of each ring slot
  static constexpr int BAR_OFF = WB_OFF + RING * WBYTES;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;
};
static_assert(Cfg<false, 3>::SMEM <= 232448, "shared memory budget");
static_assert(Cfg<false, 2>::SMEM <= 232448, "shared memory budget");
static_assert(Cfg<true, 2>::SMEM <= 232448, "shared memory budget");

// sr[j] += D[re column t + j], si[j] += D[im column t + BN + j], j < 32, sixteen columns at a time
// (keeps the running sums and one half of the drained columns in registers)
__device__ __forceinline__ void drain_add(uint32_t t, float (&sr)[32], float (&si)[32]) {
  uint32_t vr[16], vi[16], wr[16], wi[16];
  tmem_ld16_nowait(t, vr);
  tmem_ld16_nowait(t + BN, vi);
  tmem_ld16_nowait(t + 16, wr);
  tmem_ld16_nowait(t + BN + 16, wi);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    sr[j] += __uint_as_float(vr[j]);
    si[j] += __uint_as_float(vi[j]);
    sr[16 + j] += __uint_as_float(wr[j]);
    si[16 + j] += __uint_as_float(wi[j]);
  }
}


struct TcParams {
  int Mrows, Ncols;   // A rows (mu or r), B rows (nu)
  int nstage, seg;    // stages per work item; stages per promotion segment
  int n_items, nw, nnb;
  const short2* tiles;  // MODE 0: (m0 / BM, n0 / BN) per tile; work item = tile * nw + w
  const float* raw;   // [Mrows][ldk] fp32 (re, im) plane of the A side (for the MODE 1 row dot)
  long long ldk;      // floats per raw row
  const float* wtab;  // weights: wtab[w * wstride + r]
  long long wstride;
  int brow_y;         // B row offset per frequency (MODE 1: one W^c per frequency)
  double scale;
  c128* out;          // MODE 0: [nw][Ncols][Ncols]
  float* S;           // MODE 1: [Mrows][nw]
  int* status;
  int tri;            // MODE 1: use the Hermitian triangle of W^c
};

struct Maps {
  CUtensorMap b[6];   // B1 pieces then B2 pieces
  CUtensorMap raw;    // A-side fp32 plane, 32 floats x 128 rows per box
  CUtensorMap a[3];   // PRE: A-side pieces, split before the launch (128 B x 128 rows per box)
};

template <int MODE>
__device__ __forceinline__ void decode_item(const TcParams& p, int item, int& m0, int& n0, int& w) {
  if constexpr (MODE == 0) {
    const short2 t = p.tiles[item / p.nw];
    w = item % p.nw;
    m0 = t.x * BM;
    n0 = t.y * BN;
  } else {
    const int nb = item % p.nnb;
    const int rest = item / p.nnb;
    w = rest % p.nw;
    m0 = (rest / p.nw) * BM;
    n0 = nb * BN;
  }
}


// MODE 1 with `tri`: W^c is Hermitian, so column block nb needs K = mu from its own block on;
// the block's own 64 ABFs form one segment (counted once), the rest a second one (counted twice).
template <int MODE, int RS>
__device__ __forceinline__ int first_stage(const TcParams& p, int n0) {
  return (MODE == 1 && p.tri) ? n0 / RS : 0;
}
template <int MODE, int RS>
__device__ __forceinline__ bool is_seg_first(const TcParams& p, int i, int i0, int F) {
  if (MODE == 1 && p.tri) return i == i0 || i == i0 + BN / RS;
  return (i % F) == 0;
}
template <int MODE, int RS>
__device__ __forceinline__ bool is_seg_end(const TcParams& p, int i, int i0, int F, int nst) {
  if (MODE == 1 && p.tri) return i == nst - 1 || i == i0 + BN / RS - 1;
  return (i % F) == F - 1 || i == nst - 1;
}

template <bool TF32, int NPC, int MODE, bool PRE>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc(const __grid_constant__ Maps maps, TcParams p) {
  using C = Cfg<TF32, NPC>;
  constexpr int NP = C::NP, STAGES = C::STAGES, STAGE = C::STAGE, RS = C::RS, RPS = C::RPS, RING = C::RING;
  static_assert(!(MODE == 1 && PRE) || RING >= RAW_BOXES, "the a tile of the row dot must fit in the ring");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem + STAGES * STAGE;
  float* wbuf = reinterpret_cast<float*>(smem + C::WB_OFF);   // [RING][16]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  uint64_t* full_b = bars;                   // [STAGES]
  uint64_t* full_a = bars + STAGES;          // [STAGES]
  uint64_t* empty = bars + 2 * STAGES;       // [STAGES]
  uint64_t* t1full = bars + 3 * STAGES;      // [2] D1 of a stage ready
  uint64_t* t1empty = bars + 3 * STAGES + 2; // [2] D1 drained
  uint64_t* t2full = bars + 3 * STAGES + 4;  // [2] D2 of a segment ready
  uint64_t* t2empty = bars + 3 * STAGES + 6; // [2] D2 drained
  uint64_t* done = bars + 3 * STAGES + 8;
  uint64_t* rfull = bars + 3 * STAGES + 9;           // [RING]
  uint64_t* rempty = bars + 3 * STAGES + 9 + RING;   // [RING]
  uint32_t* tmem_base_p = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 9 + 2 * RING);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&full_a[s], PRE ? 1 : 4);       // one elected arrival per transform warp
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t1full[b], 1);
      mbar_init(&t1empty[b], 8);                // one per epilogue warp
      mbar_init(&t2full[b], 1);
      mbar_init(&t2empty[b], 8);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(&rfull[r], 1);
      mbar_init(&rempty[r], PRE ? 8 : 4);        // PRE: the a tile of the row dot, read by the epilogue
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
  const int nst = p.nstage;
  const int F = p.seg;

  if (warp == 0) {
    // ---------------- TMA producer: B1 / B2 pieces ----------------
    if (lane == 0) {
      uint32_t gs = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item<MODE>(p, item, m0, n0, w);
        const int yrow = w * p.brow_y + n0;
        for (int i = first_stage<MODE, RS>(p, n0); i < nst; ++i, ++gs) {
          const int s = gs % STAGES;
          if (!mbar_wait(&empty[s], ((gs / STAGES) & 1) ^ 1, p.status)) { ok = false; break; }
          uint8_t* st = smem + s * STAGE;
          mbar_arrive_expect_tx(&full_b[s], NP * TILE);
          const int x = i * (ROWB / (TF32 ? 4 : 2));
#pragma unroll
          for (int pc = 0; pc < NP; ++pc) {
            tma_load_2d(st + pc * TILE, &maps.b[pc], &full_b[s], x, yrow);              // B1 rows 0..63
            tma_load_2d(st + pc * TILE + HALF, &maps.b[NP + pc], &full_b[s], x, yrow);  // B2 rows 64..127
          }
        }
      }
    }
  } else if (warp == 14 && PRE) {
    // ---------------- TMA producer: A pieces (split before the launch) into the stages ----------------
    if (lane == 0) {
      uint32_t gs = 0, gt = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item<MODE>(p, item, m0, n0, w);
        for (int i = first_stage<MODE, RS>(p, n0); i < nst; ++i, ++gs) {
          const int s = gs % STAGES;
          if (!mbar_wait(&empty[s], ((gs / STAGES) & 1) ^ 1, p.status)) { ok = false; break; }
          uint8_t* at = smem + s * STAGE + NP * TILE;
          mbar_arrive_expect_tx(&full_a[s], NP * TILE);
          const int x = i * (ROWB / (TF32 ? 4 : 2));
#pragma unroll
          for (int pc = 0; pc < NP; ++pc) tma_load_2d(at + pc * TILE, &maps.a[pc], &full_a[s], x, m0);
        }
        if (MODE == 1 && ok) {
          // the fp32 a tile of the epilogue's row dot (rows m0.., columns n0..n0+BN-1) into the ring:
          // RAW_BOXES boxes of 32 floats x 128 rows; issued after the item's stages, since it is read
          // only at the item's end, once the previous item's epilogue has released it
          const uint32_t par = (gt & 1) ^ 1;
          if (!mbar_wait(&rempty[0], par, p.status)) break;
          mbar_arrive_expect_tx(&rfull[0], RAW_BOXES * RAW);
#pragma unroll
          for (int c = 0; c < RAW_BOXES; ++c) tma_load_2d(ring + c * RAW, &maps.raw, &rfull[0], 2 * n0 + 32 * c, m0);
          ++gt;
        }
      }
    }
  } else if (warp == 14) {
    // ---------------- TMA producer: A rows of the fp32 plane and their weights into the ring ----------------
    if (lane == 0) {
      uint32_t gr = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item<MODE>(p, item, m0, n0, w);
        const float* wrow = p.wtab + (long long)w * p.wstride;
        for (int i = first_stage<MODE, RS>(p, n0) * RPS; i < nst * RPS; ++i, ++gr) {
          const int slot = gr % RING;
          if (!mbar_wait(&rempty[slot], ((gr / RING) & 1) ^ 1, p.status)) { ok = false; break; }
          mbar_arrive_expect_tx(&rfull[slot], RAW + WBYTES);
          tma_load_2d(ring + slot * RAW, &maps.raw, &rfull[slot], i * 32, m0);
          // pair rows 16 i .. 16 i + 15 (16-byte aligned: the weight rows are Kpad = 0 mod 32 floats apart)
          bulk_load(wbuf + slot * 16, wrow + 16 * i, WBYTES, &rfull[slot]);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t fmt = TF32 ? 2u : 1u;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)((2 * BN) >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);
      uint32_t gs = 0, gseg = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item<MODE>(p, item, m0, n0, w);
        const int i0 = first_stage<MODE, RS>(p, n0);
        for (int i = i0; i < nst; ++i, ++gs) {
          const int s = gs % STAGES;
          const int b2 = gseg & 1;
          // MODE 0 drains D1 after every stage; MODE 1 (K <= n_aux) once per segment, like D2
          const int b = (MODE == 0) ? (gs & 1) : b2;
          const bool seg_first = is_seg_first<MODE, RS>(p, i, i0, F);
          if constexpr (MODE == 0) {
            if (gs >= 2 && !mbar_wait(&t1empty[b], ((gs >> 1) - 1) & 1, p.status)) { ok = false; break; }
          } else {
            if (seg_first && gseg >= 2 && !mbar_wait(&t1empty[b], ((gseg >> 1) - 1) & 1, p.status)) {
              ok = false;
              break;
            }
          }
          if (seg_first && gseg >= 2 && !mbar_wait(&t2empty[b2], ((gseg >> 1) - 1) & 1, p.status)) {
            ok = false;
            break;
          }
          if (!mbar_wait(&full_b[s], (gs / STAGES) & 1, p.status)) { ok = false; break; }
          if (!mbar_wait(&full_a[s], (gs / STAGES) & 1, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t bbase = smem_u32(smem + s * STAGE);
          const uint32_t abase = bbase + NP * TILE;
          const uint32_t d1 = tmem + D1_COL + b * DBUF;
          const uint32_t d2 = tmem + D2_COL + b2 * DBUF;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t ko = kk * 32;
            const uint32_t acc1 = (MODE == 0) ? (kk == 0 ? 0u : 1u) : ((seg_first && kk == 0) ? 0u : 1u);
            const uint32_t acc2 = (seg_first && kk == 0) ? 0u : 1u;
            const uint64_t A0 = sdesc(abase + ko), B0 = sdesc(bbase + ko);
            const uint64_t A1 = sdesc(abase + TILE + ko), B1 = sdesc(bbase + TILE + ko);
            mma<TF32>(d1, A0, B0, idesc, acc1);
            mma<TF32>(d2, A0, B1, idesc, acc2);
            mma<TF32>(d2, A1, B0, idesc, 1u);
            if constexpr (NP == 3) {
              const uint64_t A2 = sdesc(abase + 2 * TILE + ko), B2 = sdesc(bbase + 2 * TILE + ko);
              mma<TF32>(d2, A0, B2, idesc, 1u);
              mma<TF32>(d2, A2, B0, idesc, 1u);
              mma<TF32>(d2, A1, B1, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
          if constexpr (MODE == 0) mma_commit(&t1full[b]);
          if (is_seg_end<MODE, RS>(p, i, i0, F, nst)) {
            if constexpr (MODE == 1) mma_commit(&t1full[b]);
            mma_commit(&t2full[b2]);
            ++gseg;
          }
        }
      }
      mma_commit(done);
      mbar_wait(done, 0, p.status);
    }
  } else if (warp >= 2 && warp <= 5 && !PRE) {
    // ---------------- transform: weighted, split A operand ----------------
    const int row = threadIdx.x - 64;          // 0..127
    uint32_t gs = 0, gr = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
      int m0, n0, w;
      decode_item<MODE>(p, item, m0, n0, w);
      for (int i = first_stage<MODE, RS>(p, n0); i < nst; ++i, ++gs) {
        const int s = gs % STAGES;
        // warp-uniform waits: the arrivals below are elected per warp
        if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ((gs / STAGES) & 1) ^ 1, p.status))) { ok = false; break; }
        uint8_t* at = smem + s * STAGE + NP * TILE;
        for (int h = 0; h < RPS; ++h, ++gr) {
          const int slot = gr % RING;
          if (!__all_sync(0xffffffffu, mbar_wait(&rfull[slot], (gr / RING) & 1, p.status))) { ok = false; break; }
          // the 16 weights of this slot's pair rows (delivered with the slot; broadcast reads)
          float wv[16];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 v = reinterpret_cast<const float4*>(wbuf + slot * 16)[c];
            wv[4 * c] = v.x;
            wv[4 * c + 1] = v.y;
            wv[4 * c + 2] = v.z;
            wv[4 * c + 3] = v.w;
          }
          // this thread's row: 16 complex pairs (8 chunks of 16 B, 128B-swizzled by TMA)
          float x[32];
          const uint8_t* rs = ring + slot * RAW;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(rs + swz(row, c));
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
          // order these generic-proxy reads before the TMA (async-proxy) refill of the slot
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&rempty[slot]);
          if constexpr (TF32) {
            // A row = 16 pairs = 8 chunks of 2 pairs
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              uint32_t o0[4], o1[4];
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const float wt = wv[2 * c + q];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  const float y = wt * x[4 * c + 2 * q + e];
                  const float hh = tf32_rn(y);
                  o0[2 * q + e] = __float_as_uint(hh);
                  o1[2 * q + e] = __float_as_uint(y - hh);
                }
              }
              const uint32_t off = swz(row, c);
              *reinterpret_cast<uint4*>(at + off) = make_uint4(o0[0], o0[1], o0[2], o0[3]);
              *reinterpret_cast<uint4*>(at + TILE + off) = make_uint4(o1[0], o1[1], o1[2], o1[3]);
            }
          } else {
            // A row = 32 pairs = 8 chunks of 4 pairs; this slot fills chunks 4h .. 4h+3
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              uint32_t o[NP][4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int pr = 4 * cc + q;     // pair within the slot
                const float wt = wv[pr];
                const float yr = wt * x[2 * pr], yi = wt * x[2 * pr + 1];
                const __nv_bfloat162 hh = __floats2bfloat162_rn(yr, yi);
                const float2 hf = __bfloat1622float2(hh);
                const float rr = yr - hf.x, ri = yi - hf.y;
                const __nv_bfloat162 mm = __floats2bfloat162_rn(rr, ri);
                const float2 mf = __bfloat1622float2(mm);
                const __nv_bfloat162 ll = __floats2bfloat162_rn(rr - mf.x, ri - mf.y);
                o[0][q] = bf2_bits(hh);
                if constexpr (NP == 3) {
                  o[1][q] = bf2_bits(mm);
                  o[2][q] = bf2_bits(ll);
                } else {
                  o[1][q] = bf2_bits(__floats2bfloat162_rn(rr, ri));
                }
              }
              const uint32_t off = swz(row, 4 * h + cc);
#pragma unroll
              for (int pc = 0; pc < NP; ++pc)
                *reinterpret_cast<uint4*>(at + pc * TILE + off) = make_uint4(o[pc][0], o[pc][1], o[pc][2], o[pc][3]);
            }
          }
        }
        if (!ok) break;
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_a[s]);
      }
    }
  } else if (warp >= 6 && warp <= 13) {
    // ---------------- epilogue: drain D1 per stage, D2 per segment, flush ----------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
    const int half = (warp - 6) >> 2;          // output columns half*32 .. half*32+31
    const int row = quad * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    uint32_t gs = 0, gseg = 0, gt = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
      int m0, n0, w;
      decode_item<MODE>(p, item, m0, n0, w);
      const int m = m0 + row;
      const int c0 = n0 + half * 32;
      bool tile_ready = false;                 // MODE 1, PRE: the a tile of this item has landed
      float sr[32], si[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) sr[j] = si[j] = 0.f;
      for (int i = first_stage<MODE, RS>(p, n0); i < nst; ++i, ++gs) {
        const bool seg_end = is_seg_end<MODE, RS>(p, i, first_stage<MODE, RS>(p, n0), F, nst);
        if (MODE == 0 || seg_end) {
          const int b = (MODE == 0) ? (gs & 1) : (gseg & 1);
          const uint32_t ph = (MODE == 0) ? ((gs >> 1) & 1) : ((gseg >> 1) & 1);
          // every lane polls the barrier; reconverge before the warp-wide (.sync.aligned) TMEM loads
          ok = __all_sync(0xffffffffu, mbar_wait(&t1full[b], ph, p.status));
          if (!ok) break;
          tc_fence_after();
          drain_add(tmem + lane_off + D1_COL + b * DBUF + half * 32, sr, si);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&t1empty[b]);
        }
        if (seg_end) {
          const int b2 = gseg & 1;
          ok = __all_sync(0xffffffffu, mbar_wait(&t2full[b2], (gseg >> 1) & 1, p.status));
          if (!ok) break;
          tc_fence_after();
          drain_add(tmem + lane_off + D2_COL + b2 * DBUF + half * 32, sr, si);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&t2empty[b2]);
          ++gseg;
          const int nmax = p.Ncols - c0;
          if (MODE == 1 && PRE && !tile_ready) {
            ok = __all_sync(0xffffffffu, mbar_wait(&rfull[0], gt & 1, p.status));
            if (!ok) break;
            tile_ready = true;
          }
          if (m < p.Mrows) {
            if constexpr (MODE == 0) {
              c128* orow = p.out + ((long long)w * p.Ncols + m) * p.Ncols + c0;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                if (j < nmax) {
                  c128 o = orow[j];
                  o.re += p.scale * (double)sr[j];
                  o.im += p.scale * (double)si[j];
                  orow[j] = o;
                }
              }
            } else if constexpr (PRE) {
              // S_r += Re sum_nu U_{r nu} conj(a_{r nu}) over this thread's 32 columns, a from the
              // ring tile (complex column 32 half + j: box 2 half + j / 16, 16-B chunk (j % 16) / 2)
              float acc = 0.f;
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const float4 a = *reinterpret_cast<const float4*>(ring + (2 * half + jj / 8) * RAW + swz(row, jj % 8));
                if (2 * jj < nmax) acc = fmaf(sr[2 * jj], a.x, fmaf(si[2 * jj], a.y, acc));
                if (2 * jj + 1 < nmax) acc = fmaf(sr[2 * jj + 1], a.z, fmaf(si[2 * jj + 1], a.w, acc));
              }
              const float wgt = (p.tri && i > first_stage<MODE, RS>(p, n0) + (BN / RS) - 1) ? 2.f : 1.f;
              atomicAdd(p.S + (long long)m * p.nw + w, wgt * acc);
            } else {
              // S_r += Re sum_nu U_{r nu} conj(a_{r nu}) over this thread's 32 columns
              const float* arow = p.raw + (long long)m * p.ldk + 2LL * c0;
              float acc = 0.f;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                if (j < nmax) {
                  const float2 a = *reinterpret_cast<const float2*>(arow + 2 * j);
                  acc = fmaf(sr[j], a.x, fmaf(si[j], a.y, acc));
                }
              }
              // triangle: the diagonal block counts once, the strictly lower blocks twice (2 Re)
              const float wgt = (p.tri && i > first_stage<MODE, RS>(p, n0) + (BN / RS) - 1) ? 2.f : 1.f;
              atomicAdd(p.S + (long long)m * p.nw + w, wgt * acc);
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) sr[j] = si[j] = 0.f;
          if (MODE == 1 && PRE && i == nst - 1) {
            // last segment of the item: release the a tile (generic reads before the TMA refill)
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&rempty[0]);
            ++gt;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// w_w(D_r) = 2 D / (w^2 + D^2) for every frequency and pair row (0 for padding rows)
__global__ void k_weights(int Kpad, int nw, const float* __restrict__ delta, const double* __restrict__ freq,
                          float* __restrict__ wtab) {
  const long long total = (long long)nw * Kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % Kpad), j = (int)(e / Kpad);
    const float d = delta[r];
    const float w = (float)freq[j];
    wtab[e] = 2.0f * d / (w * w + d * d);
  }
}

// chi0[w][i][j] = conj(chi0[w][j][i]) for i < j (the kernel writes lower tiles only)
__global__ void k_herm_fill(int N, int nw, c128* chi0) {
  const long long total = (long long)nw * N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % N), i = (int)((e / N) % N);
    const long long w = e / ((long long)N * N);
    if (i < j) {
      const c128 v = chi0[(w * N + j) * N + i];
      chi0[(w * N + i) * N + j] = c128{v.re, -v.im};
    }
  }
}

// A pieces of an fp32 (re, im) plane [rows][ldk] for the pre-split path, two pieces:
// BF16: h = bf16(y), l = bf16(y - h);  TF32: h = tf32(y), l = y - h (read as TF32 by the MMA).
__global__ void k_a_planes(long long n, const float* __restrict__ raw, void* p0, void* p1, int tf32) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 y = reinterpret_cast<const float2*>(raw)[e];
    if (tf32) {
      const float hr = tf32_rn(y.x), hi = tf32_rn(y.y);
      reinterpret_cast<float2*>(p0)[e] = make_float2(hr, hi);
      reinterpret_cast<float2*>(p1)[e] = make_float2(y.x - hr, y.y - hi);
    } else {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(y.x, y.y);
      const float2 hf = __bfloat1622float2(hh);
      reinterpret_cast<__nv_bfloat162*>(p0)[e] = hh;
      reinterpret_cast<__nv_bfloat162*>(p1)[e] = __floats2bfloat162_rn(y.x - hf.x, y.y - hf.y);
    }
  }
}

// B planes of W^c (conj: of conj(W^c)) for the Sigma contraction: row (j, nu), K index 2 mu + {0, 1}:
// B1 = split(Re W_{nu mu}, Im W_{nu mu}), B2 = split(-Im, Re); mu >= N is zero padding.
__global__ void k_w_planes(int N, int nw, int Kpad, const c128* __restrict__ Wc, PlaneSet P, int tf32, int np,
                           int conj) {
  const long long total = (long long)nw * N * Kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(e % Kpad);
    const long long row = e / Kpad;                 // j * N + nu
    float v1[2] = {0.f, 0.f};
    if (mu < N) {
      const c128 w = Wc[row * N + mu];
      v1[0] = (float)w.re;
      v1[1] = conj ? -(float)w.im : (float)w.im;
    }
    const float v2[2] = {-v1[1], v1[0]};
    const long long o = row * 2LL * Kpad + 2LL * mu;
    for (int half = 0; half < 2; ++half) {
      const float* v = half ? v2 : v1;
      if (tf32) {
        const float h0 = tf32_rn(v[0]), h1 = tf32_rn(v[1]);
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.b[2 * half]) + o) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.b[2 * half + 1]) + o) = make_float2(v[0] - h0, v[1] - h1);
      } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
        const float2 hf = __bfloat1622float2(h);
        const float r0 = v[0] - hf.x, r1 = v[1] - hf.y;
        const __nv_bfloat162 mm = __floats2bfloat162_rn(r0, r1);
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[np * half]) + o) = h;
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[np * half + 1]) + o) = mm;
        if (np == 3) {
          const float2 mf = __bfloat1622float2(mm);
          const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[np * half + 2]) + o) = l;
        }
      }
    }
  }
}

__global__ void k_fill(float* p, long long n, float v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    p[e] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map over a row-major plane [rows][ldk] of 16-bit (bf16) or 32-bit (fp32/tf32) elements,
// box = 128 B of one row x box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int four_byte, long long ldk, long long rows, int box_rows,
              std::string& err) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    err = "cuTensorMapEncodeTiled is unavailable";
    return false;
  }
  const int esz = four_byte ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ldk * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, four_byte ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

template <bool TF32, int NPC, int MODE, bool PRE = false>
gw_status launch_tc(const Maps& maps, const TcParams& p, cudaStream_t st, std::string& err) {
  const int smem = Cfg<TF32, NPC>::SMEM;
  cudaFuncSetAttribute(k_tc<TF32, NPC, MODE, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int grid = std::min(p.n_items, num_sms());
  ++::gw::g_launch_count, k_tc<TF32, NPC, MODE, PRE><<<grid, NTHREADS, smem, st>>>(maps, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("k_tc launch: ") + cudaGetErrorString(e);
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace

bool tc_available() { return get_encode() != nullptr; }

TcWorkspace::~TcWorkspace() {
  if (tiles) cudaFree(tiles);
  if (ones) cudaFree(ones);
}

gw_status TcWorkspace::ensure(int ntiles_needed, int ones_needed, cudaStream_t st, std::string& err) {
  if (ntiles_needed > tile_cap) {
    if (tiles) cudaFree(tiles);
    tiles = nullptr;
    ++::gw::g_alloc_count;
    if (cudaMalloc(&tiles, sizeof(short2) * ntiles_needed) != cudaSuccess) {
      err = "tile table allocation failed";
      tile_cap = 0;
      return GW_ERR_NOMEM;
    }
    tile_cap = ntiles_needed;
  }
  if (ones_needed > ones_cap) {
    if (ones) cudaFree(ones);
    ones = nullptr;
    ++::gw::g_alloc_count;
    if (cudaMalloc(&ones, sizeof(float) * ones_needed) != cudaSuccess) {
      err = "weight table allocation failed";
      ones_cap = 0;
      return GW_ERR_NOMEM;
    }
    ++::gw::g_launch_count, k_fill<<<std::min(((long long)ones_needed + 255) / 256, 1024LL), 256, 0, st>>>(ones, ones_needed, 1.0f);
    ones_cap = ones_needed;
  }
  return GW_OK;
}

gw_status tc_chi0_run(const TcChi0Args& a, TcWorkspace& ws, cudaStream_t st, std::string& err) {
  const bool tf32 = a.tf32 != 0;
  const int RS = tf32 ? Cfg<true, 2>::RS : Cfg<false, 3>::RS;
  const int NP = tf32 ? 2 : 3;
  if (a.Kpad % 32 != 0 || a.N < 1) {
    err = "tc_chi0: Kpad must be a multiple of 32";
    return GW_ERR_ARG;
  }
  // lower-triangle tiles: every (mb, nb) with some nu <= mu inside
  std::vector<short2> tiles;
  const int nmb = (a.N + BM - 1) / BM, nnb = (a.N + BN - 1) / BN;
  for (int mb = 0; mb < nmb; ++mb)
    for (int nb = 0; nb < nnb; ++nb)
      if (nb * BN <= std::min(a.N, (mb + 1) * BM) - 1) tiles.push_back(make_short2((short)mb, (short)nb));
  const int nt = (int)tiles.size();
  if (nt > MAX_TILES) {
    err = "tc_chi0: n_aux too large for the tile table";
    return GW_ERR_ARG;
  }
  gw_status s = ws.ensure(std::max(nt, MAX_TILES / 8), 1, st, err);
  if (s != GW_OK) return s;
  Maps maps;
  const long long ldk = 2LL * a.Kpad;
  for (int i = 0; i < 2 * NP; ++i)
    if (!make_map(&maps.b[i], a.bpl[i], tf32, ldk, a.N, BN, err)) return GW_ERR_CUDA;
  if (!make_map(&maps.raw, a.raw, 1, ldk, a.N, BM, err)) return GW_ERR_CUDA;
  cudaError_t e = cudaMemcpyAsync(ws.tiles, tiles.data(), nt * sizeof(short2), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    err = std::string("tc_chi0 tile table: ") + cudaGetErrorString(e);
    return GW_ERR_CUDA;
  }
  if (!a.wtab_ready)
    ++::gw::g_launch_count, k_weights<<<std::min<long long>(((long long)a.nw * a.Kpad + 255) / 256, 152 * 32), 256, 0, st>>>(
        a.Kpad, a.nw, a.delta, a.freq, a.wtab);
  TcParams p{};
  p.Mrows = a.N;
  p.Ncols = a.N;
  p.nstage = a.Kpad / RS;
  p.seg = std::max(1, a.seg_rows / RS);
  p.n_items = nt * a.nw;
  p.nw = a.nw;
  p.nnb = nnb;
  p.tiles = ws.tiles;
  p.raw = a.raw;
  p.ldk = ldk;
  p.wtab = a.wtab;
  p.wstride = a.Kpad;
  p.brow_y = 0;
  p.scale = a.scale;
  p.out = a.chi0;
  p.status = a.status;
  return tf32 ? launch_tc<true, 2, 0>(maps, p, st, err) : launch_tc<false, 3, 0>(maps, p, st, err);
}

gw_status tc_sigma_run(const TcSigmaArgs& a, TcWorkspace& ws, cudaStream_t st, std::string& err) {
  const bool tf32 = a.tf32 != 0;
  // Sigma_c needs ~1e-5 relative accuracy: two pieces per operand (hh, hl, lh) in both kinds
  const int RS = tf32 ? Cfg<true, 2>::RS : Cfg<false, 2>::RS;
  const int NP = 2;
  if (a.Kpad % 32 != 0) {
    err = "tc_sigma: Kpad must be a multiple of 32";
    return GW_ERR_ARG;
  }
  const int nmb = (a.R + BM - 1) / BM, nnb = (a.N + BN - 1) / BN;
  const long long items = (long long)nmb * nnb * a.nw;
  if (items > 0x7fffffffLL) {
    err = "tc_sigma: too many work items";
    return GW_ERR_ARG;
  }
  gw_status s = ws.ensure(1, a.Kpad, st, err);
  if (s != GW_OK) return s;
  Maps maps;
  const long long ldk = 2LL * a.Kpad;
  for (int i = 0; i < 2 * NP; ++i)
    if (!make_map(&maps.b[i], a.bpl[i], tf32, ldk, (long long)a.nw * a.N, BN, err)) return GW_ERR_CUDA;
  if (!make_map(&maps.raw, a.raw, 1, ldk, a.R, BM, err)) return GW_ERR_CUDA;
  const bool pre = a.apl[0] != nullptr && a.apl[1] != nullptr;
  if (pre) {
    const long long n = (long long)a.R * a.Kpad;   // complex elements
    ++::gw::g_launch_count, k_a_planes<<<std::min<long long>((n + 255) / 256, 152 * 64), 256, 0, st>>>(
        n, a.raw, a.apl[0], a.apl[1], tf32 ? 1 : 0);
    for (int i = 0; i < NP; ++i)
      if (!make_map(&maps.a[i], a.apl[i], tf32, ldk, a.R, BM, err)) return GW_ERR_CUDA;
  }
  TcParams p{};
  p.Mrows = a.R;
  p.Ncols = a.N;
  p.nstage = a.Kpad / RS;
  p.seg = p.nstage;           // one segment per work item: K = n_aux is short
  p.n_items = (int)items;
  p.nw = a.nw;
  p.nnb = nnb;
  p.tiles = ws.tiles;
  p.raw = a.raw;
  p.ldk = ldk;
  p.wtab = ws.ones;
  p.wstride = 0;
  p.brow_y = a.N;
  p.scale = 1.0;
  p.S = a.S;
  p.tri = 1;
  p.status = a.status;
  if (pre) return tf32 ? launch_tc<true, 2, 1, true>(maps, p, st, err) : launch_tc<false, 2, 1, true>(maps, p, st, err);
  return tf32 ? launch_tc<true, 2, 1>(maps, p, st, err) : launch_tc<false, 2, 1>(maps, p, st, err);
}

void tc_w_planes(int N, int nw, int Kpad, const c128* Wc, const PlaneSet& P, int tf32, cudaStream_t st, int conj) {
  const long long total = (long long)nw * N * Kpad;
  ++::gw::g_launch_count, k_w_planes<<<std::min<long long>((total + 255) / 256, 152 * 64), 256, 0, st>>>(N, nw, Kpad, Wc, P, tf32, 2, conj);
}

void tc_herm_fill(int N, int nw, c128* chi0, cudaStream_t st) {
  const long long total = (long long)nw * N * N;
  ++::gw::g_launch_count, k_herm_fill<<<std::min<long long>((total + 255) / 256, 152 * 64), 256, 0, st>>>(N, nw, chi0);
}

}  // namespace gw
